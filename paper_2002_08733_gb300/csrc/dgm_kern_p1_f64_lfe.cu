// Fused stage kernel: degree 1, double fields, leapfrog E half step.
#define DGM_P 1
#define DGM_REAL double
#define DGM_MODE MODE_LF_E
#define DGM_LAUNCH launch_p1_f64_lfe
#include "dgm_kern_impl.cuh"
