// Fused stage kernel: degree 3, float fields, leapfrog E half step.
#define DGM_P 3
#define DGM_REAL float
#define DGM_MODE MODE_LF_E
#define DGM_LAUNCH launch_p3_f32_lfe
#include "dgm_kern_impl.cuh"
