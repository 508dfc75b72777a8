// Fused stage kernel: degree 1, double fields, LSRK4 stage.
#define DGM_P 1
#define DGM_REAL double
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p1_f64_lsrk
#include "dgm_kern_impl.cuh"
