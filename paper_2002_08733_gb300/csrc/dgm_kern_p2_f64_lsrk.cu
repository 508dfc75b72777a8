// Fused stage kernel: degree 2, double fields, LSRK4 stage.
#define DGM_P 2
#define DGM_REAL double
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p2_f64_lsrk
#include "dgm_kern_impl.cuh"
