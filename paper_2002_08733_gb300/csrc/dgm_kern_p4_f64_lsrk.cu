// Fused stage kernel: degree 4, double fields, LSRK4 stage.
#define DGM_P 4
#define DGM_REAL double
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p4_f64_lsrk
#include "dgm_kern_impl.cuh"
