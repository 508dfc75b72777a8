// Fused stage kernel: degree 1, float fields, LSRK4 stage.
#define DGM_P 1
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p1_f32_lsrk
#include "dgm_kern_impl.cuh"
