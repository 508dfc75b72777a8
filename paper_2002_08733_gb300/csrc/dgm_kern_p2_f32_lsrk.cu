// Fused stage kernel: degree 2, float fields, LSRK4 stage.
#define DGM_P 2
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p2_f32_lsrk
#include "dgm_kern_impl.cuh"
