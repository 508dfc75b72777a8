// Fused stage kernel: degree 5, float fields, LSRK4 stage.
#define DGM_P 5
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_LAUNCH launch_p5_f32_lsrk
#include "dgm_kern_impl.cuh"
