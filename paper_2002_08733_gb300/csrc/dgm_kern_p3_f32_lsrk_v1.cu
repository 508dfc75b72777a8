// Fused stage kernel: degree 3, float fields, LSRK4 stage, tile variant 1
// (32 columns x 192 threads per CTA) for the autotuner.
#define DGM_P 3
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_TE 32
#define DGM_NT 192
#define DGM_LAUNCH launch_p3_f32_lsrk_v1
#include "dgm_kern_impl.cuh"
