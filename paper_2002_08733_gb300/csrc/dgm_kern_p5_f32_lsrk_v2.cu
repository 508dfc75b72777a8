// Fused stage kernel: degree 5, float fields, LSRK4 stage, tile variant 2
// (16 columns x 192 threads per CTA) for the autotuner.
#define DGM_P 5
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_TE 16
#define DGM_NT 192
#define DGM_LAUNCH launch_p5_f32_lsrk_v2
#include "dgm_kern_impl.cuh"
