// Fused stage kernel: degree 5, float fields, LSRK4 stage, tile variant 3
// (32 columns x 512 threads: one CTA per SM at this degree, 16 warps).
#define DGM_P 5
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_TE 32
#define DGM_NT 512
#define DGM_LAUNCH launch_p5_f32_lsrk_v3
#include "dgm_kern_impl.cuh"
