// Fused stage kernel: degree 3, float fields, LSRK4 stage, tile variant 5:
// tensor-core variant (64 columns, 512 threads; curl and lift as TF32 split
// products on tcgen05).
#define DGM_P 3
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_TC 1
#define DGM_TE 64
#define DGM_NT 512
#define DGM_LAUNCH launch_p3_f32_lsrk_v5
#include "dgm_kern_impl.cuh"
