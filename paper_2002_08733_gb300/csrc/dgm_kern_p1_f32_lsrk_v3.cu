// Paired stage kernel: degree 1, float fields, LSRK4 stage, tile variant 3
// (64 columns, two per thread, 384 threads per CTA, packed FP32x2 arithmetic).
#define DGM_P 1
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_PAIR F2x
#define DGM_TE 32
#define DGM_NT 384
#define DGM_LAUNCH launch_p1_f32_lsrk_v3
#include "dgm_kern_impl.cuh"
