// Paired stage kernel: degree 2, float fields, LSRK4 stage, tile variant 4
// (64 columns, two per thread, 384 threads per CTA, scalar arithmetic).
#define DGM_P 2
#define DGM_REAL float
#define DGM_MODE MODE_LSRK
#define DGM_PAIR P2
#define DGM_TE 32
#define DGM_NT 384
#define DGM_LAUNCH launch_p2_f32_lsrk_v4
#include "dgm_kern_impl.cuh"
