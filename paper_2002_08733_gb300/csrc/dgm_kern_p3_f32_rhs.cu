// Fused stage kernel: degree 3, float fields, right-hand side only.
#define DGM_P 3
#define DGM_REAL float
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p3_f32_rhs
#include "dgm_kern_impl.cuh"
