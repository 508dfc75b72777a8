// Fused stage kernel: degree 4, float fields, right-hand side only.
#define DGM_P 4
#define DGM_REAL float
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p4_f32_rhs
#include "dgm_kern_impl.cuh"
