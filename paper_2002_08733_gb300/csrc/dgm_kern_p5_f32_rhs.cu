// Fused stage kernel: degree 5, float fields, right-hand side only.
#define DGM_P 5
#define DGM_REAL float
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p5_f32_rhs
#include "dgm_kern_impl.cuh"
