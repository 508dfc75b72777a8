// Fused stage kernel: degree 3, double fields, right-hand side only.
#define DGM_P 3
#define DGM_REAL double
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p3_f64_rhs
#include "dgm_kern_impl.cuh"
