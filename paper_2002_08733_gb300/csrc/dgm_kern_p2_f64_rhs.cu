// Fused stage kernel: degree 2, double fields, right-hand side only.
#define DGM_P 2
#define DGM_REAL double
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p2_f64_rhs
#include "dgm_kern_impl.cuh"
