// Fused stage kernel: degree 1, double fields, right-hand side only.
#define DGM_P 1
#define DGM_REAL double
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p1_f64_rhs
#include "dgm_kern_impl.cuh"
