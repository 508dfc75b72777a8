// Fused stage kernel: degree 4, double fields, right-hand side only.
#define DGM_P 4
#define DGM_REAL double
#define DGM_MODE MODE_RHS
#define DGM_LAUNCH launch_p4_f64_rhs
#include "dgm_kern_impl.cuh"
