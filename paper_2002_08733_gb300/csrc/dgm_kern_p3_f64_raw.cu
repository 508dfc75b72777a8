// Fused stage kernel: degree 3, double fields, forward quantities for the adjoint.
#define DGM_P 3
#define DGM_REAL double
#define DGM_MODE MODE_RAW
#define DGM_LAUNCH launch_p3_f64_raw
#include "dgm_kern_impl.cuh"
