// Fused stage kernel: degree 4, double fields, forward quantities for the adjoint.
#define DGM_P 4
#define DGM_REAL double
#define DGM_MODE MODE_RAW
#define DGM_LAUNCH launch_p4_f64_raw
#include "dgm_kern_impl.cuh"
