// Fused stage kernel: degree 1, float fields, forward quantities for the adjoint.
#define DGM_P 1
#define DGM_REAL float
#define DGM_MODE MODE_RAW
#define DGM_LAUNCH launch_p1_f32_raw
#include "dgm_kern_impl.cuh"
