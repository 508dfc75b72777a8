// Fused stage kernel: degree 2, float fields, forward quantities for the adjoint.
#define DGM_P 2
#define DGM_REAL float
#define DGM_MODE MODE_RAW
#define DGM_LAUNCH launch_p2_f32_raw
#include "dgm_kern_impl.cuh"
