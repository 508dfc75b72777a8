// Fused stage kernel: degree 2, float fields, leapfrog H half step.
#define DGM_P 2
#define DGM_REAL float
#define DGM_MODE MODE_LF_H
#define DGM_LAUNCH launch_p2_f32_lfh
#include "dgm_kern_impl.cuh"
