// Fused stage kernel: degree 3, double fields, leapfrog H half step.
#define DGM_P 3
#define DGM_REAL double
#define DGM_MODE MODE_LF_H
#define DGM_LAUNCH launch_p3_f64_lfh
#include "dgm_kern_impl.cuh"
