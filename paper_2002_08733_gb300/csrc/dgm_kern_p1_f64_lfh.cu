// Fused stage kernel: degree 1, double fields, leapfrog H half step.
#define DGM_P 1
#define DGM_REAL double
#define DGM_MODE MODE_LF_H
#define DGM_LAUNCH launch_p1_f64_lfh
#include "dgm_kern_impl.cuh"
