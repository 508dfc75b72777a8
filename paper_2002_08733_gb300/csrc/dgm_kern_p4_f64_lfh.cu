// Fused stage kernel: degree 4, double fields, leapfrog H half step.
#define DGM_P 4
#define DGM_REAL double
#define DGM_MODE MODE_LF_H
#define DGM_LAUNCH launch_p4_f64_lfh
#include "dgm_kern_impl.cuh"
