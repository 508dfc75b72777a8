// Adjoint stage kernel: degree 3, double fields.
#define DGM_P 3
#define DGM_REAL double
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p3_f64_adj
#include "dgm_kern_impl.cuh"
