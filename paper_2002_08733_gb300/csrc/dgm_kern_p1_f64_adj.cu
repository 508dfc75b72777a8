// Adjoint stage kernel: degree 1, double fields.
#define DGM_P 1
#define DGM_REAL double
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p1_f64_adj
#include "dgm_kern_impl.cuh"
