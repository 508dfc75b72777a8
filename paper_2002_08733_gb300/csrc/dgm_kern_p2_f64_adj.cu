// Adjoint stage kernel: degree 2, double fields.
#define DGM_P 2
#define DGM_REAL double
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p2_f64_adj
#include "dgm_kern_impl.cuh"
