// Adjoint stage kernel: degree 4, double fields.
#define DGM_P 4
#define DGM_REAL double
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p4_f64_adj
#include "dgm_kern_impl.cuh"
