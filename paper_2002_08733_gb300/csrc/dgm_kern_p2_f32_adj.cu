// Adjoint stage kernel: degree 2, float fields.
#define DGM_P 2
#define DGM_REAL float
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p2_f32_adj
#include "dgm_kern_impl.cuh"
