// Adjoint stage kernel: degree 1, float fields.
#define DGM_P 1
#define DGM_REAL float
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p1_f32_adj
#include "dgm_kern_impl.cuh"
