// Adjoint stage kernel: degree 4, float fields.
#define DGM_P 4
#define DGM_REAL float
#define DGM_ADJ 1
#define DGM_LAUNCH launch_p4_f32_adj
#include "dgm_kern_impl.cuh"
