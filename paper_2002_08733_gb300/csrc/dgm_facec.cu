// The stage kernels' precomputed face constants (face_consts_kernel), one
// thread per element, in the plan's precision.
#include <cuda_runtime.h>

#include "dgm_internal.h"
#include "dgm_stage.cuh"
#include "dgmax.h"

namespace dgm {

int launch_face_consts(const StageParams& prm, int real_size, bool sip, void* out, void* stream) {
    if (prm.K <= 0) return DGM_OK;
    const unsigned grid = unsigned((prm.K + 127) / 128);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (real_size == 8) {
        if (sip) face_consts_kernel<double, true><<<grid, 128, 0, st>>>(prm, static_cast<double*>(out));
        else face_consts_kernel<double, false><<<grid, 128, 0, st>>>(prm, static_cast<double*>(out));
    } else {
        if (sip) face_consts_kernel<float, true><<<grid, 128, 0, st>>>(prm, static_cast<float*>(out));
        else face_consts_kernel<float, false><<<grid, 128, 0, st>>>(prm, static_cast<float*>(out));
    }
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

}  // namespace dgm
