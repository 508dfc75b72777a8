// Body of one kernel translation unit: instantiates the fused stage kernel for
// one polynomial degree (DGM_P), one field precision (DGM_REAL) and one mode
// (DGM_MODE) and exports its launcher DGM_LAUNCH.  Included by the
// dgm_kern_p<P>_<precision>_<mode>.cu files; one mode per file keeps the
// heavily unrolled kernels compiling in parallel.
#include <cuda_runtime.h>

#include <vector>

#include "dgm_internal.h"
#include "dgmax.h"

#include "dgm_stage.cuh"

namespace dgm {
namespace {

constexpr int kP = DGM_P;
using Real = DGM_REAL;
constexpr int kTE = sizeof(Real) == 8 ? 16 : 32;   // columns per CTA
constexpr int kNT = 192;                            // threads per CTA

int launch_mode(const StageParams& prm, cudaStream_t st) {
    constexpr size_t smem = stage_smem_bytes<kP, Real, kTE>();
    static bool configured = false;
    auto k = stage_kernel<kP, Real, kTE, kNT, DGM_MODE>;
    if (!configured) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
            return DGM_ECUDA;
        configured = true;
    }
    const int64_t C = prm.K * prm.S;
    if (C <= 0) return DGM_OK;
    const unsigned grid = unsigned((C + kTE - 1) / kTE);
    k<<<grid, kNT, smem, st>>>(prm);
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

}  // namespace

int DGM_LAUNCH(const StageParams& prm, void* stream) {
    return launch_mode(prm, static_cast<cudaStream_t>(stream));
}



}  // namespace dgm
