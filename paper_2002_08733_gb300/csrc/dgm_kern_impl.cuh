// Body of one kernel translation unit: instantiates the fused stage kernel for
// one polynomial degree (DGM_P), one field precision (DGM_REAL) and one mode
// (DGM_MODE) and exports its launcher DGM_LAUNCH.  Included by the
// dgm_kern_p<P>_<precision>_<mode>.cu files; one mode per file keeps the
// heavily unrolled kernels compiling in parallel.
#include <cuda_runtime.h>

#include <vector>

#include "dgm_internal.h"
#include "dgmax.h"

#ifdef DGM_ADJ
#include "dgm_adjoint.cuh"
#elif defined(DGM_PAIR)
#include "dgm_stage2.cuh"
#else
#include "dgm_stage.cuh"
#endif

namespace dgm {
namespace {

constexpr int kP = DGM_P;
using Real = DGM_REAL;
// tile shape: columns per CTA and threads per CTA (DGM_TE / DGM_NT select an
// autotuner variant; the defaults are the shapes measured best at p = 3)
#ifdef DGM_TC
constexpr bool kTC = true;    // tensor-core variant (curl and lift on tcgen05)
#else
constexpr bool kTC = false;
#endif
#ifdef DGM_TE
constexpr int kTE = DGM_TE;
constexpr int kNT = DGM_NT;
#else
constexpr int kTE = sizeof(Real) == 8 ? 16 : 32;
constexpr int kNT = sizeof(Real) == 8 ? 192 : 384;
#endif

#ifdef DGM_ADJ
constexpr int kTEA = sizeof(Real) == 8 ? 16 : 32;
constexpr int kNTA = sizeof(Real) == 8 ? 192 : 384;
template <typename IX>
int launch_adj_ix(const AdjParams& prm, unsigned grid, cudaStream_t st) {
    constexpr size_t smem = adjoint_smem_bytes<kP, Real, kTEA, kNTA>();
    static bool configured = false;
    auto k = adjoint_kernel<kP, Real, kTEA, kNTA, IX>;
    if (!configured) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
            return DGM_ECUDA;
        configured = true;
    }
    k<<<grid, kNTA, smem, st>>>(prm);
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

// true when every index the adjoint kernel forms is below 2^32: field rows
// (6N x C), face jumps (24 NF x C), auxiliaries, geometry, the per-face
// table, neighbours and the two gradient rows (2C)
bool fits_32bit(const AdjParams& p) {
    const uint64_t lim = uint64_t(1) << 32;
    const uint64_t K = uint64_t(p.K), C = K * uint64_t(p.S);
    const uint64_t N = uint64_t(nmodes(kP)), NF = uint64_t(nfmodes(kP));
    return 6 * N * C < lim && 24 * NF * C < lim && 6 * N * uint64_t(p.npml) * uint64_t(p.S) < lim &&
           uint64_t(G_COUNT) * K < lim && 4 * uint64_t(FNB_COUNT) * K < lim && 4 * K < lim &&
           2 * C < lim;
}

int launch_adj(const AdjParams& prm, cudaStream_t st) {
    const int64_t C = prm.K * prm.S;
    if (C <= 0) return DGM_OK;
    const unsigned grid = unsigned((C + kTEA - 1) / kTEA);
    return (!prm.force_index64 && fits_32bit(prm)) ? launch_adj_ix<uint32_t>(prm, grid, st)
                                                    : launch_adj_ix<int64_t>(prm, grid, st);
}
#elif defined(DGM_PAIR)
// paired kernel: 64 columns per CTA, two per thread (LSRK stages only)
template <typename IX>
int launch_pair_ix(const StageParams& q, unsigned grid, cudaStream_t st) {
    using Pair = DGM_PAIR;
    constexpr size_t smem = stage2_smem_bytes<kP, Pair>();
    static bool configured = false;
    auto k = stage2_kernel<kP, Pair, kNT, IX>;
    if (!configured) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
            return DGM_ECUDA;
        configured = true;
    }
    k<<<grid, kNT, smem, st>>>(q);
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

// every index below 2^32 (the same buffers as the single-column kernel)
bool fits_32bit(const StageParams& p) {
    const uint64_t lim = uint64_t(1) << 32;
    const uint64_t K = uint64_t(p.K), C = K * uint64_t(p.S);
    const uint64_t N = uint64_t(nmodes(kP));
    return 6 * N * C + 64 < lim && 6 * N * uint64_t(p.npml) * uint64_t(p.S) < lim &&
           uint64_t(G_COUNT) * K < lim && 4 * uint64_t(FNB_COUNT) * K < lim && 4 * K < lim;
}

int launch_mode(const StageParams& prm, cudaStream_t st) {
    const int64_t C = prm.K_active * prm.S;   // columns updated
    if (C <= 0) return DGM_OK;
    const unsigned grid = unsigned((C + 63) / 64);
    StageParams q = prm;
    q.dt_f = float(prm.dt);
    q.a_f = float(prm.a);
    q.b_f = float(prm.b);
    return (!q.force_index64 && fits_32bit(q)) ? launch_pair_ix<uint32_t>(q, grid, st)
                                               : launch_pair_ix<int64_t>(q, grid, st);
}
#else
// the interior penalty's kernels: LSRK and right-hand-side modes, default tile shape
#if !defined(DGM_TE) && !defined(DGM_TC)
constexpr bool kSIP = (DGM_MODE == MODE_LSRK || DGM_MODE == MODE_RHS);
#else
constexpr bool kSIP = false;
#endif

template <typename IX, bool SIP>
int launch_ix(const StageParams& q, unsigned grid, cudaStream_t st) {
    constexpr size_t smem = stage_smem_bytes<kP, Real, kTE, kTC, SIP>();
    static bool configured = false;
    auto k = stage_kernel<kP, Real, kTE, kNT, DGM_MODE, IX, kTC, SIP>;
    if (kTC && q.tc_b == nullptr) return DGM_EUNSUP;   // no operator image for this plan
    if (!configured) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
            return DGM_ECUDA;
        configured = true;
    }
    k<<<grid, kNT, smem, st>>>(q);
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

// true when every index the stage kernel forms for this plan is below 2^32:
// field rows (6N x C), face jumps (24 NF x C), auxiliaries (6N x npml S),
// geometry (G_COUNT x K), the per-face table (4 FNB_COUNT x K), neighbours (4K)
bool fits_32bit(const StageParams& p) {
    const uint64_t lim = uint64_t(1) << 32;
    const uint64_t K = uint64_t(p.K), C = K * uint64_t(p.S);
    const uint64_t N = uint64_t(nmodes(kP)), NF = uint64_t(nfmodes(kP));
    return 6 * N * C < lim && 24 * NF * C < lim && 6 * N * uint64_t(p.npml) * uint64_t(p.S) < lim &&
           uint64_t(G_COUNT) * K < lim && 4 * uint64_t(FNB_COUNT) * K < lim && 4 * K < lim;
}

int launch_mode(const StageParams& prm, cudaStream_t st) {
    const int64_t C = prm.K_active * prm.S;   // columns updated
    if (C <= 0) return DGM_OK;
    const unsigned grid = unsigned((C + kTE - 1) / kTE);
    StageParams q = prm;
    q.dt_f = float(prm.dt);
    q.a_f = float(prm.a);
    q.b_f = float(prm.b);
    const bool i32 = !q.force_index64 && fits_32bit(q);
    // phase-1 bulk copies: the plan's tensor-map set of this tile width (rows
    // of 128 bytes, or 16 FP32 columns) and the map of this stage's input
    q.tm_u = -1;
    constexpr int kSet = kTC ? -1 : (kTE * int(sizeof(Real)) == 128 ? 0 : (sizeof(Real) == 4 && kTE == 16 ? 1 : -1));
    if (kSet >= 0 && q.tmaps != nullptr && q.S == 1) {
        q.tmaps = static_cast<const char*>(q.tmaps) + size_t(kSet) * TMAP_COUNT * TMAP_BYTES;
        q.tm_u = q.u == q.tm_f0 ? TM_U0
                 : q.u == q.tm_f1 ? TM_U1
                 : (q.tm_fw != nullptr && q.u == q.tm_fw) ? TM_UW : -1;
    }
    if (q.hs != nullptr) {   // interior penalty
        if constexpr (kSIP) {
            return i32 ? launch_ix<uint32_t, true>(q, grid, st) : launch_ix<int64_t, true>(q, grid, st);
        } else {
            return DGM_EUNSUP;
        }
    }
    return i32 ? launch_ix<uint32_t, false>(q, grid, st) : launch_ix<int64_t, false>(q, grid, st);
}
#endif

}  // namespace

#ifdef DGM_ADJ
int DGM_LAUNCH(const AdjParams& prm, void* stream) {
    return launch_adj(prm, static_cast<cudaStream_t>(stream));
}
#else
int DGM_LAUNCH(const StageParams& prm, void* stream) {
    return launch_mode(prm, static_cast<cudaStream_t>(stream));
}
#endif



}  // namespace dgm
