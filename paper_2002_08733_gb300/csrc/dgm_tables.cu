// Dispatch tables over the per-(degree, precision, mode) kernel modules.
// FP32 LSRK stage variants for the autotuner: 0 = 32 columns x 384 threads,
// 1 = 32 x 192, 2 = 16 x 192, and up to p = 3 (where 64 columns of pairs fit
// in shared memory) 3 = paired kernel with packed FP32x2 arithmetic,
// 4 = paired kernel with scalar arithmetic; at p >= 4 (one CTA per SM)
// 3 = 32 x 512; at p = 2, 3 also 5 = tensor-core variant (64 columns x 512
// threads, curl and lift on tcgen05).
#include "dgm_internal.h"
#include "dgmax.h"

namespace dgm {

int launch_p1_f32_rhs(const StageParams&, void*);
int launch_p1_f32_lsrk(const StageParams&, void*);
int launch_p1_f32_lfe(const StageParams&, void*);
int launch_p1_f32_lfh(const StageParams&, void*);
int launch_p1_f32_raw(const StageParams&, void*);
int launch_p1_f32_adj(const AdjParams&, void*);
int launch_p1_f32_lsrk_v1(const StageParams&, void*);
int launch_p1_f32_lsrk_v2(const StageParams&, void*);
int launch_p1_f32_lsrk_v3(const StageParams&, void*);
int launch_p1_f32_lsrk_v4(const StageParams&, void*);
int launch_p1_f64_rhs(const StageParams&, void*);
int launch_p1_f64_lsrk(const StageParams&, void*);
int launch_p1_f64_lfe(const StageParams&, void*);
int launch_p1_f64_lfh(const StageParams&, void*);
int launch_p1_f64_raw(const StageParams&, void*);
int launch_p1_f64_adj(const AdjParams&, void*);
int launch_p2_f32_rhs(const StageParams&, void*);
int launch_p2_f32_lsrk(const StageParams&, void*);
int launch_p2_f32_lfe(const StageParams&, void*);
int launch_p2_f32_lfh(const StageParams&, void*);
int launch_p2_f32_raw(const StageParams&, void*);
int launch_p2_f32_adj(const AdjParams&, void*);
int launch_p2_f32_lsrk_v1(const StageParams&, void*);
int launch_p2_f32_lsrk_v2(const StageParams&, void*);
int launch_p2_f32_lsrk_v3(const StageParams&, void*);
int launch_p2_f32_lsrk_v4(const StageParams&, void*);
int launch_p2_f32_lsrk_v5(const StageParams&, void*);
int launch_p2_f64_rhs(const StageParams&, void*);
int launch_p2_f64_lsrk(const StageParams&, void*);
int launch_p2_f64_lfe(const StageParams&, void*);
int launch_p2_f64_lfh(const StageParams&, void*);
int launch_p2_f64_raw(const StageParams&, void*);
int launch_p2_f64_adj(const AdjParams&, void*);
int launch_p3_f32_rhs(const StageParams&, void*);
int launch_p3_f32_lsrk(const StageParams&, void*);
int launch_p3_f32_lfe(const StageParams&, void*);
int launch_p3_f32_lfh(const StageParams&, void*);
int launch_p3_f32_raw(const StageParams&, void*);
int launch_p3_f32_adj(const AdjParams&, void*);
int launch_p3_f32_lsrk_v1(const StageParams&, void*);
int launch_p3_f32_lsrk_v2(const StageParams&, void*);
int launch_p3_f32_lsrk_v3(const StageParams&, void*);
int launch_p3_f32_lsrk_v4(const StageParams&, void*);
int launch_p3_f32_lsrk_v5(const StageParams&, void*);
int launch_p3_f64_rhs(const StageParams&, void*);
int launch_p3_f64_lsrk(const StageParams&, void*);
int launch_p3_f64_lfe(const StageParams&, void*);
int launch_p3_f64_lfh(const StageParams&, void*);
int launch_p3_f64_raw(const StageParams&, void*);
int launch_p3_f64_adj(const AdjParams&, void*);
int launch_p4_f32_rhs(const StageParams&, void*);
int launch_p4_f32_lsrk(const StageParams&, void*);
int launch_p4_f32_lfe(const StageParams&, void*);
int launch_p4_f32_lfh(const StageParams&, void*);
int launch_p4_f32_raw(const StageParams&, void*);
int launch_p4_f32_adj(const AdjParams&, void*);
int launch_p4_f32_lsrk_v1(const StageParams&, void*);
int launch_p4_f32_lsrk_v2(const StageParams&, void*);
int launch_p4_f32_lsrk_v3(const StageParams&, void*);
int launch_p4_f64_rhs(const StageParams&, void*);
int launch_p4_f64_lsrk(const StageParams&, void*);
int launch_p4_f64_lfe(const StageParams&, void*);
int launch_p4_f64_lfh(const StageParams&, void*);
int launch_p4_f64_raw(const StageParams&, void*);
int launch_p4_f64_adj(const AdjParams&, void*);
int launch_p5_f32_rhs(const StageParams&, void*);
int launch_p5_f32_lsrk(const StageParams&, void*);
int launch_p5_f32_lfe(const StageParams&, void*);
int launch_p5_f32_lfh(const StageParams&, void*);
int launch_p5_f32_raw(const StageParams&, void*);
int launch_p5_f32_adj(const AdjParams&, void*);
int launch_p5_f32_lsrk_v1(const StageParams&, void*);
int launch_p5_f32_lsrk_v2(const StageParams&, void*);
int launch_p5_f32_lsrk_v3(const StageParams&, void*);

namespace {

int launch_p1_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p1_f32_rhs(prm, st);
        case MODE_LSRK:
            if (prm.variant == 1) return launch_p1_f32_lsrk_v1(prm, st);
            if (prm.variant == 2) return launch_p1_f32_lsrk_v2(prm, st);
            if (prm.variant == 3) return launch_p1_f32_lsrk_v3(prm, st);
            if (prm.variant == 4) return launch_p1_f32_lsrk_v4(prm, st);
            return launch_p1_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p1_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p1_f32_lfh(prm, st);
        case MODE_RAW: return launch_p1_f32_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p1_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p1_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p1_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p1_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p1_f64_lfh(prm, st);
        case MODE_RAW: return launch_p1_f64_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p2_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p2_f32_rhs(prm, st);
        case MODE_LSRK:
            if (prm.variant == 1) return launch_p2_f32_lsrk_v1(prm, st);
            if (prm.variant == 2) return launch_p2_f32_lsrk_v2(prm, st);
            if (prm.variant == 3) return launch_p2_f32_lsrk_v3(prm, st);
            if (prm.variant == 4) return launch_p2_f32_lsrk_v4(prm, st);
            if (prm.variant == 5) return launch_p2_f32_lsrk_v5(prm, st);
            return launch_p2_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p2_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p2_f32_lfh(prm, st);
        case MODE_RAW: return launch_p2_f32_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p2_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p2_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p2_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p2_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p2_f64_lfh(prm, st);
        case MODE_RAW: return launch_p2_f64_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p3_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p3_f32_rhs(prm, st);
        case MODE_LSRK:
            if (prm.variant == 1) return launch_p3_f32_lsrk_v1(prm, st);
            if (prm.variant == 2) return launch_p3_f32_lsrk_v2(prm, st);
            if (prm.variant == 3) return launch_p3_f32_lsrk_v3(prm, st);
            if (prm.variant == 4) return launch_p3_f32_lsrk_v4(prm, st);
            if (prm.variant == 5) return launch_p3_f32_lsrk_v5(prm, st);
            return launch_p3_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p3_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p3_f32_lfh(prm, st);
        case MODE_RAW: return launch_p3_f32_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p3_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p3_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p3_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p3_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p3_f64_lfh(prm, st);
        case MODE_RAW: return launch_p3_f64_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p4_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p4_f32_rhs(prm, st);
        case MODE_LSRK:
            if (prm.variant == 1) return launch_p4_f32_lsrk_v1(prm, st);
            if (prm.variant == 2) return launch_p4_f32_lsrk_v2(prm, st);
            if (prm.variant == 3) return launch_p4_f32_lsrk_v3(prm, st);
            return launch_p4_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p4_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p4_f32_lfh(prm, st);
        case MODE_RAW: return launch_p4_f32_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p4_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p4_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p4_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p4_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p4_f64_lfh(prm, st);
        case MODE_RAW: return launch_p4_f64_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

int launch_p5_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p5_f32_rhs(prm, st);
        case MODE_LSRK:
            if (prm.variant == 1) return launch_p5_f32_lsrk_v1(prm, st);
            if (prm.variant == 2) return launch_p5_f32_lsrk_v2(prm, st);
            if (prm.variant == 3) return launch_p5_f32_lsrk_v3(prm, st);
            return launch_p5_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p5_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p5_f32_lfh(prm, st);
        case MODE_RAW: return launch_p5_f32_raw(prm, st);
        default: return DGM_EINVAL;
    }
}

}  // namespace

extern const KernelTable kernels_p1_f32 = {launch_p1_f32, 4, launch_p1_f32_adj, 5};
extern const KernelTable kernels_p1_f64 = {launch_p1_f64, 8, launch_p1_f64_adj, 1};
extern const KernelTable kernels_p2_f32 = {launch_p2_f32, 4, launch_p2_f32_adj, 6};
extern const KernelTable kernels_p2_f64 = {launch_p2_f64, 8, launch_p2_f64_adj, 1};
extern const KernelTable kernels_p3_f32 = {launch_p3_f32, 4, launch_p3_f32_adj, 6};
extern const KernelTable kernels_p3_f64 = {launch_p3_f64, 8, launch_p3_f64_adj, 1};
extern const KernelTable kernels_p4_f32 = {launch_p4_f32, 4, launch_p4_f32_adj, 4};
extern const KernelTable kernels_p4_f64 = {launch_p4_f64, 8, launch_p4_f64_adj, 1};
extern const KernelTable kernels_p5_f32 = {launch_p5_f32, 4, launch_p5_f32_adj, 4};

}  // namespace dgm
