// Dispatch tables over the per-(degree, precision, mode) kernel modules.
#include "dgm_internal.h"
#include "dgmax.h"

namespace dgm {

int launch_p1_f32_rhs(const StageParams&, void*);
int setref_p1_f32_rhs(const double*, const double*);
int launch_p1_f32_lsrk(const StageParams&, void*);
int setref_p1_f32_lsrk(const double*, const double*);
int launch_p1_f32_lfe(const StageParams&, void*);
int setref_p1_f32_lfe(const double*, const double*);
int launch_p1_f32_lfh(const StageParams&, void*);
int setref_p1_f32_lfh(const double*, const double*);
int launch_p1_f64_rhs(const StageParams&, void*);
int setref_p1_f64_rhs(const double*, const double*);
int launch_p1_f64_lsrk(const StageParams&, void*);
int setref_p1_f64_lsrk(const double*, const double*);
int launch_p1_f64_lfe(const StageParams&, void*);
int setref_p1_f64_lfe(const double*, const double*);
int launch_p1_f64_lfh(const StageParams&, void*);
int setref_p1_f64_lfh(const double*, const double*);
int launch_p2_f32_rhs(const StageParams&, void*);
int setref_p2_f32_rhs(const double*, const double*);
int launch_p2_f32_lsrk(const StageParams&, void*);
int setref_p2_f32_lsrk(const double*, const double*);
int launch_p2_f32_lfe(const StageParams&, void*);
int setref_p2_f32_lfe(const double*, const double*);
int launch_p2_f32_lfh(const StageParams&, void*);
int setref_p2_f32_lfh(const double*, const double*);
int launch_p2_f64_rhs(const StageParams&, void*);
int setref_p2_f64_rhs(const double*, const double*);
int launch_p2_f64_lsrk(const StageParams&, void*);
int setref_p2_f64_lsrk(const double*, const double*);
int launch_p2_f64_lfe(const StageParams&, void*);
int setref_p2_f64_lfe(const double*, const double*);
int launch_p2_f64_lfh(const StageParams&, void*);
int setref_p2_f64_lfh(const double*, const double*);
int launch_p3_f32_rhs(const StageParams&, void*);
int setref_p3_f32_rhs(const double*, const double*);
int launch_p3_f32_lsrk(const StageParams&, void*);
int setref_p3_f32_lsrk(const double*, const double*);
int launch_p3_f32_lfe(const StageParams&, void*);
int setref_p3_f32_lfe(const double*, const double*);
int launch_p3_f32_lfh(const StageParams&, void*);
int setref_p3_f32_lfh(const double*, const double*);
int launch_p3_f64_rhs(const StageParams&, void*);
int setref_p3_f64_rhs(const double*, const double*);
int launch_p3_f64_lsrk(const StageParams&, void*);
int setref_p3_f64_lsrk(const double*, const double*);
int launch_p3_f64_lfe(const StageParams&, void*);
int setref_p3_f64_lfe(const double*, const double*);
int launch_p3_f64_lfh(const StageParams&, void*);
int setref_p3_f64_lfh(const double*, const double*);
int launch_p4_f32_rhs(const StageParams&, void*);
int setref_p4_f32_rhs(const double*, const double*);
int launch_p4_f32_lsrk(const StageParams&, void*);
int setref_p4_f32_lsrk(const double*, const double*);
int launch_p4_f32_lfe(const StageParams&, void*);
int setref_p4_f32_lfe(const double*, const double*);
int launch_p4_f32_lfh(const StageParams&, void*);
int setref_p4_f32_lfh(const double*, const double*);
int launch_p4_f64_rhs(const StageParams&, void*);
int setref_p4_f64_rhs(const double*, const double*);
int launch_p4_f64_lsrk(const StageParams&, void*);
int setref_p4_f64_lsrk(const double*, const double*);
int launch_p4_f64_lfe(const StageParams&, void*);
int setref_p4_f64_lfe(const double*, const double*);
int launch_p4_f64_lfh(const StageParams&, void*);
int setref_p4_f64_lfh(const double*, const double*);
int launch_p5_f32_rhs(const StageParams&, void*);
int setref_p5_f32_rhs(const double*, const double*);
int launch_p5_f32_lsrk(const StageParams&, void*);
int setref_p5_f32_lsrk(const double*, const double*);
int launch_p5_f32_lfe(const StageParams&, void*);
int setref_p5_f32_lfe(const double*, const double*);
int launch_p5_f32_lfh(const StageParams&, void*);
int setref_p5_f32_lfh(const double*, const double*);

namespace {
int launch_p1_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p1_f32_rhs(prm, st);
        case MODE_LSRK: return launch_p1_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p1_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p1_f32_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p1_f32(const double* S, const double* R) {
    int rc = setref_p1_f32_rhs(S, R);
    if (!rc) rc = setref_p1_f32_lsrk(S, R);
    if (!rc) rc = setref_p1_f32_lfe(S, R);
    if (!rc) rc = setref_p1_f32_lfh(S, R);
    return rc;
}
int launch_p1_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p1_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p1_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p1_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p1_f64_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p1_f64(const double* S, const double* R) {
    int rc = setref_p1_f64_rhs(S, R);
    if (!rc) rc = setref_p1_f64_lsrk(S, R);
    if (!rc) rc = setref_p1_f64_lfe(S, R);
    if (!rc) rc = setref_p1_f64_lfh(S, R);
    return rc;
}
int launch_p2_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p2_f32_rhs(prm, st);
        case MODE_LSRK: return launch_p2_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p2_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p2_f32_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p2_f32(const double* S, const double* R) {
    int rc = setref_p2_f32_rhs(S, R);
    if (!rc) rc = setref_p2_f32_lsrk(S, R);
    if (!rc) rc = setref_p2_f32_lfe(S, R);
    if (!rc) rc = setref_p2_f32_lfh(S, R);
    return rc;
}
int launch_p2_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p2_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p2_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p2_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p2_f64_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p2_f64(const double* S, const double* R) {
    int rc = setref_p2_f64_rhs(S, R);
    if (!rc) rc = setref_p2_f64_lsrk(S, R);
    if (!rc) rc = setref_p2_f64_lfe(S, R);
    if (!rc) rc = setref_p2_f64_lfh(S, R);
    return rc;
}
int launch_p3_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p3_f32_rhs(prm, st);
        case MODE_LSRK: return launch_p3_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p3_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p3_f32_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p3_f32(const double* S, const double* R) {
    int rc = setref_p3_f32_rhs(S, R);
    if (!rc) rc = setref_p3_f32_lsrk(S, R);
    if (!rc) rc = setref_p3_f32_lfe(S, R);
    if (!rc) rc = setref_p3_f32_lfh(S, R);
    return rc;
}
int launch_p3_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p3_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p3_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p3_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p3_f64_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p3_f64(const double* S, const double* R) {
    int rc = setref_p3_f64_rhs(S, R);
    if (!rc) rc = setref_p3_f64_lsrk(S, R);
    if (!rc) rc = setref_p3_f64_lfe(S, R);
    if (!rc) rc = setref_p3_f64_lfh(S, R);
    return rc;
}
int launch_p4_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p4_f32_rhs(prm, st);
        case MODE_LSRK: return launch_p4_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p4_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p4_f32_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p4_f32(const double* S, const double* R) {
    int rc = setref_p4_f32_rhs(S, R);
    if (!rc) rc = setref_p4_f32_lsrk(S, R);
    if (!rc) rc = setref_p4_f32_lfe(S, R);
    if (!rc) rc = setref_p4_f32_lfh(S, R);
    return rc;
}
int launch_p4_f64(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p4_f64_rhs(prm, st);
        case MODE_LSRK: return launch_p4_f64_lsrk(prm, st);
        case MODE_LF_E: return launch_p4_f64_lfe(prm, st);
        case MODE_LF_H: return launch_p4_f64_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p4_f64(const double* S, const double* R) {
    int rc = setref_p4_f64_rhs(S, R);
    if (!rc) rc = setref_p4_f64_lsrk(S, R);
    if (!rc) rc = setref_p4_f64_lfe(S, R);
    if (!rc) rc = setref_p4_f64_lfh(S, R);
    return rc;
}
int launch_p5_f32(const StageParams& prm, int mode, void* st) {
    switch (mode) {
        case MODE_RHS: return launch_p5_f32_rhs(prm, st);
        case MODE_LSRK: return launch_p5_f32_lsrk(prm, st);
        case MODE_LF_E: return launch_p5_f32_lfe(prm, st);
        case MODE_LF_H: return launch_p5_f32_lfh(prm, st);
        default: return DGM_EINVAL;
    }
}
int setref_p5_f32(const double* S, const double* R) {
    int rc = setref_p5_f32_rhs(S, R);
    if (!rc) rc = setref_p5_f32_lsrk(S, R);
    if (!rc) rc = setref_p5_f32_lfe(S, R);
    if (!rc) rc = setref_p5_f32_lfh(S, R);
    return rc;
}
}  // namespace

extern const KernelTable kernels_p1_f32 = {launch_p1_f32, setref_p1_f32, 4};
extern const KernelTable kernels_p1_f64 = {launch_p1_f64, setref_p1_f64, 8};
extern const KernelTable kernels_p2_f32 = {launch_p2_f32, setref_p2_f32, 4};
extern const KernelTable kernels_p2_f64 = {launch_p2_f64, setref_p2_f64, 8};
extern const KernelTable kernels_p3_f32 = {launch_p3_f32, setref_p3_f32, 4};
extern const KernelTable kernels_p3_f64 = {launch_p3_f64, setref_p3_f64, 8};
extern const KernelTable kernels_p4_f32 = {launch_p4_f32, setref_p4_f32, 4};
extern const KernelTable kernels_p4_f64 = {launch_p4_f64, setref_p4_f64, 8};
extern const KernelTable kernels_p5_f32 = {launch_p5_f32, setref_p5_f32, 4};

}  // namespace dgm
