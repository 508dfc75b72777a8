// C ABI of the dgmax library: plans, binding of caller-owned device memory,
// the time-stepping drivers (LSRK4 stages, leapfrog half steps), the FP64
// energy reduction, point sources and L2 projection of initial values.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dgm_internal.h"
#include "dgm_ops_gen.cuh"
#include "dgmax.h"

namespace dgm {

#define DECL(p, r) extern const KernelTable kernels_p##p##_##r;
DECL(1, f32) DECL(2, f32) DECL(3, f32) DECL(4, f32) DECL(5, f32)
DECL(1, f64) DECL(2, f64) DECL(3, f64) DECL(4, f64)
#undef DECL

const KernelTable* kernel_table(int p, int precision) {
    static const KernelTable* f32[] = {nullptr, &kernels_p1_f32, &kernels_p2_f32, &kernels_p3_f32,
                                       &kernels_p4_f32, &kernels_p5_f32};
    static const KernelTable* f64[] = {nullptr, &kernels_p1_f64, &kernels_p2_f64, &kernels_p3_f64,
                                       &kernels_p4_f64, nullptr};
    if (p < 1 || p > PMAX) return nullptr;
    return precision == DGM_FP64 ? f64[p] : (precision == DGM_FP32 ? f32[p] : nullptr);
}

// Carpenter & Kennedy (1994) five-stage, fourth-order, 2N-storage Runge-Kutta.
static const double LSRK_A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                                 -2404267990393.0 / 2016746695238.0,
                                 -3550918686646.0 / 2091501179385.0,
                                 -1275806237668.0 / 842570457699.0};
static const double LSRK_B[5] = {1432997174477.0 / 9575080441755.0,
                                 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0,
                                 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};
static const double LSRK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                                 2526269341429.0 / 6820363962896.0,
                                 2006345519317.0 / 3224310063776.0,
                                 2802321613138.0 / 2924317926251.0};

constexpr int ENERGY_BLOCKS = 304;   // 2 per SM
constexpr int REC_HDR = 4;           // receiver record: [elem, 0, 0, 0, W[3][3N]]
constexpr int ENERGY_THREADS = 256;

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// incident plane-wave table: header values, values per face, largest face rule,
// stage slots of the jump terms
constexpr int INC_HDR = 8, INC_FACE = 6, INC_MAXQ = 128, INC_SLOTS = 5;
static_assert((PMAX + 6) * (PMAX + 6) <= INC_MAXQ, "face rule larger than a warp's four rounds");

// Bytes of the tensor-core variant's operator image for degree p (0: no variant).
static size_t tc_image_bytes(int p) {
    switch (p) {
        case 2: return TcShape<2>::B_BYTES;
        case 3: return TcShape<3>::B_BYTES;
        default: return 0;
    }
}

// x rounded to the nearest TF32 value (11 significant bits), as a float
static float tf32_nearest(double x) {
    if (x == 0.0 || !std::isfinite(x)) return float(x);
    int ex;
    const double m = std::frexp(x, &ex);   // x = m 2^ex, 0.5 <= |m| < 1
    return float(std::ldexp(std::round(std::ldexp(m, 11)), ex - 11));
}

// The operator image of the tensor-core stage variant (TcShape): the reference
// curl B_curl[(i, m)][(j, l)] = eps_jai S_a[l][m] (Eq. (matrix_free_curl)) and
// the lift B_lift[(f, m)][l] = R_f[m][l] (Eqs. (uwc)/(cwc)), each as TF32 hi
// and lo parts (hi = tf32(x), lo = tf32(x - hi)) in the K-major core-matrix
// layout of tc_b_offset.  Entries below 1e-13 of the matrix maximum are the
// round-off of exact zeros and are dropped, as in the compiled operators.
template <int P>
static void build_tc_image_p(const std::vector<double>& S, const std::vector<double>& R,
                             std::vector<unsigned char>& out) {
    using TS = TcShape<P>;
    constexpr int N = TS::N, NF = TS::NF;
    out.assign(TS::B_BYTES, 0);
    double smax = 0, rmax = 0;
    for (double v : S) smax = std::fmax(smax, std::fabs(v));
    for (double v : R) rmax = std::fmax(rmax, std::fabs(v));
    auto put = [&](size_t base, int n, int k, int K, float v) {
        std::memcpy(out.data() + base + tc_b_offset(n, k, K), &v, sizeof(float));
    };
    auto split = [&](size_t hi_base, size_t lo_base, int n, int k, int K, double x) {
        const float hi = tf32_nearest(x);
        put(hi_base, n, k, K, hi);
        put(lo_base, n, k, K, tf32_nearest(x - double(hi)));
    };
    for (int i = 0; i < 3; ++i)          // input component
        for (int j = 0; j < 3; ++j) {    // output component
            if (i == j) continue;
            const int a = 3 - i - j;     // curl_j = eps_jai d_a v_i
            const double eps = ((j - a + 3) % 3 == 2) ? 1.0 : -1.0;   // eps_jai with (j, a, i) a permutation
            for (int m = 0; m < N; ++m)
                for (int l = 0; l < N; ++l) {
                    double v = S[(size_t(a) * N + l) * N + m];
                    if (!(std::fabs(v) > 1e-13 * smax)) continue;
                    split(0, TS::B_CURL, j * TS::NL + l, i * N + m, TS::KC, eps * v);
                }
        }
    for (int f = 0; f < 4; ++f)
        for (int m = 0; m < NF; ++m)
            for (int l = 0; l < N; ++l) {
                const double v = R[(size_t(f) * NF + m) * N + l];
                if (!(std::fabs(v) > 1e-13 * rmax)) continue;
                split(2 * TS::B_CURL, 2 * TS::B_CURL + TS::B_LIFT, l, f * NF + m, TS::KL, v);
            }
}

static void build_tc_image(int p, const std::vector<double>& S, const std::vector<double>& R,
                           std::vector<unsigned char>& out) {
    if (p == 2) build_tc_image_p<2>(S, R, out);
    else if (p == 3) build_tc_image_p<3>(S, R, out);
    else out.clear();
}

}  // namespace dgm

using namespace dgm;

struct dgm_plan {
    dgm_options opt;
    HostMesh mesh;
    const KernelTable* kt = nullptr;
    std::vector<double> S, R;   // reference matrices (FP64), degree pE
    int N = 0, NF = 0;          // modes per component (E's on a mixed-order plan)
    int mixed = 0;              // E of degree p + 1, H of degree p (dgm_plan_create_mixed)
    int pE = 0;                 // degree of E (= opt.p unless mixed)
    int NH = 0, NFH = 0;        // modes per H component (= N, NF unless mixed)
    bool has_pml = false;
    // geometry buffer layout (byte offsets)
    size_t off_geo = 0, off_nbr = 0, off_pml = 0, off_src = 0, off_part = 0, off_status = 0,
           off_rec = 0, off_time = 0, off_geo32 = 0, off_fnb = 0, off_fnb32 = 0, off_tcb = 0,
           bytes_tcb = 0, off_ops = 0, bytes_ops = 0, bytes_geom = 0;
    int n_rec = 0;
    std::vector<double> src_host;   // S * (SRC_HDR + 3N)
    bool have_src = false;
    // bound state
    bool bound = false;
    unsigned char* geom = nullptr;
    void* fields[2] = {nullptr, nullptr};
    void* res = nullptr;
    void* aux[2] = {nullptr, nullptr};
    void* aux_res = nullptr;
    cudaStream_t stream = nullptr;
    int cur = 0;
    int device = -1;
    int variant = 0;          // LSRK stage tile shape chosen by dgm_autotune
    int force_index64 = 0;    // dgm_set_index64
    int tile_groups = 1;      // tile visiting order (dgm_autotune, dgm_set_tile_groups)
    int64_t k_active = 0;     // elements updated (dgm_set_active); the rest are halo copies
    float variant_ms[8] = {0};
    // incident plane wave (dgm_set_incident)
    int64_t n_bfaces = 0;     // boundary faces of the mesh: capacity of the incident tables
    int64_t n_inc = 0;        // incident faces (codes -2 - i in the neighbour table)
    int inc_nq = 0;           // points of the face rule
    size_t off_inc = 0, off_incv = 0;
    std::vector<double> inc_host;    // the FP64 table (layout at incident_eval)
    std::vector<int32_t> nbr_plain;  // neighbour table without incident codes
    // interior penalty with a facet field (dgm_set_sip, dgm_bind_sip)
    double sip_alpha = 0.0;          // 0: off
    int64_t n_facets = 0;            // interior facets
    size_t off_sfid = 0;             // [4][K] int32: (facet << 1) | owner, or -1
    size_t off_fcp = 0;              // [FC_ROWS][K] precomputed face constants (plan precision)
    std::vector<int32_t> sfid_host;
    void* hs[2] = {nullptr, nullptr};
    void* hs_res = nullptr;
    // tensor maps of the stage kernels' phase-1 bulk copies (built at bind)
    size_t off_tmap = 0;             // TMAP_SETS x TMAP_COUNT maps of TMAP_BYTES
    bool tmaps_ok = false;           // built: one column per element, aligned rows
    int tile_loads = 0;              // dgm_set_tile_loads: 1 forces per-thread loads
    std::vector<CUtensorMap> tmap_host;
};

// bytes of one stage slot of the incident jump terms (every boundary face)
static size_t inc_slot_bytes(const dgm_plan* P) {
    return size_t(P->kt->real_size) * 3 * P->NF * P->n_bfaces;
}

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
    return fail(DGM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace dgm {
int partition_fail(int code, const std::string& msg) { return fail(code, msg); }
}

// ---------------------------------------------------------------------------
// FP64 energy: W_s = 1/2 sum_T |det| sum_l (eps u_l^T G u_l + mu h_l^T G h_l), G = A^-1 A^-T
template <typename R>
__global__ void __launch_bounds__(ENERGY_THREADS)
energy_partial(const R* __restrict__ u, const double* __restrict__ geo, int64_t K, int64_t Kact,
               int S, int N, int NH, double* __restrict__ part) {
    __shared__ double red[ENERGY_THREADS];
    const int s = blockIdx.y;
    const int64_t C = K * S;
    double acc = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < Kact;
         e += int64_t(gridDim.x) * blockDim.x) {
        double a[9];
        for (int k = 0; k < 9; ++k) a[k] = geo[int64_t(G_AIT + k) * K + e];
        double G[3][3];   // G = Ait^T Ait
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) G[i][j] = a[i] * a[j] + a[3 + i] * a[3 + j] + a[6 + i] * a[6 + j];
        const double vol = fabs(geo[int64_t(G_DET) * K + e]);
        const double mat[2] = {geo[int64_t(G_EPS) * K + e], geo[int64_t(G_MU) * K + e]};
        const int64_t col = e * S + s;
        double w = 0.0;
        for (int fld = 0; fld < 2; ++fld) {   // E rows c N + l, H rows 3 N + c NH + l
            double wf = 0.0;
            const int nm = fld == 0 ? N : NH;
            for (int l = 0; l < nm; ++l) {
                double v[3];
                for (int j = 0; j < 3; ++j)
                    v[j] = double(u[int64_t(fld == 0 ? j * N + l : 3 * N + j * NH + l) * C + col]);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) wf += v[i] * G[i][j] * v[j];
            }
            w += mat[fld] * wf;
        }
        acc += 0.5 * vol * w;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = ENERGY_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[int64_t(s) * gridDim.x + blockIdx.x] = red[0];
}

// Final sum per column; a non-finite energy (a NaN or an overflow anywhere in
// the column's state) latches ST_NAN in the plan's device status word.
__global__ void energy_final(const double* __restrict__ part, int nblk, int S, double* __restrict__ out,
                             int32_t* status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[int64_t(s) * nblk + b];
    out[s] = acc;
    if (!isfinite(acc)) atomicOr(status, int32_t(ST_NAN));
}

// E at receiver points: out[s][r][c] = sum_{j,l} W_r[c][j N + l] u[(j N + l)][e_r S + s],
// W_r[c][j N + l] = A^-T[c][j] phi_l(r_hat)
template <typename R>
__global__ void sample_receivers(const R* __restrict__ u, const double* __restrict__ rec, int nrec,
                                 int64_t K, int S, int N, double* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(nrec) * S) return;
    const int r = int(i / S), s = int(i % S);
    const double* w = rec + int64_t(r) * (REC_HDR + 9 * N);
    const int64_t e = int64_t(w[0]);
    const int64_t C = K * S;
    const int64_t col = e * S + s;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int jl = 0; jl < 3 * N; ++jl) {
        const double v = double(u[int64_t(jl) * C + col]);
        for (int c = 0; c < 3; ++c) acc[c] += w[REC_HDR + c * 3 * N + jl] * v;
    }
    for (int c = 0; c < 3; ++c) out[(int64_t(s) * nrec + r) * 3 + c] = acc[c];
}

// ---------------------------------------------------------------------------
extern "C" {

const char* dgm_last_error(void) { return g_err.c_str(); }

static int plan_create(dgm_plan** out, int64_t nv, const double* xyz, int64_t nt, const int64_t* tets,
                       const double* eps, const double* mu, const dgm_pml* pml,
                       const dgm_options* opt, int mixed) {
    if (!out || !opt) return fail(DGM_EINVAL, "null plan pointer or options");
    *out = nullptr;
    if (opt->n_columns < 1) return fail(DGM_EINVAL, "n_columns must be >= 1");
    if (!(opt->dt > 0.0) || !std::isfinite(opt->dt)) return fail(DGM_EINVAL, "dt must be positive");
    if (opt->flux != DGM_CENTRAL && opt->flux != DGM_UPWIND) return fail(DGM_EINVAL, "unknown flux");
    if (opt->integrator != DGM_LEAPFROG && opt->integrator != DGM_LSRK4)
        return fail(DGM_EINVAL, "unknown integrator");
    if (opt->integrator == DGM_LEAPFROG && opt->flux != DGM_CENTRAL)
        return fail(DGM_EUNSUP, "leapfrog needs the central flux");
    const int pE = mixed ? opt->p + 1 : opt->p;
    if (mixed && (pml || opt->integrator != DGM_LSRK4))
        return fail(DGM_EUNSUP, "mixed-order plans support LSRK4 without a PML");
    const KernelTable* kt = mixed ? kernel_table_mixed(pE, opt->precision)
                                  : kernel_table(opt->p, opt->precision);
    if (!kt) return fail(DGM_EUNSUP, "unsupported polynomial degree / precision");
    if (pml) {
        if (!(pml->thickness > 0.0) || !(pml->sigma_max >= 0.0) || pml->order < 0)
            return fail(DGM_EINVAL, "invalid PML parameters");
        for (int a = 0; a < 3; ++a)
            if (!(pml->hi[a] > pml->lo[a])) return fail(DGM_EINVAL, "invalid PML box");
    }
    dgm_plan* P = new dgm_plan();
    P->opt = *opt;
    P->kt = kt;
    P->mixed = mixed;
    P->pE = pE;
    P->N = nmodes(pE);
    P->NF = nfmodes(pE);
    P->NH = nmodes(opt->p);
    P->NFH = nfmodes(opt->p);
    P->has_pml = pml != nullptr;
    std::string err;
    int rc = build_mesh(nv, xyz, nt, tets, eps, mu, pml ? pml->lo : nullptr, pml ? pml->hi : nullptr,
                        pml ? pml->thickness : 1.0, pml ? pml->sigma_max : 0.0,
                        pml ? pml->order : 0, P->has_pml, P->mesh, err);
    if (rc) {
        delete P;
        return fail(rc, err);
    }
    if (build_refmats(pE, P->S, P->R, err)) {
        delete P;
        return fail(DGM_EINVAL, err);
    }
    if (mixed) {   // H's operators must be the leading submatrices of E's (hierarchical bases)
        std::vector<double> Sh, Rh;
        if (build_refmats(opt->p, Sh, Rh, err)) {
            delete P;
            return fail(DGM_EINVAL, err);
        }
        const int N = P->N, NF = P->NF, NH = P->NH, NFH = P->NFH;
        double worst = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int l = 0; l < NH; ++l)
                for (int m = 0; m < NH; ++m)
                    worst = std::fmax(worst, std::fabs(Sh[(a * NH + l) * NH + m] - P->S[(a * N + l) * N + m]));
        for (int f = 0; f < 4; ++f)
            for (int m = 0; m < NFH; ++m)
                for (int l = 0; l < NH; ++l)
                    worst = std::fmax(worst, std::fabs(Rh[(f * NFH + m) * NH + l] - P->R[(f * NF + m) * N + l]));
        if (!(worst <= 1e-12)) {
            delete P;
            return fail(DGM_EINVAL, "degree-p operators are not submatrices of degree p + 1");
        }
    }
    if (!mixed) {   // the kernels carry the reference operators as compiled literals: check them
        const double* cs = ref_S_compiled(opt->p);
        const double* cr = ref_R_compiled(opt->p);
        double worst = 0.0, scale = 0.0;
        for (size_t i = 0; i < P->S.size(); ++i) {
            worst = std::fmax(worst, std::fabs(P->S[i] - cs[i]));
            scale = std::fmax(scale, std::fabs(P->S[i]));
        }
        for (size_t i = 0; i < P->R.size(); ++i) {
            worst = std::fmax(worst, std::fabs(P->R[i] - cr[i]));
            scale = std::fmax(scale, std::fabs(P->R[i]));
        }
        if (!(worst <= 1e-13 * scale)) {
            delete P;
            return fail(DGM_EINVAL, "compiled reference operators differ from the run-time ones");
        }
    }
    const int64_t K = P->mesh.K;
    const int Sc = opt->n_columns;
    size_t off = 0;
    P->off_geo = off;
    off = align256(off + sizeof(double) * G_COUNT * K);
    P->off_geo32 = off;   // FP32 copy of the geometry for FP32 kernels
    off = align256(off + sizeof(float) * G_COUNT * K);
    P->off_fnb = off;     // per-face neighbour table, FP64 and FP32
    off = align256(off + sizeof(double) * 4 * FNB_COUNT * K);
    P->off_fnb32 = off;
    off = align256(off + sizeof(float) * 4 * FNB_COUNT * K);
    P->off_nbr = off;
    off = align256(off + sizeof(int32_t) * 4 * K);
    P->off_pml = off;
    off = align256(off + sizeof(int32_t) * K);
    P->off_src = off;
    off = align256(off + sizeof(double) * size_t(Sc) * (SRC_HDR + 3 * P->N));
    P->off_part = off;
    off = align256(off + sizeof(double) * (size_t(Sc) * ENERGY_BLOCKS + Sc));
    P->off_status = off;
    off = align256(off + 64);
    P->off_time = off;   // device clock used by graph replays (dgm_batch)
    off = align256(off + 64);
    if (opt->max_receivers < 0) {
        delete P;
        return fail(DGM_EINVAL, "max_receivers must be >= 0");
    }
    P->off_rec = off;
    off = align256(off + sizeof(double) * size_t(opt->max_receivers) * (REC_HDR + 9 * P->N));
    // operator image of the tensor-core stage variant (FP32, p = 2, 3)
    P->bytes_tcb = (opt->precision == DGM_FP32 && !mixed) ? tc_image_bytes(opt->p) : 0;
    P->off_tcb = off;
    off = align256(off + P->bytes_tcb);
    // dense reference operators of a mixed-order plan (S then R, degree p + 1)
    P->bytes_ops = mixed ? (P->S.size() + P->R.size()) * size_t(kt->real_size) : 0;
    P->off_ops = off;
    off = align256(off + P->bytes_ops);
    // incident plane wave: FP64 table and per-stage jump terms, sized for every boundary face
    for (int64_t i = 0; i < 4 * K; ++i) P->n_bfaces += P->mesh.nbr[i] < 0;
    P->inc_nq = (pE + 6) * (pE + 6);
    P->off_inc = off;
    if (!mixed) {
        off = align256(off + sizeof(double) * (INC_HDR + size_t(P->inc_nq) * (2 + P->NF) +
                                               size_t(INC_FACE) * P->n_bfaces));
        P->off_incv = off;   // jump terms: one slot per LSRK stage of a step
        off = align256(off + INC_SLOTS * inc_slot_bytes(P));
    }
    P->nbr_plain = P->mesh.nbr;
    P->off_sfid = off;   // facet codes of the interior penalty
    off = align256(off + sizeof(int32_t) * 4 * K);
    P->off_fcp = off;    // precomputed face constants of the stage kernels
    off = align256(off + size_t(kt->real_size) * FC_ROWS * K);
    P->off_tmap = off;   // tensor maps of the phase-1 bulk copies
    off = align256(off + size_t(TMAP_SETS) * TMAP_COUNT * TMAP_BYTES);
    P->bytes_geom = off;
    P->k_active = K;
    P->src_host.assign(size_t(Sc) * (SRC_HDR + 3 * P->N), 0.0);
    for (int s = 0; s < Sc; ++s) P->src_host[size_t(s) * (SRC_HDR + 3 * P->N)] = -1.0;
    *out = P;
    return DGM_OK;
}

int dgm_plan_create(dgm_plan** out, int64_t nv, const double* xyz, int64_t nt, const int64_t* tets,
                    const double* eps, const double* mu, const dgm_pml* pml,
                    const dgm_options* opt) {
    return plan_create(out, nv, xyz, nt, tets, eps, mu, pml, opt, 0);
}

int dgm_plan_create_mixed(dgm_plan** out, int64_t nv, const double* xyz, int64_t nt,
                          const int64_t* tets, const double* eps, const double* mu,
                          const dgm_pml* pml, const dgm_options* opt) {
    return plan_create(out, nv, xyz, nt, tets, eps, mu, pml, opt, 1);
}

void dgm_plan_destroy(dgm_plan* plan) { delete plan; }

int dgm_plan_info(const dgm_plan* P, dgm_info* out) {
    if (!P || !out) return fail(DGM_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->K = P->mesh.K;
    out->n_pml = P->mesh.npml;
    out->N = P->N;
    out->NF = P->NF;
    out->S = P->opt.n_columns;
    out->real_size = P->kt->real_size;
    out->bytes_fields = size_t(3) * (P->N + P->NH) * P->mesh.K * P->opt.n_columns * P->kt->real_size;
    out->bytes_aux = size_t(6) * P->N * P->mesh.npml * P->opt.n_columns * P->kt->real_size;
    out->bytes_geom = P->bytes_geom;
    out->n_quad = (P->pE + 3) * (P->pE + 3) * (P->pE + 3);
    out->N_H = P->NH;
    out->n_facets = P->n_facets;
    out->bytes_facets = size_t(P->n_facets) * P->opt.n_columns * 3 * P->NF * P->kt->real_size;
    return DGM_OK;
}

// Per-face neighbour table (FnbSlot) from the FP64 geometry, in FP64 and FP32.
__global__ void face_table_kernel(const double* __restrict__ geo, const int32_t* __restrict__ nbr,
                                  int64_t K, double* __restrict__ t64, float* __restrict__ t32) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= 4 * K) return;
    const int f = int(i / K);
    const int64_t e = i - int64_t(f) * K;
    const int32_t code = nbr[i];
    const int64_t src = (code >= 0 && (code >> 2) < K) ? int64_t(code >> 2) : e;
    for (int k = 0; k < 9; ++k) {
        const double v = geo[int64_t(G_AIT + k) * K + src];
        t64[int64_t(f * FNB_COUNT + FNB_AIT + k) * K + e] = v;
        t32[int64_t(f * FNB_COUNT + FNB_AIT + k) * K + e] = float(v);
    }
    const double z = sqrt(geo[int64_t(G_MU) * K + src] / geo[int64_t(G_EPS) * K + src]);
    t64[int64_t(f * FNB_COUNT + FNB_Z) * K + e] = z;
    t32[int64_t(f * FNB_COUNT + FNB_Z) * K + e] = float(z);
    const int gs[3] = {G_DET, G_EPS, G_MU};
    for (int k = 0; k < 3; ++k) {
        const double v = geo[int64_t(gs[k]) * K + src];
        t64[int64_t(f * FNB_COUNT + FNB_DET + k) * K + e] = v;
        t32[int64_t(f * FNB_COUNT + FNB_DET + k) * K + e] = float(v);
    }
}

static void stage_params(dgm_plan* P, StageParams& prm);

// The per-face neighbour table and, from it, the stage kernels' precomputed
// face constants (after binding, and whenever materials or boundary codes change).
// The driver's tensor-map encoder, looked up once through the runtime (null
// when the driver does not provide it; the stage kernels then load per thread).
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();   // a failed lookup must not surface at the next launch check
    });
    return fn;
}

// Tensor maps of the stage kernels' phase-1 bulk copies (TmapIndex), for the
// bound field buffers, the element constants and the face-constant table.
// Built when each element has one column (S = 1: a tile's columns are
// consecutive elements in every table) and every row starts on a 16-byte
// boundary; otherwise, or when the driver has no encoder, the kernels keep
// their per-thread loads.  The maps hold addresses only, so they stay valid
// until the next bind.
static_assert(sizeof(CUtensorMap) == TMAP_BYTES, "tensor-map slot size");

// tile width of a tensor-map set: rows of 128 bytes (set 0), 16 FP32 columns
// (set 1, FP32 plans only); 0 when the set does not exist for the plan
static cuuint32_t tmap_tile(const dgm_plan* P, int set) {
    const int rs = P->kt->real_size;
    return set == 0 ? cuuint32_t(128 / rs) : (rs == 4 ? 16u : 0u);
}

static bool tmap_encode(const dgm_plan* P, CUtensorMap* out, void* base, cuuint32_t rank,
                        const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tmap_encoder();
    const cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        P->kt->real_size == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return encode != nullptr &&
           encode(out, dt, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the field-shaped buffer `base` ([6][N][C], C = K) into map `slot` of every
// set of the host copy; false if a buffer is misaligned or the encoder refuses
static bool tmap_fields(dgm_plan* P, void* base, int slot) {
    if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
    const cuuint64_t row = cuuint64_t(P->mesh.K) * cuuint64_t(P->kt->real_size);
    const cuuint64_t dims[3] = {cuuint64_t(P->mesh.K), cuuint64_t(P->N), 6};
    const cuuint64_t str[2] = {row, row * cuuint64_t(P->N)};
    for (int set = 0; set < TMAP_SETS; ++set) {
        const cuuint32_t te = tmap_tile(P, set);
        if (te == 0) continue;
        const cuuint32_t box[3] = {te, cuuint32_t(P->N), 6};
        if (!tmap_encode(P, &P->tmap_host[size_t(set) * TMAP_COUNT + slot], base, 3, dims, str, box))
            return false;
    }
    return true;
}

// upload the host copy of the maps (on the plan's stream; the host copy lives
// in the plan, so it outlasts the copy)
static int tmap_upload(dgm_plan* P) {
    cudaError_t e = cudaMemcpyAsync(P->geom + P->off_tmap, P->tmap_host.data(),
                                    P->tmap_host.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                                    P->stream);
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "upload tensor maps");
}

// Tensor maps of the stage kernels' phase-1 bulk copies (TmapIndex), for the
// bound field buffers, the element constants and the face-constant table.
// Built when each element has one column (S = 1: a tile's columns are
// consecutive elements in every table) and every row starts on a 16-byte
// boundary; otherwise, or when the driver has no encoder, the kernels keep
// their per-thread loads.  The maps hold addresses only, so they stay valid
// until the next bind.
static int build_tmaps(dgm_plan* P) {
    P->tmaps_ok = false;
    const int rs = P->kt->real_size;
    const int64_t K = P->mesh.K;
    // (mixed-order plans run their own kernel on fields of 3 (N + N_H) rows)
    if (P->mixed || P->opt.n_columns != 1 || K <= 0 || (K * rs) % 16 != 0 || K >= (int64_t(1) << 31))
        return DGM_OK;
    if (tmap_encoder() == nullptr) return DGM_OK;
    P->tmap_host.assign(size_t(TMAP_SETS) * TMAP_COUNT, CUtensorMap{});
    for (int b = 0; b < 2; ++b)
        if (P->fields[b] != nullptr && !tmap_fields(P, P->fields[b], TM_U0 + b)) return DGM_OK;
    const cuuint64_t Ke = cuuint64_t(K), row = cuuint64_t(K) * cuuint64_t(rs);   // row stride in bytes
    unsigned char* geo = P->geom + (rs == 8 ? P->off_geo : P->off_geo32);
    unsigned char* fcp = P->geom + P->off_fcp;
    for (int set = 0; set < TMAP_SETS; ++set) {
        const cuuint32_t te = tmap_tile(P, set);
        if (te == 0) continue;
        CUtensorMap* m = P->tmap_host.data() + size_t(set) * TMAP_COUNT;
        bool ok = true;
        {   // element constants [G_COUNT][K]
            const cuuint64_t dims[2] = {Ke, cuuint64_t(G_COUNT)};
            const cuuint32_t box[2] = {te, cuuint32_t(TM_ROWS_EG)};
            ok = ok && tmap_encode(P, &m[TM_GEO], geo, 2, dims, &row, box);
        }
        {   // face constants [4][16][K]: 15 rows per face, 16 with the penalty
            const cuuint64_t dims[3] = {Ke, cuuint64_t(TM_ROWS_FACE), 4};
            const cuuint64_t str[2] = {row, row * cuuint64_t(TM_ROWS_FACE)};
            const cuuint32_t box[3] = {te, cuuint32_t(TM_ROWS_FC), 4};
            const cuuint32_t boxs[3] = {te, cuuint32_t(TM_ROWS_FACE), 4};
            ok = ok && tmap_encode(P, &m[TM_FC], fcp, 3, dims, str, box);
            ok = ok && tmap_encode(P, &m[TM_FCS], fcp, 3, dims, str, boxs);
        }
        {   // metric (and A^T) rows of the table [FC_ROWS][K], from row 4 * 16
            const cuuint64_t dims[2] = {Ke, cuuint64_t(FC_ROWS)};
            const cuuint32_t box[2] = {te, cuuint32_t(TM_ROWS_GM)};
            const cuuint32_t boxs[2] = {te, cuuint32_t(TM_ROWS_GM + TM_ROWS_GA)};
            ok = ok && tmap_encode(P, &m[TM_GM], fcp, 2, dims, &row, box);
            ok = ok && tmap_encode(P, &m[TM_GMGA], fcp, 2, dims, &row, boxs);
        }
        if (!ok) return DGM_OK;   // a shape the encoder refuses: per-thread loads
    }
    if (int rc = tmap_upload(P)) return rc;
    P->tmaps_ok = true;
    return DGM_OK;
}

static int build_face_table(dgm_plan* P) {
    const int64_t K = P->mesh.K;
    if (K == 0) return DGM_OK;
    const unsigned grid = unsigned((4 * K + 255) / 256);
    face_table_kernel<<<grid, 256, 0, P->stream>>>(
        reinterpret_cast<const double*>(P->geom + P->off_geo),
        reinterpret_cast<const int32_t*>(P->geom + P->off_nbr), K,
        reinterpret_cast<double*>(P->geom + P->off_fnb), reinterpret_cast<float*>(P->geom + P->off_fnb32));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "face table");
    if (P->mixed) return DGM_OK;   // the mixed-order kernel forms its face terms itself
    StageParams prm;
    stage_params(P, prm);
    const bool sip = P->sip_alpha > 0.0;
    prm.sfid = sip ? reinterpret_cast<const int32_t*>(P->geom + P->off_sfid) : nullptr;
    const int rc = launch_face_consts(prm, P->kt->real_size, sip, P->geom + P->off_fcp, P->stream);
    return rc ? fail(rc, "face constants") : DGM_OK;
}

int dgm_bind(dgm_plan* P, void* geom, void* fields0, void* fields1, void* res, void* aux0,
             void* aux1, void* aux_res, void* stream) {
    if (!P || !geom || !fields0) return fail(DGM_EINVAL, "null plan, geometry or field buffer");
    if (reinterpret_cast<uintptr_t>(geom) % 256) return fail(DGM_EINVAL, "geometry buffer must be 256-byte aligned");
    if (P->opt.integrator == DGM_LSRK4 && (!fields1 || !res))
        return fail(DGM_EINVAL, "LSRK4 needs fields1 and res");
    if (P->has_pml && P->mesh.npml > 0 && (!aux0 || (P->opt.integrator == DGM_LSRK4 && (!aux1 || !aux_res))))
        return fail(DGM_EINVAL, "PML plan needs auxiliary buffers");
    cudaError_t e = cudaGetDevice(&P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    P->geom = static_cast<unsigned char*>(geom);
    P->fields[0] = fields0;
    P->fields[1] = fields1;
    P->res = res;
    P->aux[0] = aux0;
    P->aux[1] = aux1;
    P->aux_res = aux_res;
    P->stream = static_cast<cudaStream_t>(stream);
    P->cur = 0;
    const int64_t K = P->mesh.K;
    cudaStream_t st = P->stream;
    if ((e = cudaMemcpyAsync(P->geom + P->off_geo, P->mesh.geo.data(), sizeof(double) * G_COUNT * K,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload geometry");
    {
        std::vector<float> g32(P->mesh.geo.begin(), P->mesh.geo.end());
        if ((e = cudaMemcpyAsync(P->geom + P->off_geo32, g32.data(), sizeof(float) * G_COUNT * K,
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "upload geometry (FP32)");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "bind sync");
    }
    if ((e = cudaMemcpyAsync(P->geom + P->off_nbr, P->mesh.nbr.data(), sizeof(int32_t) * 4 * K,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload neighbours");
    if ((e = cudaMemcpyAsync(P->geom + P->off_pml, P->mesh.pml_idx.data(), sizeof(int32_t) * K,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload PML index");
    if ((e = cudaMemcpyAsync(P->geom + P->off_src, P->src_host.data(),
                             sizeof(double) * P->src_host.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e, "upload sources");
    if ((e = cudaMemsetAsync(P->geom + P->off_status, 0, 64, st)) != cudaSuccess)
        return cuda_fail(e, "clear status");
    std::vector<unsigned char> tcimg;
    if (P->bytes_tcb) {
        build_tc_image(P->opt.p, P->S, P->R, tcimg);
        if ((e = cudaMemcpyAsync(P->geom + P->off_tcb, tcimg.data(), tcimg.size(),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "upload tensor-core operator image");
    }
    std::vector<unsigned char> ops(P->bytes_ops);
    if (P->bytes_ops) {
        const size_t n = P->S.size() + P->R.size();
        for (size_t i = 0; i < n; ++i) {
            const double v = i < P->S.size() ? P->S[i] : P->R[i - P->S.size()];
            if (P->kt->real_size == 8) std::memcpy(ops.data() + 8 * i, &v, 8);
            else { const float f = float(v); std::memcpy(ops.data() + 4 * i, &f, 4); }
        }
        if ((e = cudaMemcpyAsync(P->geom + P->off_ops, ops.data(), ops.size(), cudaMemcpyHostToDevice,
                                 st)) != cudaSuccess)
            return cuda_fail(e, "upload mixed-order operators");
    }
    if (P->n_inc > 0 &&
        (e = cudaMemcpyAsync(P->geom + P->off_inc, P->inc_host.data(), sizeof(double) * P->inc_host.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload incident table");
    if (P->sip_alpha > 0.0 &&
        (e = cudaMemcpyAsync(P->geom + P->off_sfid, P->sfid_host.data(), sizeof(int32_t) * 4 * K,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "upload facet codes");
    if (int rc = build_face_table(P)) return rc;
    if (int rc = build_tmaps(P)) return rc;
    // the host copies above are pageable: finish them before the host vectors can change
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "bind sync");
    P->bound = true;
    return DGM_OK;
}

static void stage_params(dgm_plan* P, StageParams& prm) {
    std::memset(&prm, 0, sizeof(prm));
    prm.geo = reinterpret_cast<const double*>(P->geom + P->off_geo);
    prm.geo_r = P->kt->real_size == 8 ? static_cast<const void*>(P->geom + P->off_geo)
                                      : static_cast<const void*>(P->geom + P->off_geo32);
    prm.nbr = reinterpret_cast<const int32_t*>(P->geom + P->off_nbr);
    prm.fnb_r = P->kt->real_size == 8 ? static_cast<const void*>(P->geom + P->off_fnb)
                                      : static_cast<const void*>(P->geom + P->off_fnb32);
    prm.pml = P->has_pml ? reinterpret_cast<const int32_t*>(P->geom + P->off_pml) : nullptr;
    prm.src = P->have_src ? reinterpret_cast<const double*>(P->geom + P->off_src) : nullptr;
    prm.status = reinterpret_cast<int32_t*>(P->geom + P->off_status);
    prm.K = P->mesh.K;
    prm.npml = P->mesh.npml;
    prm.S = P->opt.n_columns;
    prm.upwind = P->opt.flux == DGM_UPWIND;
    prm.dt = P->opt.dt;
    prm.variant = P->variant;
    prm.force_index64 = P->force_index64;
    prm.tile_groups = P->tile_groups;
    prm.tc_b = P->bytes_tcb ? static_cast<const void*>(P->geom + P->off_tcb) : nullptr;
    prm.K_active = P->k_active;
    prm.ops = P->bytes_ops ? static_cast<const void*>(P->geom + P->off_ops) : nullptr;
    prm.inc = P->n_inc > 0 ? static_cast<const void*>(P->geom + P->off_incv) : nullptr;
    prm.sip_alpha = P->sip_alpha;
    prm.n_facets = P->n_facets;
    prm.fcp = P->geom + P->off_fcp;
    if (P->tmaps_ok && P->tile_loads == 0) {   // phase-1 bulk copies (the launchers pick the map)
        prm.tmaps = P->geom + P->off_tmap;
        prm.tm_f0 = P->fields[0];
        prm.tm_f1 = P->fields[1];
    }
    prm.tm_u = -1;
    if (P->sip_alpha > 0.0 && P->hs[0] != nullptr) {
        prm.sfid = reinterpret_cast<const int32_t*>(P->geom + P->off_sfid);
        prm.hs = P->hs[P->cur];
        prm.hs_out = P->hs[1 - P->cur];
        prm.hs_res = P->hs_res;
    }
}

// The facet buffers of one LSRK stage: input of the current state, output the other.
static void sip_stage(const dgm_plan* P, StageParams& prm) {
    if (prm.hs == nullptr) return;
    prm.hs = P->hs[P->cur];
    prm.hs_out = P->hs[1 - P->cur];
}

}  // extern "C"

// Incident plane-wave table (FP64, in the geometry buffer):
//   [0, INC_HDR)  header: f0, bw, t0, nq, n_faces, 0, 0, 0
//   then the face rule: (s_q, t_q) (2 nq values), W[m][q] = w_q psi_m(s_q, t_q)
//       (NF nq values; the parametrisation of the trace operators)
//   then per incident face i (INC_FACE values): A^T E0 (the polarisation's
//       covariant components in the face's element), and tau_q = c0 + s_q cs + t_q ct,
//       the plane-wave delay d . r_q / speed, linear on the face
// incident_eval writes, for the stage time t, v[i][m][r] = 2 (A^T E0)_r s_m(t) with
//   s_m(t) = sum_q W[m][q] g(t - t0 - tau_q),  g(x) = cos(2 pi f0 x) exp(-x^2 / (2 s^2)),
//   s = 1 / (2 pi bw): the face-mode traces of the E jump 2 E_inc (e+ = e- + 2 E_inc).
// One warp per face: the lanes take the rule's points, then reduce per mode.
// The delay x = t - t0 - tau_q is formed in FP64 (t may be large against the
// pulse width); the pulse and the sums run in the plan's precision (an FP32
// plan rounds the jump terms to FP32 anyway).
struct IncTimes {
    double t[INC_SLOTS];
};
template <typename R>
__global__ void incident_eval(const double* __restrict__ tab, int NF, IncTimes ts, int64_t slot,
                              R* __restrict__ out) {
    const double t = ts.t[blockIdx.y];
    out += int64_t(blockIdx.y) * slot;
    const int lane = threadIdx.x & 31;
    const int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nf = int64_t(tab[4]);
    if (i >= nf) return;
    const double twopi = 6.283185307179586476925286766559;
    const R f0 = R(tab[0]), sg = R(1.0 / (twopi * tab[1]));
    const double t0 = tab[2];
    const int nq = int(tab[3]);
    const double* pts = tab + INC_HDR;
    const double* W = pts + 2 * nq;
    const double* fc = W + int64_t(NF) * nq + i * INC_FACE;
    R g[INC_MAXQ / 32];
#pragma unroll
    for (int k = 0; k < INC_MAXQ / 32; ++k) {
        const int q = lane + 32 * k;
        g[k] = R(0);
        if (q < nq) {
            const R x = R(t - t0 - (fc[3] + pts[2 * q] * fc[4] + pts[2 * q + 1] * fc[5]));
            g[k] = cos(R(twopi) * f0 * x) * exp(-x * x / (R(2) * sg * sg));
        }
    }
    for (int m = 0; m < NF; ++m) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < INC_MAXQ / 32; ++k) {
            const int q = lane + 32 * k;
            if (q < nq) acc += R(W[int64_t(m) * nq + q]) * g[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane < 3) out[(i * NF + m) * 3 + lane] = R(2) * R(fc[lane]) * acc;
    }
}

// The incident jump terms at n (<= INC_SLOTS) times, into slots 0 .. n-1: one
// launch for the five stages of an LSRK step.
static int incident_eval_times(dgm_plan* P, const double* t, int n, cudaStream_t st) {
    IncTimes ts{};
    for (int k = 0; k < n; ++k) ts.t[k] = t[k];
    const double* tab = reinterpret_cast<const double*>(P->geom + P->off_inc);
    const dim3 grid(unsigned((P->n_inc + 3) / 4), unsigned(n));
    const int64_t slot = int64_t(P->n_inc) * P->NF * 3;   // reals per slot in use
    if (P->kt->real_size == 8)
        incident_eval<double><<<grid, 128, 0, st>>>(tab, P->NF, ts, slot,
                                                     reinterpret_cast<double*>(P->geom + P->off_incv));
    else
        incident_eval<float><<<grid, 128, 0, st>>>(tab, P->NF, ts, slot,
                                                    reinterpret_cast<float*>(P->geom + P->off_incv));
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

// A stage launch.  With incident faces the kernel reads the jump terms of
// `slot`, evaluated by the caller for this stage's time; slot < 0 evaluates
// them here at prm.t (into slot 0).
static int launch_stage(dgm_plan* P, StageParams& prm, int mode, cudaStream_t st, int slot = -1) {
    if (P->n_inc > 0) {
        if (slot < 0) {
            if (int rc = incident_eval_times(P, &prm.t, 1, st)) return rc;
            slot = 0;
        }
        prm.inc = P->geom + P->off_incv +
                  size_t(slot) * size_t(P->n_inc) * P->NF * 3 * size_t(P->kt->real_size);
    }
    return P->kt->launch_stage(prm, mode, st);
}

// The paired FP32 stage kernels (variants 3 and 4 up to p = 3) have neither
// incident faces nor the interior penalty.
static bool variant_has_incident(const dgm_plan* P, int v) {
    return !(P->kt->real_size == 4 && P->opt.p <= 3 && (v == 3 || v == 4));
}
static bool needs_single_column_kernel(const dgm_plan* P) { return P->n_inc > 0 || P->sip_alpha > 0.0; }
// The interior penalty is instantiated for the default tile shape only.
static bool variant_ok(const dgm_plan* P, int v) {
    if (P->sip_alpha > 0.0 && v != 0) return false;
    return !needs_single_column_kernel(P) || variant_has_incident(P, v);
}

extern "C" {

int dgm_set_sources(dgm_plan* P, int32_t n, const int32_t* column, const double* pos,
                    const double* dir, const double* f0, const double* bw, const double* t0) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (n < 0 || (n > 0 && (!column || !pos || !dir || !f0 || !bw || !t0)))
        return fail(DGM_EINVAL, "invalid source arrays");
    const int N = P->N;
    const size_t rec = SRC_HDR + 3 * N;
    const int64_t K = P->mesh.K;
    std::vector<double> host(P->src_host.size(), 0.0);
    for (int s = 0; s < P->opt.n_columns; ++s) host[s * rec] = -1.0;
    for (int i = 0; i < n; ++i) {
        const int s = column[i];
        if (s < 0 || s >= P->opt.n_columns) return fail(DGM_EINVAL, "source column out of range");
        if (host[s * rec] >= 0.0) return fail(DGM_EINVAL, "one source per column");
        if (!(bw[i] > 0.0)) return fail(DGM_EINVAL, "source bandwidth must be positive");
        const double* r = pos + 3 * i;
        int64_t found = -1;
        double xr[3];
        for (int64_t e = 0; e < K && found < 0; ++e) {
            const double* V = &P->mesh.verts[12 * e];
            double d[3] = {r[0] - V[0], r[1] - V[1], r[2] - V[2]};
            double lam[3];
            for (int a = 0; a < 3; ++a)   // r_hat = A^-1 (r - v0), A^-1[a][c] = Ait[c][a]
                lam[a] = P->mesh.geo[(G_AIT + 3 * 0 + a) * K + e] * d[0] +
                         P->mesh.geo[(G_AIT + 3 * 1 + a) * K + e] * d[1] +
                         P->mesh.geo[(G_AIT + 3 * 2 + a) * K + e] * d[2];
            const double tol = 1e-12;
            if (lam[0] >= -tol && lam[1] >= -tol && lam[2] >= -tol && lam[0] + lam[1] + lam[2] <= 1 + tol) {
                found = e;
                for (int a = 0; a < 3; ++a) xr[a] = lam[a];
            }
        }
        if (found < 0) return fail(DGM_EINVAL, "source point outside the mesh");
        double* out = &host[s * rec];
        out[0] = double(found);
        out[1] = f0[i];
        out[2] = bw[i];
        out[3] = t0[i];
        std::vector<double> phi(N);
        ref_basis_values(P->pE, xr, phi.data());
        // w_{j,l} = dir . (A^-T e_j) phi_l(r_hat) = sum_c Ait[c][j] dir_c phi_l
        for (int j = 0; j < 3; ++j) {
            double dj = 0.0;
            for (int cc = 0; cc < 3; ++cc) dj += P->mesh.geo[(G_AIT + 3 * cc + j) * K + found] * dir[3 * i + cc];
            for (int l = 0; l < N; ++l) out[SRC_HDR + j * N + l] = dj * phi[l];
        }
    }
    P->src_host = host;
    P->have_src = n > 0;
    cudaError_t e = cudaMemcpyAsync(P->geom + P->off_src, P->src_host.data(),
                                    sizeof(double) * P->src_host.size(), cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload sources");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "source sync");
    return DGM_OK;
}

// lowest-index element containing r (barycentric >= -1e-12); fills reference coordinates
static int64_t locate_point(const dgm_plan* P, const double* r, double xr[3]) {
    const int64_t K = P->mesh.K;
    for (int64_t e = 0; e < K; ++e) {
        const double* V = &P->mesh.verts[12 * e];
        double d[3] = {r[0] - V[0], r[1] - V[1], r[2] - V[2]};
        double lam[3];
        for (int a = 0; a < 3; ++a)   // r_hat = A^-1 (r - v0), A^-1[a][c] = A^-T[c][a]
            lam[a] = P->mesh.geo[(G_AIT + 3 * 0 + a) * K + e] * d[0] +
                     P->mesh.geo[(G_AIT + 3 * 1 + a) * K + e] * d[1] +
                     P->mesh.geo[(G_AIT + 3 * 2 + a) * K + e] * d[2];
        const double tol = 1e-12;
        if (lam[0] >= -tol && lam[1] >= -tol && lam[2] >= -tol && lam[0] + lam[1] + lam[2] <= 1 + tol) {
            for (int a = 0; a < 3; ++a) xr[a] = lam[a];
            return e;
        }
    }
    return -1;
}

int dgm_set_receivers(dgm_plan* P, int32_t n, const double* pos) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (n < 0 || n > P->opt.max_receivers || (n > 0 && !pos))
        return fail(DGM_EINVAL, "receiver count exceeds max_receivers or null positions");
    const int N = P->N;
    const int64_t K = P->mesh.K;
    const size_t rec = REC_HDR + 9 * N;
    std::vector<double> host(size_t(n) * rec, 0.0), phi(N);
    for (int i = 0; i < n; ++i) {
        double xr[3];
        const int64_t e = locate_point(P, pos + 3 * i, xr);
        if (e < 0) return fail(DGM_EINVAL, "receiver point outside the mesh");
        double* w = &host[i * rec];
        w[0] = double(e);
        ref_basis_values(P->pE, xr, phi.data());
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < N; ++l)
                    w[REC_HDR + c * 3 * N + j * N + l] = P->mesh.geo[(G_AIT + 3 * c + j) * K + e] * phi[l];
    }
    P->n_rec = n;
    if (n == 0) return DGM_OK;
    cudaError_t e = cudaMemcpyAsync(P->geom + P->off_rec, host.data(), sizeof(double) * host.size(),
                                    cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload receivers");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "receiver sync");
    return DGM_OK;
}

int dgm_sample_receivers(dgm_plan* P, const void* fields, double* out_device) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!fields || !out_device) return fail(DGM_EINVAL, "null argument");
    if (P->n_rec == 0) return DGM_OK;
    const int64_t n = int64_t(P->n_rec) * P->opt.n_columns;
    const double* rec = reinterpret_cast<const double*>(P->geom + P->off_rec);
    const unsigned grid = unsigned((n + 127) / 128);
    if (P->kt->real_size == 8)
        sample_receivers<double><<<grid, 128, 0, P->stream>>>(static_cast<const double*>(fields), rec,
                                                              P->n_rec, P->mesh.K, P->opt.n_columns,
                                                              P->N, out_device);
    else
        sample_receivers<float><<<grid, 128, 0, P->stream>>>(static_cast<const float*>(fields), rec,
                                                             P->n_rec, P->mesh.K, P->opt.n_columns,
                                                             P->N, out_device);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "receiver kernel launch");
}

int dgm_rhs(dgm_plan* P, const void* fields, const void* aux, void* dfields, void* daux, double t) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->sip_alpha > 0.0 && P->hs[0] == nullptr)
        return fail(DGM_ESTATE, "facet buffers of the interior penalty not bound (dgm_bind_sip)");
    if (!fields || !dfields) return fail(DGM_EINVAL, "null field buffer");
    if (P->has_pml && P->mesh.npml > 0 && (!aux || !daux)) return fail(DGM_EINVAL, "PML plan needs aux/daux");
    StageParams prm;
    stage_params(P, prm);
    prm.u = fields;
    prm.u_out = dfields;
    prm.aux = aux;
    prm.aux_out = daux;
    prm.t = t;
    if (prm.hs != nullptr) prm.hs_out = P->hs_res;   // dh_s/dt of the current facet field
    int rc = launch_stage(P, prm, MODE_RHS, P->stream);
    return rc ? fail(rc, "stage kernel launch failed") : DGM_OK;
}

int dgm_leapfrog_start(dgm_plan* P, double t0) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->opt.integrator != DGM_LEAPFROG) return fail(DGM_ESTATE, "not a leapfrog plan");
    StageParams prm;
    stage_params(P, prm);
    prm.u = P->fields[P->cur];
    prm.u_out = P->fields[P->cur];
    prm.aux = P->aux[P->cur];       // PML auxiliaries, updated in place
    prm.aux_out = P->aux[P->cur];
    prm.dt = 0.5 * P->opt.dt;
    prm.t = t0;
    int rc = launch_stage(P, prm, MODE_LF_H, P->stream);
    return rc ? fail(rc, "stage kernel launch failed") : DGM_OK;
}

int dgm_advance(dgm_plan* P, int64_t n_steps, double t0) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->sip_alpha > 0.0 && P->hs[0] == nullptr)
        return fail(DGM_ESTATE, "facet buffers of the interior penalty not bound (dgm_bind_sip)");
    if (n_steps < 0) return fail(DGM_EINVAL, "negative step count");
    StageParams prm;
    stage_params(P, prm);
    const double dt = P->opt.dt;
    for (int64_t n = 0; n < n_steps; ++n) {
        const double t = t0 + double(n) * dt;
        if (P->opt.integrator == DGM_LSRK4) {
            if (P->n_inc > 0) {   // the step's five stage times in one launch
                double ts[5];
                for (int k = 0; k < 5; ++k) ts[k] = t + LSRK_C[k] * dt;
                if (int rc = incident_eval_times(P, ts, 5, P->stream)) return fail(rc, "incident launch failed");
            }
            for (int k = 0; k < 5; ++k) {
                prm.u = P->fields[P->cur];
                prm.u_out = P->fields[1 - P->cur];
                prm.res = P->res;
                prm.aux = P->aux[P->cur];
                prm.aux_out = P->aux[1 - P->cur];
                prm.aux_res = P->aux_res;
                prm.t = t + LSRK_C[k] * dt;
                prm.a = LSRK_A[k];
                prm.b = LSRK_B[k];
                sip_stage(P, prm);
                int rc = launch_stage(P, prm, MODE_LSRK, P->stream, k);
                if (rc) return fail(rc, "stage kernel launch failed");
                P->cur = 1 - P->cur;
            }
        } else {
            prm.u = P->fields[P->cur];
            prm.u_out = P->fields[P->cur];
            prm.aux = P->aux[P->cur];   // PML auxiliaries, updated in place
            prm.aux_out = P->aux[P->cur];
            prm.t = t + 0.5 * dt;
            int rc = launch_stage(P, prm, MODE_LF_E, P->stream);
            if (rc) return fail(rc, "stage kernel launch failed");
            prm.t = t + dt;
            rc = launch_stage(P, prm, MODE_LF_H, P->stream);
            if (rc) return fail(rc, "stage kernel launch failed");
        }
    }
    return DGM_OK;
}

int dgm_current(const dgm_plan* P) { return P ? P->cur : -1; }

int dgm_stage(dgm_plan* P, int32_t k, double t) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->sip_alpha > 0.0 && P->hs[0] == nullptr)
        return fail(DGM_ESTATE, "facet buffers of the interior penalty not bound (dgm_bind_sip)");
    if (P->opt.integrator != DGM_LSRK4) return fail(DGM_ESTATE, "dgm_stage needs an LSRK4 plan");
    if (k < 0 || k > 4) return fail(DGM_EINVAL, "stage index must be 0..4");
    StageParams prm;
    stage_params(P, prm);
    const double dt = P->opt.dt;
    prm.u = P->fields[P->cur];
    prm.u_out = P->fields[1 - P->cur];
    prm.res = P->res;
    prm.aux = P->aux[P->cur];
    prm.aux_out = P->aux[1 - P->cur];
    prm.aux_res = P->aux_res;
    prm.t = t + LSRK_C[k] * dt;
    prm.a = LSRK_A[k];
    prm.b = LSRK_B[k];
    sip_stage(P, prm);
    int rc = launch_stage(P, prm, MODE_LSRK, P->stream);
    if (rc) return fail(rc, "stage kernel launch failed");
    P->cur = 1 - P->cur;
    return DGM_OK;
}

int dgm_set_incident(dgm_plan* P, int64_t n, const int64_t* faces, const dgm_incident* w) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (n < 0) return fail(DGM_EINVAL, "negative face count");
    if (n > 0 && (!faces || !w)) return fail(DGM_EINVAL, "null faces or wave");
    if (n > 0 && P->mixed) return fail(DGM_EUNSUP, "mixed-order plans have no incident faces");
    if (n > 0 && P->opt.integrator != DGM_LSRK4) return fail(DGM_EUNSUP, "incident faces need LSRK4");
    if (n > P->n_bfaces) return fail(DGM_EINVAL, "more incident faces than boundary faces");
    const int64_t K = P->mesh.K;
    std::vector<int32_t> nbr = P->nbr_plain;
    std::vector<double> tab;
    if (n > 0) {
        bool ok = w->bw > 0.0 && w->speed > 0.0 && std::isfinite(w->bw) && std::isfinite(w->speed) &&
                  std::isfinite(w->f0) && std::isfinite(w->t0);
        for (int c = 0; c < 3; ++c) ok = ok && std::isfinite(w->E0[c]) && std::isfinite(w->direction[c]);
        if (!ok) return fail(DGM_EINVAL, "invalid incident wave parameters");
        // boundary faces by sorted vertex triple
        struct Key {
            int64_t a, b, c, id;
            bool operator<(const Key& o) const {
                return a != o.a ? a < o.a : b != o.b ? b < o.b : c != o.c ? c < o.c : id < o.id;
            }
        };
        std::vector<Key> bf;
        bf.reserve(size_t(P->n_bfaces));
        for (int64_t e = 0; e < K; ++e)
            for (int f = 0; f < 4; ++f) {
                if (P->nbr_plain[size_t(f) * K + e] >= 0) continue;
                int64_t t[3], c = 0;
                for (int i = 0; i < 4; ++i)
                    if (i != f) t[c++] = P->mesh.vid[4 * e + i];
                bf.push_back(Key{t[0], t[1], t[2], 4 * e + f});
            }
        std::sort(bf.begin(), bf.end());
        const int q1 = P->pE + 6;
        std::vector<double> pts, wq, psi;
        face_rule(P->pE, q1, pts, wq, psi);
        const int nq = int(wq.size()), NF = P->NF;
        tab.assign(INC_HDR + size_t(nq) * (2 + NF) + size_t(INC_FACE) * n, 0.0);
        tab[0] = w->f0;
        tab[1] = w->bw;
        tab[2] = w->t0;
        tab[3] = nq;
        tab[4] = double(n);
        for (int q = 0; q < nq; ++q) {
            tab[INC_HDR + 2 * q] = pts[2 * q];
            tab[INC_HDR + 2 * q + 1] = pts[2 * q + 1];
            for (int m = 0; m < NF; ++m) tab[INC_HDR + 2 * nq + size_t(m) * nq + q] = wq[q] * psi[size_t(q) * NF + m];
        }
        double* fc = tab.data() + INC_HDR + size_t(nq) * (2 + NF);
        for (int64_t i = 0; i < n; ++i) {
            int64_t v[3] = {faces[3 * i], faces[3 * i + 1], faces[3 * i + 2]};
            std::sort(v, v + 3);
            const Key k{v[0], v[1], v[2], -1};
            auto it = std::lower_bound(bf.begin(), bf.end(), k);
            if (it == bf.end() || it->a != v[0] || it->b != v[1] || it->c != v[2])
                return fail(DGM_EINVAL, "incident face " + std::to_string(i) + " is not a boundary face");
            const int64_t e = it->id / 4;
            const int f = int(it->id % 4);
            if (nbr[size_t(f) * K + e] != P->nbr_plain[size_t(f) * K + e])
                return fail(DGM_EINVAL, "incident face " + std::to_string(i) + " given twice");
            nbr[size_t(f) * K + e] = int32_t(-2 - i);
            const double* X = P->mesh.verts.data() + 12 * e;   // sorted local vertices
            int loc[3], c = 0;
            for (int j = 0; j < 4; ++j)
                if (j != f) loc[c++] = j;
            for (int j = 0; j < 3; ++j) {   // (A^T E0)_j = (X_{j+1} - X_0) . E0
                double acc = 0.0;
                for (int r = 0; r < 3; ++r) acc += (X[3 * (j + 1) + r] - X[r]) * w->E0[r];
                fc[INC_FACE * i + j] = acc;
            }
            double dpa = 0.0, dpb = 0.0, dpc = 0.0;   // d . P_a, d . (P_b - P_a), d . (P_c - P_a)
            for (int r = 0; r < 3; ++r) {
                const double pa = X[3 * loc[0] + r];
                dpa += w->direction[r] * pa;
                dpb += w->direction[r] * (X[3 * loc[1] + r] - pa);
                dpc += w->direction[r] * (X[3 * loc[2] + r] - pa);
            }
            fc[INC_FACE * i + 3] = dpa / w->speed;
            fc[INC_FACE * i + 4] = dpb / w->speed;
            fc[INC_FACE * i + 5] = dpc / w->speed;
        }
    }
    P->mesh.nbr = nbr;
    P->inc_host = tab;
    P->n_inc = n;
    if (n > 0 && !variant_has_incident(P, P->variant)) P->variant = 0;
    if (P->bound) {
        cudaStream_t st = P->stream;
        cudaError_t e = cudaMemcpyAsync(P->geom + P->off_nbr, P->mesh.nbr.data(), sizeof(int32_t) * 4 * K,
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(P->geom + P->off_inc, P->inc_host.data(), sizeof(double) * P->inc_host.size(),
                                cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "upload incident faces");
        if (int rc = build_face_table(P)) return rc;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "upload incident faces");
    }
    return DGM_OK;
}

int dgm_set_active(dgm_plan* P, int64_t n) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (n < 1 || n > P->mesh.K) return fail(DGM_EINVAL, "active element count must be in 1..K");
    if (n < P->mesh.K && P->sip_alpha > 0.0)
        return fail(DGM_EUNSUP, "the interior penalty needs every element active");
    P->k_active = n;
    return DGM_OK;
}

int dgm_set_sip(dgm_plan* P, double alpha) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(DGM_EINVAL, "alpha must be finite and >= 0");
    if (P->bound) return fail(DGM_ESTATE, "set the penalty before dgm_bind");
    if (alpha > 0.0) {
        if (P->opt.flux != DGM_CENTRAL) return fail(DGM_EUNSUP, "the interior penalty needs the central flux");
        if (P->opt.integrator != DGM_LSRK4) return fail(DGM_EUNSUP, "the interior penalty needs LSRK4");
        if (P->mixed) return fail(DGM_EUNSUP, "mixed-order plans have no interior penalty");
        if (P->has_pml) return fail(DGM_EUNSUP, "the interior penalty is not built with a PML");
        if (P->k_active < P->mesh.K) return fail(DGM_EUNSUP, "the interior penalty needs every element active");
    }
    const int64_t K = P->mesh.K;
    P->sip_alpha = alpha;
    P->n_facets = 0;
    P->sfid_host.assign(size_t(4) * K, -1);
    if (alpha == 0.0) return DGM_OK;
    // facets numbered by (lower element, its local face), ascending; the lower
    // element owns the facet (it advances h_s)
    for (int64_t e = 0; e < K; ++e)
        for (int f = 0; f < 4; ++f) {
            const int32_t code = P->nbr_plain[size_t(f) * K + e];
            if (code < 0 || int64_t(code >> 2) <= e) continue;
            const int64_t e2 = code >> 2;
            const int f2 = code & 3;
            if (P->n_facets >= (int64_t(1) << 30)) return fail(DGM_EUNSUP, "too many facets");
            P->sfid_host[size_t(f) * K + e] = int32_t((P->n_facets << 1) | 1);
            P->sfid_host[size_t(f2) * K + e2] = int32_t(P->n_facets << 1);
            ++P->n_facets;
        }
    P->variant = 0;
    return DGM_OK;
}

int dgm_bind_sip(dgm_plan* P, void* hs0, void* hs1, void* hs_res) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!(P->sip_alpha > 0.0)) return fail(DGM_ESTATE, "no interior penalty on this plan");
    if (!hs0 || !hs1 || !hs_res) return fail(DGM_EINVAL, "null facet buffer");
    P->hs[0] = P->cur == 0 ? hs0 : hs1;   // hs0 holds the current state
    P->hs[1] = P->cur == 0 ? hs1 : hs0;
    P->hs_res = hs_res;
    return DGM_OK;
}

}  // extern "C"

// Halo copies: buf[(r n + i) S + s] <-> fields[(r K + idx[i]) S + s], r = c N + l.
// An element id outside 0..K-1 is skipped and latched as ST_BAD_INDEX.
template <typename R>
__global__ void halo_copy(R* __restrict__ fields, const int64_t* __restrict__ idx, int64_t n,
                          int64_t K, int S, int rows, R* __restrict__ buf, int to_buf,
                          int32_t* status) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t per = n * S;
    if (i >= per * rows) return;
    const int64_t r = i / per, rem = i - r * per;
    const int64_t j = rem / S;
    const int s = int(rem - j * S);
    const int64_t e = idx[j];
    if (e < 0 || e >= K) {
        atomicOr(status, int32_t(ST_BAD_INDEX));
        return;
    }
    const int64_t g = (r * K + e) * S + s;
    if (to_buf) buf[i] = fields[g];
    else fields[g] = buf[i];
}

static int halo_copy_launch(dgm_plan* P, void* fields, const int64_t* idx, int64_t n, void* buf,
                            int to_buf) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (n < 0 || (n > 0 && (!fields || !idx || !buf))) return fail(DGM_EINVAL, "null halo argument");
    if (n == 0) return DGM_OK;
    const int rows = 3 * (P->N + P->NH), S = P->opt.n_columns;
    const int64_t total = n * S * rows;
    const unsigned grid = unsigned((total + 255) / 256);
    int32_t* status = reinterpret_cast<int32_t*>(P->geom + P->off_status);
    if (P->kt->real_size == 8)
        halo_copy<double><<<grid, 256, 0, P->stream>>>(static_cast<double*>(fields), idx, n, P->mesh.K,
                                                        S, rows, static_cast<double*>(buf), to_buf, status);
    else
        halo_copy<float><<<grid, 256, 0, P->stream>>>(static_cast<float*>(fields), idx, n, P->mesh.K, S,
                                                       rows, static_cast<float*>(buf), to_buf, status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "halo copy");
}

extern "C" {

int dgm_halo_pack(dgm_plan* P, const void* fields, const int64_t* idx, int64_t n, void* buf) {
    return halo_copy_launch(P, const_cast<void*>(fields), idx, n, buf, 1);
}

int dgm_halo_unpack(dgm_plan* P, void* fields, const int64_t* idx, int64_t n, const void* buf) {
    return halo_copy_launch(P, fields, idx, n, const_cast<void*>(buf), 0);
}

int dgm_advance_host(dgm_plan* P, const void* fields_in, void* fields_out, int64_t n_steps, double t0) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!fields_in || !fields_out) return fail(DGM_EINVAL, "null host buffer");
    dgm_info info;
    dgm_plan_info(P, &info);
    cudaError_t e = cudaMemcpyAsync(P->fields[P->cur], fields_in, info.bytes_fields,
                                    cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
    int rc = dgm_advance(P, n_steps, t0);
    if (rc) return rc;
    e = cudaMemcpyAsync(fields_out, P->fields[P->cur], info.bytes_fields, cudaMemcpyDeviceToHost, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
    e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return DGM_OK;
}

int dgm_energy(dgm_plan* P, const void* fields, double* out) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!fields || !out) return fail(DGM_EINVAL, "null argument");
    const int Sc = P->opt.n_columns;
    double* part = reinterpret_cast<double*>(P->geom + P->off_part);
    double* res = part + size_t(Sc) * ENERGY_BLOCKS;
    const double* geo = reinterpret_cast<const double*>(P->geom + P->off_geo);
    dim3 grid(ENERGY_BLOCKS, Sc);
    if (P->kt->real_size == 8)
        energy_partial<double><<<grid, ENERGY_THREADS, 0, P->stream>>>(
            static_cast<const double*>(fields), geo, P->mesh.K, P->k_active, Sc, P->N, P->NH, part);
    else
        energy_partial<float><<<grid, ENERGY_THREADS, 0, P->stream>>>(
            static_cast<const float*>(fields), geo, P->mesh.K, P->k_active, Sc, P->N, P->NH, part);
    energy_final<<<(Sc + 127) / 128, 128, 0, P->stream>>>(
        part, ENERGY_BLOCKS, Sc, res, reinterpret_cast<int32_t*>(P->geom + P->off_status));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    e = cudaMemcpyAsync(out, res, sizeof(double) * Sc, cudaMemcpyDeviceToHost, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "energy copy");
    e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "energy sync");
    for (int s = 0; s < Sc; ++s)
        if (!std::isfinite(out[s]))
            return fail(DGM_ENAN, "non-finite energy in column " + std::to_string(s) +
                                      " (latched in the device status word)");
    return DGM_OK;
}

int dgm_pml_elements(const dgm_plan* P, int64_t* out) {
    if (!P || (!out && P->mesh.npml > 0)) return fail(DGM_EINVAL, "null argument");
    for (int64_t e = 0; e < P->mesh.K; ++e)
        if (P->mesh.pml_idx[e] >= 0) out[P->mesh.pml_idx[e]] = e;
    return DGM_OK;
}

int dgm_quad_points(const dgm_plan* P, double* xyz_out) {
    if (!P || !xyz_out) return fail(DGM_EINVAL, "null argument");
    std::vector<double> pts, w;
    tet_rule(P->pE + 3, pts, w);
    const size_t nq = w.size();
    const int64_t K = P->mesh.K;
    for (int64_t e = 0; e < K; ++e) {
        const double* V = &P->mesh.verts[12 * e];
        for (size_t q = 0; q < nq; ++q)
            for (int a = 0; a < 3; ++a)
                xyz_out[(e * nq + q) * 3 + a] = V[a] + pts[3 * q] * (V[3 + a] - V[a]) +
                                                pts[3 * q + 1] * (V[6 + a] - V[a]) +
                                                pts[3 * q + 2] * (V[9 + a] - V[a]);
    }
    return DGM_OK;
}

int dgm_project(dgm_plan* P, const double* samples, int32_t column, void* fields) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!samples || !fields || column < 0 || column >= P->opt.n_columns)
        return fail(DGM_EINVAL, "invalid projection arguments");
    std::vector<double> pts, w;
    tet_rule(P->pE + 3, pts, w);
    const size_t nq = w.size();
    const int64_t K = P->mesh.K;
    const int N = P->N;
    std::vector<double> phi(nq * N);
    for (size_t q = 0; q < nq; ++q) ref_basis_values(P->pE, &pts[3 * q], &phi[q * N]);
    // covariant coefficients u_l = A^T sum_q w_q phi_l(q) f(r_q)  (closed-form block mass inverse)
    const int rs = P->kt->real_size;
    const int NH = P->NH;   // H keeps its first NH modes (the projection onto its own space)
    const size_t rows = size_t(3) * (N + NH);
    std::vector<unsigned char> host(rows * K * rs);
    for (int64_t e = 0; e < K; ++e) {
        double AT[3][3];   // A^T[j][r] = edge j, coordinate r
        const double* V = &P->mesh.verts[12 * e];
        for (int j = 0; j < 3; ++j)
            for (int r = 0; r < 3; ++r) AT[j][r] = V[3 * (j + 1) + r] - V[r];
        for (int fld = 0; fld < 2; ++fld)
            for (int l = 0; l < (fld == 0 ? N : NH); ++l) {
                double m[3] = {0, 0, 0};
                for (size_t q = 0; q < nq; ++q) {
                    const double* f = &samples[(e * nq + q) * 6 + 3 * fld];
                    for (int r = 0; r < 3; ++r) m[r] += w[q] * phi[q * N + l] * f[r];
                }
                for (int j = 0; j < 3; ++j) {
                    const double v = AT[j][0] * m[0] + AT[j][1] * m[1] + AT[j][2] * m[2];
                    const size_t idx = size_t(fld == 0 ? j * N + l : 3 * N + j * NH + l) * K + e;
                    if (rs == 8)
                        reinterpret_cast<double*>(host.data())[idx] = v;
                    else
                        reinterpret_cast<float*>(host.data())[idx] = float(v);
                }
            }
    }
    const int Sc = P->opt.n_columns;
    cudaError_t e = cudaMemcpy2DAsync(static_cast<unsigned char*>(fields) + size_t(column) * rs,
                                      size_t(Sc) * rs, host.data(), rs, rs, rows * K,
                                      cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "projection copy");
    e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "projection sync");
    return DGM_OK;
}

int dgm_status_check(dgm_plan* P) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, P->geom + P->off_status, sizeof(st), cudaMemcpyDeviceToHost, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    if ((e = cudaMemsetAsync(P->geom + P->off_status, 0, sizeof(st), P->stream)) != cudaSuccess)
        return cuda_fail(e, "status clear");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "status sync");
    if (st & ST_TIMEOUT) return fail(DGM_ETIMEOUT, "a device-side wait gave up");
    if (st & ST_NAN) return fail(DGM_ENAN, "non-finite values detected");
    if (st & ST_BAD_INDEX) return fail(DGM_EINVAL, "halo element id out of range (skipped)");
    if (st & ST_BAD_NEIGHBOUR) return fail(DGM_EMESH, "out-of-range neighbour index on the device");
    return DGM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free energy (dgm_energy_noalloc): same kernels as dgm_energy, with
// the per-block partial sums in a fixed file-scope device array instead of the
// caller's geometry/workspace buffer.  Host code must not pass the symbol
// itself to a kernel (on the host it names a stand-in, not device memory): its
// device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_energy_scratch[DGM_NOALLOC_MAX_COLUMNS * ENERGY_BLOCKS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_energy_scratch on the current device (looked up on first use).
int scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(DGM_EUNSUP, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_energy_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(energy scratch)");
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return DGM_OK;
}
}  // namespace

extern "C" int dgm_energy_noalloc(dgm_plan* P, const void* fields, double* out_device) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!fields || !out_device) return fail(DGM_EINVAL, "null argument");
    const int Sc = P->opt.n_columns;
    if (Sc > DGM_NOALLOC_MAX_COLUMNS)
        return fail(DGM_EINVAL, "dgm_energy_noalloc supports at most " +
                                    std::to_string(DGM_NOALLOC_MAX_COLUMNS) + " columns, plan has " +
                                    std::to_string(Sc));
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != P->device) return fail(DGM_ESTATE, "current device is not the plan's device");
    double* part = nullptr;
    int rc = scratch_for_current_device(&part);
    if (rc) return rc;
    const double* geo = reinterpret_cast<const double*>(P->geom + P->off_geo);
    dim3 grid(ENERGY_BLOCKS, Sc);
    if (P->kt->real_size == 8)
        energy_partial<double><<<grid, ENERGY_THREADS, 0, P->stream>>>(
            static_cast<const double*>(fields), geo, P->mesh.K, P->k_active, Sc, P->N, P->NH, part);
    else
        energy_partial<float><<<grid, ENERGY_THREADS, 0, P->stream>>>(
            static_cast<const float*>(fields), geo, P->mesh.K, P->k_active, Sc, P->N, P->NH, part);
    energy_final<<<(Sc + 127) / 128, 128, 0, P->stream>>>(
        part, ENERGY_BLOCKS, Sc, out_device, reinterpret_cast<int32_t*>(P->geom + P->off_status));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    return DGM_OK;
}

// ---------------------------------------------------------------------------
// Batched advance through a captured CUDA graph (dgm_batch_*).
__global__ void advance_clock(double* t, double dt) { *t += dt; }

struct dgm_batch {
    std::vector<dgm_plan*> members;
    cudaStream_t user = nullptr;     // caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;   // the batch's own stream: graphs are captured/launched here
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_release(dgm_batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto s : B->side) cudaStreamDestroy(s);
    for (auto e : B->join) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

// one LSRK4 step of member P on stream st with the device clock
static int member_step(dgm_plan* P, cudaStream_t st) {
    StageParams prm;
    stage_params(P, prm);
    double* clock = reinterpret_cast<double*>(P->geom + P->off_time);
    prm.tdev = clock;
    const double dt = P->opt.dt;
    for (int k = 0; k < 5; ++k) {
        prm.u = P->fields[P->cur];
        prm.u_out = P->fields[1 - P->cur];
        prm.res = P->res;
        prm.aux = P->aux[P->cur];
        prm.aux_out = P->aux[1 - P->cur];
        prm.aux_res = P->aux_res;
        prm.t = LSRK_C[k] * dt;
        prm.a = LSRK_A[k];
        prm.b = LSRK_B[k];
        int rc = P->kt->launch_stage(prm, MODE_LSRK, st);
        if (rc) return rc;
        P->cur = 1 - P->cur;
    }
    advance_clock<<<1, 1, 0, st>>>(clock, dt);
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

extern "C" int dgm_batch_create(dgm_batch** out, dgm_plan* const* members, int32_t n, void* stream) {
    if (!out || !members || n < 1) return fail(DGM_EINVAL, "empty batch");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!members[i] || !members[i]->bound) return fail(DGM_EINVAL, "batch member not bound");
        if (members[i]->opt.integrator != DGM_LSRK4) return fail(DGM_EINVAL, "batch members must use LSRK4");
        if (members[i]->k_active < members[i]->mesh.K)
            return fail(DGM_EINVAL, "batch members must have every element active (no halo)");
        if (members[i]->mixed) return fail(DGM_EUNSUP, "mixed-order plans are not batched");
        if (members[i]->n_inc > 0) return fail(DGM_EUNSUP, "plans with incident faces are not batched");
        if (members[i]->sip_alpha > 0.0) return fail(DGM_EUNSUP, "plans with the interior penalty are not batched");
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return fail(DGM_EINVAL, "duplicate batch member");
    }
    dgm_batch* B = new dgm_batch();
    B->members.assign(members, members + n);
    B->user = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "stream create");
    }
    if ((e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming)) != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "event create");
    }
    for (int i = 0; i < n; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            batch_release(B);
            return cuda_fail(e, "stream/event create");
        }
        B->side.push_back(st);
        B->join.push_back(ev);
    }
    // capture two LSRK4 steps of every member: ten stages return the ping-pong
    // buffers to their starting roles, so the graph can be replayed as is
    std::vector<int> cur0(n);
    for (int i = 0; i < n; ++i) cur0[i] = B->members[i]->cur;
    if ((e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "begin capture");
    }
    int rc = DGM_OK;
    cudaEventRecord(B->fork, B->stream);
    for (int i = 0; i < n && rc == DGM_OK; ++i) {
        cudaStreamWaitEvent(B->side[i], B->fork, 0);
        for (int step = 0; step < 2 && rc == DGM_OK; ++step) rc = member_step(B->members[i], B->side[i]);
        cudaEventRecord(B->join[i], B->side[i]);
        cudaStreamWaitEvent(B->stream, B->join[i], 0);
    }
    e = cudaStreamEndCapture(B->stream, &B->graph);
    for (int i = 0; i < n; ++i) B->members[i]->cur = cur0[i];
    if (rc != DGM_OK || e != cudaSuccess) {
        batch_release(B);
        return rc ? fail(rc, "stage launch during capture failed") : cuda_fail(e, "end capture");
    }
    if ((e = cudaGraphInstantiate(&B->exec, B->graph, 0)) != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "graph instantiate");
    }
    *out = B;
    return DGM_OK;
}

extern "C" int dgm_batch_advance(dgm_batch* B, int64_t n_steps, const double* t0) {
    if (!B) return fail(DGM_EINVAL, "null batch");
    if (n_steps < 0) return fail(DGM_EINVAL, "negative step count");
    const int n = int(B->members.size());
    cudaError_t e;
    // order after work queued on the caller's stream and on each member's stream
    if ((e = cudaEventRecord(B->fork, B->user)) != cudaSuccess) return cuda_fail(e, "event record");
    if ((e = cudaStreamWaitEvent(B->stream, B->fork, 0)) != cudaSuccess) return cuda_fail(e, "wait");
    for (int i = 0; i < n; ++i) {
        dgm_plan* P = B->members[i];
        if ((e = cudaEventRecord(B->join[i], P->stream)) != cudaSuccess) return cuda_fail(e, "event record");
        if ((e = cudaStreamWaitEvent(B->stream, B->join[i], 0)) != cudaSuccess) return cuda_fail(e, "wait");
        const double t = t0 ? t0[i] : 0.0;
        if ((e = cudaMemcpyAsync(P->geom + P->off_time, &t, sizeof(double), cudaMemcpyHostToDevice,
                                 B->stream)) != cudaSuccess)
            return cuda_fail(e, "clock upload");
    }
    // the clock uploads read host memory: finish them before it goes out of scope
    if ((e = cudaStreamSynchronize(B->stream)) != cudaSuccess) return cuda_fail(e, "clock sync");
    for (int64_t k = 0; k + 1 < n_steps; k += 2)
        if ((e = cudaGraphLaunch(B->exec, B->stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    if (n_steps % 2) {
        for (int i = 0; i < n; ++i) {
            int rc = member_step(B->members[i], B->stream);
            if (rc) return fail(rc, "stage kernel launch failed");
        }
    }
    if ((e = cudaEventRecord(B->fork, B->stream)) != cudaSuccess) return cuda_fail(e, "event record");
    for (int i = 0; i < n; ++i)
        if ((e = cudaStreamWaitEvent(B->members[i]->stream, B->fork, 0)) != cudaSuccess)
            return cuda_fail(e, "wait");
    if ((e = cudaStreamWaitEvent(B->user, B->fork, 0)) != cudaSuccess) return cuda_fail(e, "wait");
    return DGM_OK;
}

extern "C" void dgm_batch_destroy(dgm_batch* B) { batch_release(B); }

// ---------------------------------------------------------------------------
// Discrete adjoint driver (dgm_forward_record / dgm_adjoint).
template <typename R>
__global__ void axpby_kernel(R* y, const R* x, double a, double b, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = (a == 0.0 ? R(0) : R(a) * y[i]) + R(b) * x[i];
}

// lu[(j N + l), e_r S + s] += sum_c W_r[c][j N + l] g[s][r][c], receivers in a fixed order
template <typename R>
__global__ void inject_receivers(R* lu, const double* rec, int nrec, int64_t K, int S, int N,
                                 const double* g) {
    // one thread per (column, component-mode row); receivers in a fixed order,
    // so that receivers sharing an element accumulate without a race
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(S) * 3 * N) return;
    const int s = int(i % S);
    const int jl = int(i / S);
    const int64_t C = K * S;
    for (int r = 0; r < nrec; ++r) {
        const double* w = rec + int64_t(r) * (REC_HDR + 9 * N);
        const int64_t col = int64_t(w[0]) * S + s;
        const double* gr = g + (int64_t(s) * nrec + r) * 3;
        lu[int64_t(jl) * C + col] +=
            R(w[REC_HDR + jl] * gr[0] + w[REC_HDR + 3 * N + jl] * gr[1] + w[REC_HDR + 6 * N + jl] * gr[2]);
    }
}

__global__ void reduce_columns(const double* gcol, int64_t K, int S, double* deps, double* dmu) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= K) return;
    const int64_t C = K * S;
    double a = 0.0, b = 0.0;
    for (int s = 0; s < S; ++s) {
        a += gcol[e * S + s];
        b += gcol[C + e * S + s];
    }
    deps[e] = a;
    dmu[e] = b;
}

namespace {
struct AdjLayout {
    size_t fb = 0, ab = 0, sb = 0;   // field, aux, state bytes
    int64_t seg = 0, nseg = 0;
    size_t ck = 0, sg = 0, tmp = 0, res = 0, lu = 0, lr = 0, raw = 0, jmp = 0, grad = 0, total = 0;
};

AdjLayout adj_layout(const dgm_plan* P, int64_t n) {
    AdjLayout L;
    const int rs = P->kt->real_size;
    const int64_t C = P->mesh.K * P->opt.n_columns;
    L.fb = align256(size_t(6) * P->N * C * rs);
    L.ab = align256(size_t(6) * P->N * P->mesh.npml * P->opt.n_columns * rs);
    L.sb = L.fb + L.ab;
    // checkpoints every seg steps; the reverse sweep recomputes one segment at
    // a time and keeps the five stage inputs of each of its steps, so states
    // held = nseg + 5 seg, minimal at seg = sqrt(n / 5)
    L.seg = std::max<int64_t>(1, int64_t(std::ceil(std::sqrt(double(std::max<int64_t>(n, 1)) / 5.0))));
    L.nseg = (n + L.seg - 1) / L.seg;
    size_t off = 0;
    L.ck = off; off += L.sb * size_t(std::max<int64_t>(L.nseg, 1));
    L.sg = off; off += L.sb * size_t(5 * L.seg);
    L.tmp = off; off += L.sb * 2;
    L.res = off; off += L.sb;
    L.lu = off; off += L.sb;
    L.lr = off; off += L.sb;
    L.raw = off; off += L.fb;
    L.jmp = off; off += align256(size_t(24) * P->NF * C * rs);
    L.grad = off; off += align256(sizeof(double) * 2 * C);
    L.total = off;
    return L;
}

struct StateRef {
    void* f;
    void* a;
};

StateRef slot(unsigned char* ws, size_t base, size_t idx, const AdjLayout& L) {
    unsigned char* p = ws + base + idx * L.sb;
    return StateRef{p, L.ab ? p + L.fb : nullptr};
}
}  // namespace

extern "C" int dgm_set_materials(dgm_plan* P, const double* eps, const double* mu) {
    if (!P || !eps || !mu) return fail(DGM_EINVAL, "null argument");
    const int64_t K = P->mesh.K;
    for (int64_t e = 0; e < K; ++e)
        if (!(eps[e] > 0.0) || !(mu[e] > 0.0) || !std::isfinite(eps[e]) || !std::isfinite(mu[e]))
            return fail(DGM_EINVAL, "eps and mu must be positive and finite");
    std::copy(eps, eps + K, P->mesh.geo.begin() + size_t(G_EPS) * K);
    std::copy(mu, mu + K, P->mesh.geo.begin() + size_t(G_MU) * K);
    if (!P->bound) return DGM_OK;
    cudaError_t e = cudaMemcpyAsync(P->geom + P->off_geo + sizeof(double) * G_EPS * K,
                                    P->mesh.geo.data() + size_t(G_EPS) * K, sizeof(double) * 2 * K,
                                    cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload materials");
    std::vector<float> m32(P->mesh.geo.begin() + size_t(G_EPS) * K, P->mesh.geo.begin() + size_t(G_MU + 1) * K);
    e = cudaMemcpyAsync(P->geom + P->off_geo32 + sizeof(float) * G_EPS * K, m32.data(),
                        sizeof(float) * 2 * K, cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload materials (FP32)");
    if (int rc = build_face_table(P)) return rc;
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(e, "materials sync");
    return DGM_OK;
}

extern "C" int dgm_adjoint_workspace(const dgm_plan* P, int64_t n_steps, size_t* bytes) {
    if (!P || !bytes || n_steps < 1) return fail(DGM_EINVAL, "invalid arguments");
    *bytes = adj_layout(P, n_steps).total;
    return DGM_OK;
}

static int copy_state(dgm_plan* P, StateRef dst, const void* f, const void* a, const AdjLayout& L) {
    cudaError_t e = cudaMemcpyAsync(dst.f, f, L.fb, cudaMemcpyDeviceToDevice, P->stream);
    if (e == cudaSuccess && L.ab && a) e = cudaMemcpyAsync(dst.a, a, L.ab, cudaMemcpyDeviceToDevice, P->stream);
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "state copy");
}

extern "C" int dgm_forward_record(dgm_plan* P, int64_t n_steps, double t0, double* records, void* ws_) {
    if (P && P->k_active < P->mesh.K) return fail(DGM_EUNSUP, "the adjoint needs every element active");
    if (P && P->mixed) return fail(DGM_EUNSUP, "the adjoint is not built for mixed-order plans");
    if (P && P->n_inc > 0) return fail(DGM_EUNSUP, "the adjoint is not built for incident faces");
    if (P && P->sip_alpha > 0.0) return fail(DGM_EUNSUP, "the adjoint is not built for the interior penalty");
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->opt.integrator != DGM_LSRK4) return fail(DGM_EUNSUP, "the adjoint needs LSRK4");
    if (!records || !ws_ || n_steps < 1) return fail(DGM_EINVAL, "invalid arguments");
    if (reinterpret_cast<uintptr_t>(ws_) % 256) return fail(DGM_EINVAL, "workspace must be 256-byte aligned");
    unsigned char* ws = static_cast<unsigned char*>(ws_);
    const AdjLayout L = adj_layout(P, n_steps);
    const int64_t per = int64_t(P->opt.n_columns) * P->n_rec * 3;
    for (int64_t n = 0; n < n_steps; ++n) {
        if (n % L.seg == 0) {
            int rc = copy_state(P, slot(ws, L.ck, size_t(n / L.seg), L), P->fields[P->cur], P->aux[P->cur], L);
            if (rc) return rc;
        }
        int rc = dgm_advance(P, 1, t0 + double(n) * P->opt.dt);
        if (rc) return rc;
        rc = dgm_sample_receivers(P, P->fields[P->cur], records + n * per);
        if (rc) return rc;
    }
    return DGM_OK;
}

// LSRK4 stages of one step from `in` (= st[0]): the inputs of stages 1..4 go to
// st[1..4] (to scratch buffers when st is null), the step's result to `out`;
// with out.f == nullptr the sweep stops after the first nst stages.
static int lsrk_stages(dgm_plan* P, StateRef in, StateRef* st, int nst, StateRef tmp0, StateRef tmp1,
                       StateRef res, StateRef out, double t) {
    StageParams prm;
    stage_params(P, prm);
    const double dt = P->opt.dt;
    StateRef cur = in;
    for (int k = 0; k < 5; ++k) {
        StateRef nxt;
        if (k < 4) nxt = st ? st[k + 1] : ((k % 2) ? tmp1 : tmp0);
        else nxt = out;
        if (k >= nst && !out.f) break;
        prm.u = cur.f;
        prm.u_out = nxt.f;
        prm.aux = cur.a;
        prm.aux_out = nxt.a;
        prm.res = res.f;
        prm.aux_res = res.a;
        prm.t = t + LSRK_C[k] * dt;
        prm.a = LSRK_A[k];
        prm.b = LSRK_B[k];
        int rc = P->kt->launch_stage(prm, MODE_LSRK, P->stream);
        if (rc) return fail(rc, "stage kernel launch failed");
        cur = nxt;
    }
    return DGM_OK;
}

template <typename R>
static int axpby(dgm_plan* P, StateRef y, StateRef x, double a, double b, const AdjLayout& L) {
    const int64_t nf = int64_t(L.fb / sizeof(R));
    axpby_kernel<R><<<1216, 256, 0, P->stream>>>(static_cast<R*>(y.f), static_cast<const R*>(x.f), a, b, nf);
    if (L.ab) {
        const int64_t na = int64_t(L.ab / sizeof(R));
        axpby_kernel<R><<<1216, 256, 0, P->stream>>>(static_cast<R*>(y.a), static_cast<const R*>(x.a), a, b, na);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "axpby launch");
}

extern "C" int dgm_adjoint(dgm_plan* P, int64_t n_steps, double t0, const double* drec, void* ws_,
                           double* deps, double* dmu) {
    if (P && P->k_active < P->mesh.K) return fail(DGM_EUNSUP, "the adjoint needs every element active");
    if (P && P->mixed) return fail(DGM_EUNSUP, "the adjoint is not built for mixed-order plans");
    if (P && P->n_inc > 0) return fail(DGM_EUNSUP, "the adjoint is not built for incident faces");
    if (P && P->sip_alpha > 0.0) return fail(DGM_EUNSUP, "the adjoint is not built for the interior penalty");
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (!drec || !ws_ || !deps || !dmu || n_steps < 1) return fail(DGM_EINVAL, "invalid arguments");
    if (reinterpret_cast<uintptr_t>(ws_) % 256) return fail(DGM_EINVAL, "workspace must be 256-byte aligned");
    unsigned char* ws = static_cast<unsigned char*>(ws_);
    const AdjLayout L = adj_layout(P, n_steps);
    const bool f64 = P->kt->real_size == 8;
    const int64_t K = P->mesh.K;
    const int Sc = P->opt.n_columns;
    const int64_t per = int64_t(Sc) * P->n_rec * 3;
    const double dt = P->opt.dt;
    StateRef lu = slot(ws, L.lu, 0, L), lr = slot(ws, L.lr, 0, L), res = slot(ws, L.res, 0, L);
    StateRef tmp0 = slot(ws, L.tmp, 0, L), tmp1 = slot(ws, L.tmp, 1, L);
    StateRef st[5];
    cudaError_t e;
    if ((e = cudaMemsetAsync(lu.f, 0, L.sb, P->stream)) != cudaSuccess) return cuda_fail(e, "clear");
    double* gcol = reinterpret_cast<double*>(ws + L.grad);
    if ((e = cudaMemsetAsync(gcol, 0, sizeof(double) * 2 * K * Sc, P->stream)) != cudaSuccess)
        return cuda_fail(e, "clear");
    const double* recw = reinterpret_cast<const double*>(P->geom + P->off_rec);
    for (int64_t sgi = L.nseg - 1; sgi >= 0; --sgi) {
        const int64_t start = sgi * L.seg, end = std::min(start + L.seg, n_steps);
        int rc = copy_state(P, slot(ws, L.sg, 0, L), slot(ws, L.ck, size_t(sgi), L).f,
                            slot(ws, L.ck, size_t(sgi), L).a, L);
        if (rc) return rc;
        // recompute the segment once, keeping the five stage inputs of each step
        for (int64_t i = start; i < end; ++i) {
            StateRef sti[5];
            for (int k = 0; k < 5; ++k) sti[k] = slot(ws, L.sg, size_t(5 * (i - start) + k), L);
            const StateRef nxt = (i + 1 < end) ? slot(ws, L.sg, size_t(5 * (i + 1 - start)), L)
                                               : StateRef{nullptr, nullptr};
            rc = lsrk_stages(P, sti[0], sti, 4, tmp0, tmp1, res, nxt, t0 + double(i) * dt);
            if (rc) return rc;
        }
        for (int64_t n = end - 1; n >= start; --n) {
            if (P->n_rec > 0) {
                const unsigned nb = unsigned((int64_t(Sc) * 3 * P->N + 127) / 128);
                if (f64)
                    inject_receivers<double><<<nb, 128, 0, P->stream>>>(
                        static_cast<double*>(lu.f), recw, P->n_rec, K, Sc, P->N, drec + n * per);
                else
                    inject_receivers<float><<<nb, 128, 0, P->stream>>>(
                        static_cast<float*>(lu.f), recw, P->n_rec, K, Sc, P->N, drec + n * per);
            }
            const double tn = t0 + double(n) * dt;
            for (int k = 0; k < 5; ++k) st[k] = slot(ws, L.sg, size_t(5 * (n - start) + k), L);
            for (int k = 4; k >= 0; --k) {
                // lr = a_{k+1} lr + b_k lu  (a_5 := 0 starts each step)
                const double a = (k == 4) ? 0.0 : LSRK_A[k + 1];
                rc = f64 ? axpby<double>(P, lr, lu, a, LSRK_B[k], L) : axpby<float>(P, lr, lu, a, LSRK_B[k], L);
                if (rc) return rc;
                StageParams prm;
                stage_params(P, prm);
                prm.u = st[k].f;
                prm.aux = st[k].a;
                prm.raw = ws + L.raw;
                prm.jumps = ws + L.jmp;
                prm.t = tn + LSRK_C[k] * dt;
                rc = P->kt->launch_stage(prm, MODE_RAW, P->stream);
                if (rc) return fail(rc, "forward kernel launch failed");
                AdjParams ap;
                std::memset(&ap, 0, sizeof(ap));
                ap.lr = lr.f;
                ap.lu = lu.f;
                ap.lr_aux = lr.a;
                ap.lu_aux = lu.a;
                ap.u = st[k].f;
                ap.aux = st[k].a;
                ap.raw = ws + L.raw;
                ap.jumps = ws + L.jmp;
                ap.geo = prm.geo;
                ap.geo_r = prm.geo_r;
                ap.fnb_r = prm.fnb_r;
                ap.nbr = prm.nbr;
                ap.pml = prm.pml;
                ap.status = prm.status;
                ap.grad = gcol;
                ap.force_index64 = P->force_index64;
                ap.tile_groups = P->tile_groups;
                ap.K = K;
                ap.npml = P->mesh.npml;
                ap.S = Sc;
                ap.upwind = prm.upwind;
                ap.dt = dt;
                rc = P->kt->launch_adjoint(ap, P->stream);
                if (rc) return fail(rc, "adjoint kernel launch failed");
            }
        }
    }
    reduce_columns<<<unsigned((K + 255) / 256), 256, 0, P->stream>>>(gcol, K, Sc, deps, dmu);
    e = cudaGetLastError();
    return e == cudaSuccess ? DGM_OK : cuda_fail(e, "reduce launch");
}

// ---------------------------------------------------------------------------
// Autotuner: times every tile-shape variant of the LSRK stage kernel on the
// plan's own state (first-stage form: reads u, writes u_out and res into the
// caller's workspace, so the plan's state is left untouched) and keeps the
// fastest for dgm_advance and dgm_batch_create.
extern "C" int dgm_autotune(dgm_plan* P, void* workspace, int32_t reps, float* ms_out) {
    if (!P || !P->bound) return fail(DGM_ESTATE, "plan not bound");
    if (P->sip_alpha > 0.0 && P->hs[0] == nullptr)
        return fail(DGM_ESTATE, "facet buffers of the interior penalty not bound (dgm_bind_sip)");
    if (!workspace) return fail(DGM_EINVAL, "null workspace");
    if (reps < 1) reps = 3;
    dgm_info info;
    dgm_plan_info(P, &info);
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    const size_t fb = align256(info.bytes_fields), ab = align256(info.bytes_aux);
    StageParams prm;
    stage_params(P, prm);
    // Phase-1 bulk copies where the plan has tensor maps: a map of the
    // workspace's first field buffer too, so that every timed launch takes
    // them; the last stage below times them against per-thread loads.
    const bool bulk_ok = P->tmaps_ok && tmap_fields(P, ws, TM_UW) && tmap_upload(P) == DGM_OK;
    if (bulk_ok) {
        prm.tmaps = P->geom + P->off_tmap;
        prm.tm_f0 = P->fields[0];
        prm.tm_f1 = P->fields[1];
        prm.tm_fw = ws;
    }
    // An LSRK4 plan is timed on stage sequences as the time loop runs them:
    // the first (untimed) launch reads the state and writes workspace buffer
    // 0, later launches ping-pong between that buffer and the plan's second
    // field buffer with the stage coefficients in turn, so each launch reads
    // an input that the previous one wrote, as in a step, and the tile
    // order's effect on L2 reuse is measured as a step sees it.  Between
    // steps the second field buffer (and the second auxiliary buffer) hold
    // nothing, so the state is only read.  Other plans repeat one launch from
    // the state into the workspace.
    const bool seq = P->opt.integrator == DGM_LSRK4 && P->fields[1 - P->cur] != nullptr &&
                     (!ab || P->aux[1 - P->cur] != nullptr);
    void* fbuf[2] = {ws, seq ? P->fields[1 - P->cur] : nullptr};
    void* abuf[2] = {ab ? ws + 2 * fb : nullptr, seq && ab ? P->aux[1 - P->cur] : nullptr};
    prm.res = ws + fb;
    prm.aux_res = ab ? ws + 2 * fb + ab : nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // mean time of `n` launches of the current shape and order (after one warm launch)
    auto time_it = [&](int n, float* ms) -> int {
        prm.u = P->fields[P->cur];
        prm.aux = P->aux[P->cur];
        prm.u_out = fbuf[0];
        prm.aux_out = abuf[0];
        prm.a = 0.0;
        prm.b = LSRK_B[0];
        int rc = launch_stage(P, prm, MODE_LSRK, P->stream);
        if (rc) return fail(rc, "stage kernel launch failed");
        int src = 0;   // buffer holding the last output
        cudaEventRecord(e0, P->stream);
        for (int r = 0; r < n; ++r) {
            if (seq) {
                const int k = (r + 1) % 5;
                prm.u = fbuf[src];
                prm.aux = abuf[src];
                prm.u_out = fbuf[1 - src];
                prm.aux_out = abuf[1 - src];
                prm.a = LSRK_A[k];
                prm.b = LSRK_B[k];
                src = 1 - src;
            }
            launch_stage(P, prm, MODE_LSRK, P->stream);
        }
        cudaEventRecord(e1, P->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= n;
        return DGM_OK;
    };
    int best = 0, rc = DGM_OK;
    float best_ms = 1e30f;
    prm.tile_groups = 1;
    for (int v = 0; v < P->kt->n_variants && rc == DGM_OK; ++v) {
        if (!variant_ok(P, v)) {
            if (ms_out) ms_out[v] = 0.f;
            continue;
        }
        prm.variant = v;
        float ms = 0.f;
        if ((rc = time_it(reps, &ms)) != DGM_OK) break;
        if (v < 8) P->variant_ms[v] = ms;
        if (ms_out) ms_out[v] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    // then the tile visiting order of the chosen shape (1 = in order)
    int best_g = 1;
    if (rc == DGM_OK) {
        prm.variant = best;
        const int cand[] = {1, 2, 3, 4, 6, 8, 12};
        float g_ms[7] = {0};
        for (int i = 0; i < 7 && rc == DGM_OK; ++i) {
            prm.tile_groups = cand[i];
            rc = time_it(reps < 10 ? 10 : reps, &g_ms[i]);   // two steps' stages at least
        }
        if (rc == DGM_OK) {
            // the fastest order, unless it is not a clear gain over the plain order
            int bi = 0;
            for (int i = 1; i < 7; ++i)
                if (g_ms[i] < g_ms[bi]) bi = i;
            if (g_ms[bi] < 0.99f * g_ms[0]) best_g = cand[bi];
        }
    }
    // then bulk copies against per-thread loads for that shape and order, each
    // timed twice in turn (the faster of its two): per-thread loads only when
    // they are faster
    int tile_loads = P->tile_loads;
    if (rc == DGM_OK && bulk_ok) {
        prm.tile_groups = best_g;
        float t_ms[2] = {1e30f, 1e30f};
        for (int r = 0; r < 4 && rc == DGM_OK; ++r) {
            const int pt = r % 2;
            prm.tmaps = pt ? nullptr : static_cast<const void*>(P->geom + P->off_tmap);
            float ms = 0.f;
            rc = time_it(reps < 10 ? 10 : reps, &ms);
            t_ms[pt] = std::min(t_ms[pt], ms);
        }
        if (rc == DGM_OK) tile_loads = t_ms[1] < t_ms[0] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DGM_OK) return rc;
    P->variant = best;
    P->tile_groups = best_g;
    P->tile_loads = tile_loads;
    return DGM_OK;
}

extern "C" int dgm_set_tile_groups(dgm_plan* P, int32_t groups) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (groups < 1 || groups > 64) return fail(DGM_EINVAL, "tile groups must be 1..64");
    P->tile_groups = groups;
    return DGM_OK;
}

extern "C" int dgm_get_tile_groups(const dgm_plan* P, int32_t* groups) {
    if (!P || !groups) return fail(DGM_EINVAL, "null argument");
    *groups = P->tile_groups;
    return DGM_OK;
}

extern "C" int dgm_autotune_info(const dgm_plan* P, int32_t* n_variants, int32_t* chosen) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (n_variants) *n_variants = P->kt->n_variants;
    if (chosen) *chosen = P->variant;
    return DGM_OK;
}

extern "C" int dgm_set_variant(dgm_plan* P, int32_t v) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (v < 0 || v >= P->kt->n_variants) return fail(DGM_EINVAL, "variant out of range");
    if (!variant_ok(P, v))
        return fail(DGM_EUNSUP, "this stage variant has neither incident faces nor the penalty "
                                "(the penalty runs in the default shape)");
    P->variant = v;
    return DGM_OK;
}

extern "C" int dgm_set_tile_loads(dgm_plan* P, int32_t per_thread) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (per_thread != 0 && per_thread != 1) return fail(DGM_EINVAL, "per_thread must be 0 or 1");
    P->tile_loads = per_thread;
    return DGM_OK;
}

extern "C" int dgm_get_tile_loads(const dgm_plan* P, int32_t* bulk) {
    if (!P || !bulk) return fail(DGM_EINVAL, "null argument");
    *bulk = (P->bound && P->tmaps_ok && P->tile_loads == 0) ? 1 : 0;
    return DGM_OK;
}

extern "C" int dgm_set_index64(dgm_plan* P, int32_t force) {
    if (!P) return fail(DGM_EINVAL, "null plan");
    if (force != 0 && force != 1) return fail(DGM_EINVAL, "force must be 0 or 1");
    P->force_index64 = force;
    return DGM_OK;
}

