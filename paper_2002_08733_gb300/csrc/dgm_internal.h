// Internal declarations shared by the host setup, the C ABI and the kernel
// translation units of the dgmax library.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace dgm {

constexpr int PMAX = 5;

__host__ __device__ constexpr int nmodes(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
__host__ __device__ constexpr int nfmodes(int p) { return (p + 1) * (p + 2) / 2; }

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Shapes of the tensor-core variant of the FP32 stage kernel (p = 2, 3; 64
// columns per CTA; tensor-memory row = (column, field)).  Per row the
// pre-mass right-hand side of one field is
//   D = A_swap B_curl + sum_j A_g,j B_lift
// with A_swap = +-sign(det A) times the other field's coefficients (K = 3N,
// index i N + m for component i, mode m), B_curl[(i, m)][(j, l)] =
// eps_jai S_a[l][m] (the reference curl of Eq. (matrix_free_curl)), A_g,j the
// pulled-back face fluxes of component j (K = 4 NF, index f NF + m) and
// B_lift[(f, m)][l] = R_f[m][l] (the lift of Eqs. (uwc)/(cwc)).  Component j
// of D occupies columns [j NL, j NL + N) (NL = N rounded up to 16), so every
// MMA output and every tensor-memory load starts on a multiple of 16 columns.
template <int P>
struct TcShape {
    static constexpr int N = nmodes(P), NF = nfmodes(P);
    static constexpr int KC = round_up(3 * N, 8);     // curl: K (TF32 steps of 8)
    static constexpr int NL = round_up(N, 16);        // lift: N per component
    static constexpr int NC = 3 * NL;                 // curl: N (all three components)
    static constexpr int KL = round_up(4 * NF, 8);    // lift: K per component
    // tensor-memory columns: A_swap hi/lo, A_g hi/lo (3 components each), D
    static constexpr int T_SWAP_HI = 0, T_SWAP_LO = KC;
    static constexpr int T_G_HI = 2 * KC, T_G_LO = 2 * KC + 3 * KL;
    static constexpr int T_D = round_up(2 * KC + 6 * KL, 32);
    static constexpr int TCOLS = 512;
    static constexpr bool FITS = T_D + NC <= TCOLS;   // tensor-memory budget
    // B image (bytes, K-major core matrices): curl hi, curl lo, lift hi, lift lo
    static constexpr int B_CURL = NC * KC * 4, B_LIFT = NL * KL * 4;
    static constexpr int B_BYTES = 2 * B_CURL + 2 * B_LIFT;
    static constexpr int SBO_CURL = KC * 32, SBO_LIFT = KL * 32;   // bytes per 8-row group
};

// byte offset of entry (n, k) of a K-major, no-swizzle B operand with K columns
// per row: 8-row x 4-value core matrices, K-adjacent ones contiguous
__host__ __device__ constexpr int tc_b_offset(int n, int k, int K) {
    return (n / 8) * (K * 32) + (k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4;
}

// Per-element FP64 record, stored structure-of-arrays: geo[k * K + e].
enum GeoSlot {
    G_AIT = 0,    // 9 entries of A^-T, row major
    G_DET = 9,    // signed det A
    G_EPS = 10,
    G_MU = 11,
    G_SIG = 12,   // 3 PML damping values
    G_PAD = 15,
    G_COUNT = 16
};

// Per-face neighbour table (rebuilt on the device whenever geometry or
// materials change): for face f of element e, slot f * FNB_COUNT + k holds
// the neighbour's A^-T (k = 0..8, row major), its impedance sqrt(mu/eps)
// (k = 9), det A, eps and mu (k = 10..12); on a boundary face the element's
// own values.  It turns the neighbour-geometry gathers of the face constants
// into coalesced reads (the stage kernel reads k = 0..9, the adjoint all).
enum FnbSlot { FNB_AIT = 0, FNB_Z = 9, FNB_DET = 10, FNB_EPS = 11, FNB_MU = 12, FNB_COUNT = 13 };

// Source record per column (FP64): [elem, f0, bw, t0, 0,0,0,0, w[3N]].
constexpr int SRC_HDR = 8;

enum Mode { MODE_RHS = 0, MODE_LSRK = 1, MODE_LF_E = 2, MODE_LF_H = 3, MODE_RAW = 4 };

enum StatusBits { ST_OK = 0, ST_BAD_NEIGHBOUR = 1, ST_NAN = 2, ST_TIMEOUT = 4, ST_BAD_INDEX = 8 };

struct StageParams {
    const void* u;        // fields in  [6][N][K][S]
    void* u_out;          // LSRK: other buffer; leapfrog: same buffer; RHS: du
    void* res;            // LSRK residual
    const void* aux;      // PML auxiliaries in [6][N][P][S]
    void* aux_out;
    void* aux_res;
    const double* geo;    // [G_COUNT][K] FP64 master copy
    const void* geo_r;    // the same in the kernel's real type (FP32 copy for FP32 kernels)
    const int32_t* nbr;   // [4][K]: (neighbour << 2) | neighbour's local face, or -1
    const void* fnb_r;    // [4][FNB_COUNT][K] per-face neighbour data in the kernel's real type
    const int32_t* pml;   // [K]: index into aux, or -1 (may be null without PML)
    const double* src;    // [S][SRC_HDR + 3N] or null
    int32_t* status;      // device status word
    int64_t K;
    int64_t npml;
    int32_t S;
    int32_t upwind;
    double t, dt, a, b;   // stage time, step, LSRK coefficients a_k, b_k
    float dt_f, a_f, b_f; // the same rounded to FP32 (set by the launchers for FP32 kernels)
    const double* tdev;   // if set: stage time = *tdev + t (device clock of graph replays)
    void* raw;            // MODE_RAW: right-hand side before the mass inverse [6][N][K][S]
    void* jumps;          // MODE_RAW: physical face jumps dE, dH [4][6][NF][K][S]
    int32_t variant;      // tile-shape variant of the LSRK stage kernel (autotuner)
    int32_t force_index64;// 1: 64-bit index arithmetic even where 32 bits suffice
    int32_t tile_groups;  // tile visiting order: G interleaved segments (1: in order)
    const void* tc_b;     // tensor-core variant: B operand image (TcShape<P>::B_BYTES), or null
    int64_t K_active;     // elements updated: the first K_active (the rest are halo copies)
    const void* ops;      // mixed-order plans: dense reference operators S, R of degree p + 1
    const void* inc;      // incident faces: [i][NF][3] reference-frame jump terms
                          // 2 A^T E_inc traced on face mode m at the stage time (R), or null
    // interior penalty with a facet field (null when off): per (face, element)
    // (facet << 1) | owner, or -1 ([4][K]); facet field h_s [3][NF][facet][S]
    // (physical components per face mode, R): stage input, output (LSRK; the
    // time derivative for MODE_RHS) and LSRK residual; the penalty alpha; facets
    const int32_t* sfid;
    const void* hs;
    void* hs_out;
    void* hs_res;
    double sip_alpha;
    int64_t n_facets;
    const void* fcp;      // precomputed face constants [FC_ROWS][K] (R), see face_consts_kernel
    // Tiled bulk copies of the stage kernel's phase 1 (null: per-thread loads).
    // tmaps: the plan's tensor maps in device memory, TMAP_SETS sets of TMAP_COUNT
    // (one set per tile width; see TmapIndex); tm_f0 / tm_f1: the field buffers
    // the u maps describe.  The launcher narrows tmaps to the set of its tile
    // width and sets tm_u to the map of prm.u (-1: per-thread loads).
    const void* tmaps;
    const void* tm_f0;
    const void* tm_f1;
    const void* tm_fw;    // the autotuner's scratch field buffer (map TM_UW), or null
    int32_t tm_u;
};

// Tensor maps (CUtensorMap, 128 bytes each) of one tile width, all with the
// tile's columns as the innermost box dimension: the field buffers as
// [6][N][C] (box TE x N x 6), the element constants [G_COUNT][K] (box TE x 16),
// the face constants as [4][16][K] (box TE x 15 x 4, or x 16 with the interior
// penalty) and the metric rows of the face-constant table [FC_ROWS][K] (box
// TE x 6, or TE x 15 with A^T); TM_UW: a field-shaped scratch buffer of the
// autotuner (dgm_autotune), encoded while it times.
enum TmapIndex {
    TM_U0 = 0, TM_U1 = 1, TM_GEO = 2, TM_FC = 3, TM_FCS = 4, TM_GM = 5, TM_GMGA = 6, TM_UW = 7,
    TMAP_COUNT = 8
};
constexpr int TMAP_BYTES = 128;
// rows of the boxes (the stage kernel's shared-memory rows): element constants,
// face constants per face (15, or 16 with the penalty) of the 16 per face of
// the table, metric, A^T
constexpr int TM_ROWS_EG = 16, TM_ROWS_FC = 15, TM_ROWS_FACE = 16, TM_ROWS_GM = 6, TM_ROWS_GA = 9;
// set 0: tiles of 128 bytes per row (32 FP32 or 16 FP64 columns); set 1: 16 FP32 columns
constexpr int TMAP_SETS = 2;

// Rows per element of the precomputed face constants: 4 faces x 16, the
// metric A^T A (6), A^T (9).
constexpr int FC_ROWS = 4 * 16 + 6 + 9;
// Computes them for a plan (dgm_facec.cu); real_size 4 or 8.
int launch_face_consts(const StageParams& prm, int real_size, bool sip, void* out, void* stream);

// One adjoint stage: lu += dt F_u^T lr, and the material-gradient terms
// dt lr . (dF/d eps_T, dF/d mu_T) u at the stage input u (per column).
struct AdjParams {
    const void* lr;       // adjoint residual (fields)      [6][N][K][S]
    void* lu;             // adjoint state (fields), updated in place
    const void* lr_aux;   // adjoint residual (PML aux)     [6][N][P][S]
    void* lu_aux;         // adjoint state (PML aux), updated in place
    const void* u;        // forward stage input (fields)
    const void* aux;      // forward stage input (PML aux)
    const void* raw;      // forward right-hand side before the mass inverse
    const void* jumps;    // forward physical face jumps
    const double* geo;
    const void* geo_r;    // geometry in the kernel's real type
    const void* fnb_r;    // per-face neighbour table in the kernel's real type
    const int32_t* nbr;
    const int32_t* pml;
    int32_t* status;
    double* grad;         // [2][K*S]: per-column d/d eps, d/d mu accumulators
    int32_t force_index64;// 1: 64-bit index arithmetic even where 32 bits suffice
    int32_t tile_groups;  // tile visiting order (as in StageParams)
    int64_t K;
    int64_t npml;
    int32_t S;
    int32_t upwind;
    double dt;
};

// Kernel translation unit entry points, one set per (order, precision).
struct KernelTable {
    int (*launch_stage)(const StageParams&, int mode, void* stream);
    int real_size;
    int (*launch_adjoint)(const AdjParams&, void* stream);
    int n_variants;   // tile-shape variants of the LSRK stage (autotuner)
};

const KernelTable* kernel_table(int p, int precision);
// Mixed-order plans (E of degree pE, H of degree pE - 1; dgm_mixed.cu).
const KernelTable* kernel_table_mixed(int pE, int precision);

// Host setup (dgm_setup.cpp)
struct HostMesh {
    int64_t K = 0;
    std::vector<double> geo;          // G_COUNT * K
    std::vector<int32_t> nbr;         // 4 * K
    std::vector<int32_t> pml_idx;     // K
    std::vector<double> verts;        // K * 12 (sorted local vertices)
    std::vector<int64_t> vid;         // K * 4 (sorted vertex ids)
    int64_t npml = 0;
};

int build_mesh(int64_t nv, const double* xyz, int64_t nt, const int64_t* tets, const double* eps,
               const double* mu, const double* pml_lo, const double* pml_hi, double pml_L,
               double pml_smax, int pml_order, bool has_pml, HostMesh& out, std::string& err);

// Reference matrices on the reference tetrahedron (dgm_refmats.cpp):
// S[a][l][m] = int phi_l d_a phi_m, R[f][m][l] = int_{face f} psi_m phi_l (ds dt).
int build_refmats(int p, std::vector<double>& S, std::vector<double>& R, std::string& err);

// Reference basis values at reference points (for projection, sources): out[N].
void ref_basis_values(int p, const double xr[3], double* out);

// Collapsed Gauss-Legendre rule on the reference tetrahedron.
void tet_rule(int q, std::vector<double>& pts, std::vector<double>& w);

// Collapsed Gauss-Legendre rule on the reference triangle {s, t >= 0, s + t <= 1}
// (q points per direction: pts [n][2], w [n]) and the orthonormal face basis of
// degree p at its points (psi [n][NF]); the parametrisation of the trace operators.
void face_rule(int p, int q, std::vector<double>& pts, std::vector<double>& w,
               std::vector<double>& psi);

}  // namespace dgm
