// Mixed-order stage kernel: E of degree PE = p + 1, H of degree p (Sec. III,
// Eqs. (triale)/(trialh)).
//
// Both spaces are spanned by the first modes of the orthonormal hierarchical
// basis of degree PE, so every operator is a submatrix of the degree-PE ones:
// the volume curl of H tested against E, S_a[l < N_E][m < N_H], and of E tested
// against H, S_a[l < N_H][m < N_E] (Eq. (matrix_free_curl)); the traces of E
// onto the N_F,E face modes and of H onto the first N_F,H; the lifts are their
// transposes, and projecting a face jump of E onto H's face space keeps its
// first N_F,H modes.  The numerical flux of Eqs. (uwc)/(cwc) (central or
// upwind, PEC ghost states) is evaluated per face mode in the physical frame:
//   g_E = 2|F| A^-1 (c_E n x dH - b_E n x (n x dE))
//   g_H = -2|F| A^-1 (c_H n x dE + b_H n x (n x dH)),   dX = X+ - X-,
// with X = A^-T x per side.  One thread per column (element x source), dense
// operator loops, the state in per-thread arrays: a plain kernel that makes
// the mixed-order method available, not a tuned one.
//
// Field rows: E component c (0..2) mode l at c N_E + l, H component c (0..2)
// mode l at 3 N_E + c N_H + l; row r of column col at r K S + col.
#include <cuda_runtime.h>

#include <cstdint>

#include "dgm_internal.h"
#include "dgmax.h"

namespace dgm {
namespace {

__device__ __forceinline__ double src_time(double t, double f0, double bw, double t0) {
    const double twopi = 6.283185307179586476925286766559;
    const double s = 1.0 / (twopi * bw);
    const double tau = t - t0;
    return sin(twopi * f0 * tau) * exp(-tau * tau / (2.0 * s * s));
}

template <typename R>
__device__ __forceinline__ void cross(const R a[3], const R b[3], R o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// eps_jai for the two axes a != j: curl_j = sum_a eps_jai d_a v_i, i = 3 - j - a
__device__ __forceinline__ int levi(int j, int a) { return ((j - a + 3) % 3 == 2) ? 1 : -1; }

template <int PE, typename R, int MODE>
__global__ void __launch_bounds__(128) mixed_stage_kernel(const StageParams prm) {
    constexpr int NE = nmodes(PE), NH = nmodes(PE - 1);
    constexpr int NFE = nfmodes(PE), NFH = nfmodes(PE - 1);
    const int64_t K = prm.K;
    const int S = prm.S;
    const int64_t C = K * S;
    const int64_t col = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (col >= prm.K_active * S) return;
    const int64_t e = col / S;
    const int s = int(col - e * S);
    const R* u = static_cast<const R*>(prm.u);
    const R* gr = static_cast<const R*>(prm.geo_r);
    const R* fnb = static_cast<const R*>(prm.fnb_r);
    const R* Sop = static_cast<const R*>(prm.ops);               // [3][NE][NE]
    const R* Rop = Sop + 3 * NE * NE;                             // [4][NFE][NE]
    auto S_at = [&](int a, int l, int m) { return __ldg(Sop + (a * NE + l) * NE + m); };
    auto R_at = [&](int f, int m, int l) { return __ldg(Rop + (f * NFE + m) * NE + l); };
    const int64_t rowH = 3 * NE;   // first H row

    R uE[3][NE], uH[3][NH], rE[3][NE], rH[3][NH];
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        for (int l = 0; l < NE; ++l) {
            uE[c][l] = u[(int64_t(c) * NE + l) * C + col];
            rE[c][l] = R(0);
        }
        for (int l = 0; l < NH; ++l) {
            uH[c][l] = u[(rowH + int64_t(c) * NH + l) * C + col];
            rH[c][l] = R(0);
        }
    }
    R ait[9];
    for (int k = 0; k < 9; ++k) ait[k] = gr[int64_t(G_AIT + k) * K + e];
    const R det = gr[int64_t(G_DET) * K + e];
    const R epsm = gr[int64_t(G_EPS) * K + e], mum = gr[int64_t(G_MU) * K + e];
    const R sgn = det < R(0) ? R(-1) : R(1);

    // volume curl: E rows from H (+s_T), H rows from E (-s_T)
#pragma unroll 1
    for (int j = 0; j < 3; ++j)
#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            if (a == j) continue;
            const int i = 3 - j - a;
            const R w = sgn * R(levi(j, a));
            for (int l = 0; l < NE; ++l) {
                R acc = R(0);
                for (int m = 0; m < NH; ++m) acc += S_at(a, l, m) * uH[i][m];
                rE[j][l] += w * acc;
            }
            for (int l = 0; l < NH; ++l) {
                R acc = R(0);
                for (int m = 0; m < NE; ++m) acc += S_at(a, l, m) * uE[i][m];
                rH[j][l] -= w * acc;
            }
        }

    // faces: traces of both sides, flux per face mode, lift
    R vE[3][NE], vH[3][NH];
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        const int32_t code = prm.nbr[int64_t(f) * K + e];
        const bool has = code >= 0 && int64_t(code >> 2) < K;
        if (code >= 0 && !has) atomicOr(prm.status, int32_t(ST_BAD_NEIGHBOUR));
        const int fn = has ? (code & 3) : 0;
        const int64_t ncol = has ? int64_t(code >> 2) * S + s : col;
        // neighbour's coefficients, the neighbour's A^-T and impedance (per-face table)
        R aitn[9];
        const R* tab = fnb + int64_t(f * FNB_COUNT) * K + e;
        for (int k = 0; k < 9; ++k) aitn[k] = tab[int64_t(FNB_AIT + k) * K];
        const R zn = tab[int64_t(FNB_Z) * K];
        if (has) {
            for (int c = 0; c < 3; ++c) {
                for (int l = 0; l < NE; ++l) vE[c][l] = u[(int64_t(c) * NE + l) * C + ncol];
                for (int l = 0; l < NH; ++l) vH[c][l] = u[(rowH + int64_t(c) * NH + l) * C + ncol];
            }
        }
        // 2|F| n = |det A| A^-T m_f, m_f = (1,1,1), -e_x, -e_y, -e_z (outward, reference face)
        const R mf[3] = {R(f == 0 ? 1 : (f == 1 ? -1 : 0)), R(f == 0 ? 1 : (f == 2 ? -1 : 0)),
                         R(f == 0 ? 1 : (f == 3 ? -1 : 0))};
        R vn[3];
        for (int r = 0; r < 3; ++r) vn[r] = ait[3 * r] * mf[0] + ait[3 * r + 1] * mf[1] + ait[3 * r + 2] * mf[2];
        const R fs = sqrt(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
        const R nrm[3] = {vn[0] / fs, vn[1] / fs, vn[2] / fs};
        const R twoF = fabs(det) * fs;
        const R zm = sqrt(mum / epsm), zp = has ? zn : zm;
        R cE = R(0.5), bE = R(0), cH = R(0.5), bH = R(0);
        if (prm.upwind) {
            const R ym = R(1) / zm, yp = R(1) / zp;
            cE = zp / (zm + zp);
            bE = R(1) / (zm + zp);
            cH = yp / (ym + yp);
            bH = R(1) / (ym + yp);
        }
#pragma unroll 1
        for (int m = 0; m < NFE; ++m) {
            const bool hm = m < NFH;   // H has this face mode
            R te[3], th[3], tne[3], tnh[3];
            for (int c = 0; c < 3; ++c) {
                R a = R(0), b = R(0), an = R(0), bn = R(0);
                for (int l = 0; l < NE; ++l) {
                    a += R_at(f, m, l) * uE[c][l];
                    if (has) an += R_at(fn, m, l) * vE[c][l];
                }
                if (hm) {
                    for (int l = 0; l < NH; ++l) {
                        b += R_at(f, m, l) * uH[c][l];
                        if (has) bn += R_at(fn, m, l) * vH[c][l];
                    }
                }
                te[c] = a; th[c] = b; tne[c] = an; tnh[c] = bn;
            }
            // physical traces and jumps (PEC: e+ = -e-, h+ = h-)
            R Eo[3], Ho[3], dE[3], dH[3];
            for (int r = 0; r < 3; ++r) {
                Eo[r] = ait[3 * r] * te[0] + ait[3 * r + 1] * te[1] + ait[3 * r + 2] * te[2];
                Ho[r] = ait[3 * r] * th[0] + ait[3 * r + 1] * th[1] + ait[3 * r + 2] * th[2];
                const R En = has ? aitn[3 * r] * tne[0] + aitn[3 * r + 1] * tne[1] + aitn[3 * r + 2] * tne[2]
                                 : -Eo[r];
                const R Hn = has ? aitn[3 * r] * tnh[0] + aitn[3 * r + 1] * tnh[1] + aitn[3 * r + 2] * tnh[2]
                                 : Ho[r];
                dE[r] = En - Eo[r];
                dH[r] = hm ? Hn - Ho[r] : R(0);
            }
            R ndE[3], ndH[3], nndE[3], nndH[3];
            cross(nrm, dE, ndE);
            cross(nrm, dH, ndH);
            cross(nrm, ndE, nndE);
            cross(nrm, ndH, nndH);
            R fE[3], fH[3];
            for (int r = 0; r < 3; ++r) {
                fE[r] = cE * ndH[r] - bE * nndE[r];
                fH[r] = cH * ndE[r] + bH * nndH[r];
            }
            // pulled back (A^-1 v)_j = sum_r A^-T[r][j] v_r, then lifted
            for (int j = 0; j < 3; ++j) {
                const R gE = twoF * (ait[j] * fE[0] + ait[3 + j] * fE[1] + ait[6 + j] * fE[2]);
                for (int l = 0; l < NE; ++l) rE[j][l] += R_at(f, m, l) * gE;
                if (hm) {
                    const R gH = -twoF * (ait[j] * fH[0] + ait[3 + j] * fH[1] + ait[6 + j] * fH[2]);
                    for (int l = 0; l < NH; ++l) rH[j][l] += R_at(f, m, l) * gH;
                }
            }
        }
    }

    // point source of the column (E equation)
    if (prm.src != nullptr) {
        const double* rec = prm.src + int64_t(s) * (SRC_HDR + 3 * NE);
        if (rec[0] >= 0.0 && int64_t(rec[0]) == e) {
            const double tt = prm.tdev ? *prm.tdev + prm.t : prm.t;
            const R g = R(src_time(tt, rec[1], rec[2], rec[3]));
            for (int c = 0; c < 3; ++c)
                for (int l = 0; l < NE; ++l) rE[c][l] -= g * R(rec[SRC_HDR + c * NE + l]);
        }
    }

    // 3x3 mass-block inverse A^T A / (material |det A|) per mode, then the update
    R at[9];
    at[0] = ait[4] * ait[8] - ait[5] * ait[7];
    at[1] = ait[2] * ait[7] - ait[1] * ait[8];
    at[2] = ait[1] * ait[5] - ait[2] * ait[4];
    at[3] = ait[5] * ait[6] - ait[3] * ait[8];
    at[4] = ait[0] * ait[8] - ait[2] * ait[6];
    at[5] = ait[2] * ait[3] - ait[0] * ait[5];
    at[6] = ait[3] * ait[7] - ait[4] * ait[6];
    at[7] = ait[1] * ait[6] - ait[0] * ait[7];
    at[8] = ait[0] * ait[4] - ait[1] * ait[3];
    for (int k = 0; k < 9; ++k) at[k] *= det;
    R G[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            G[j][k] = at[3 * j] * at[3 * k] + at[3 * j + 1] * at[3 * k + 1] + at[3 * j + 2] * at[3 * k + 2];
    const R ie = R(1) / (epsm * fabs(det)), ih = R(1) / (mum * fabs(det));
    R* uo = static_cast<R*>(prm.u_out);
    R* res = static_cast<R*>(prm.res);
    const R dt = sizeof(R) == 4 ? R(prm.dt_f) : R(prm.dt);
    const R ca = sizeof(R) == 4 ? R(prm.a_f) : R(prm.a);
    const R cb = sizeof(R) == 4 ? R(prm.b_f) : R(prm.b);
    auto update = [&](int64_t row, R du, R uv) {
        const int64_t gi = row * C + col;
        if (MODE == MODE_RHS) {
            uo[gi] = du;
        } else {
            const R rr = (ca == R(0) ? R(0) : ca * res[gi]) + dt * du;
            res[gi] = rr;
            uo[gi] = uv + cb * rr;
        }
    };
#pragma unroll 1
    for (int l = 0; l < NE; ++l)
        for (int j = 0; j < 3; ++j) {
            const R du = ie * (G[j][0] * rE[0][l] + G[j][1] * rE[1][l] + G[j][2] * rE[2][l]);
            update(int64_t(j) * NE + l, du, uE[j][l]);
        }
#pragma unroll 1
    for (int l = 0; l < NH; ++l)
        for (int j = 0; j < 3; ++j) {
            const R du = ih * (G[j][0] * rH[0][l] + G[j][1] * rH[1][l] + G[j][2] * rH[2][l]);
            update(rowH + int64_t(j) * NH + l, du, uH[j][l]);
        }
}

template <int PE, typename R>
int launch_mixed(const StageParams& prm, int mode, void* stream) {
    const int64_t C = prm.K_active * prm.S;
    if (C <= 0) return DGM_OK;
    StageParams q = prm;
    q.dt_f = float(prm.dt);
    q.a_f = float(prm.a);
    q.b_f = float(prm.b);
    const unsigned grid = unsigned((C + 127) / 128);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == MODE_RHS) mixed_stage_kernel<PE, R, MODE_RHS><<<grid, 128, 0, st>>>(q);
    else if (mode == MODE_LSRK) mixed_stage_kernel<PE, R, MODE_LSRK><<<grid, 128, 0, st>>>(q);
    else return DGM_EUNSUP;
    return cudaGetLastError() == cudaSuccess ? DGM_OK : DGM_ECUDA;
}

}  // namespace

#define MIXED_TABLE(PE, R, NAME, RS)                                                   \
    static int NAME##_launch(const StageParams& p, int mode, void* st) {              \
        return launch_mixed<PE, R>(p, mode, st);                                        \
    }                                                                                    \
    static const KernelTable NAME = {NAME##_launch, RS, nullptr, 1};
MIXED_TABLE(2, float, mixed_p2_f32, 4)
MIXED_TABLE(3, float, mixed_p3_f32, 4)
MIXED_TABLE(4, float, mixed_p4_f32, 4)
MIXED_TABLE(2, double, mixed_p2_f64, 8)
MIXED_TABLE(3, double, mixed_p3_f64, 8)
MIXED_TABLE(4, double, mixed_p4_f64, 8)
#undef MIXED_TABLE

// Kernels of mixed-order plans: E degree pE = 2..4 (H degree pE - 1).
const KernelTable* kernel_table_mixed(int pE, int precision) {
    static const KernelTable* f32[] = {nullptr, nullptr, &mixed_p2_f32, &mixed_p3_f32, &mixed_p4_f32};
    static const KernelTable* f64[] = {nullptr, nullptr, &mixed_p2_f64, &mixed_p3_f64, &mixed_p4_f64};
    if (pE < 2 || pE > 4) return nullptr;
    return precision == DGM_FP64 ? f64[pE] : (precision == DGM_FP32 ? f32[pE] : nullptr);
}

}  // namespace dgm
