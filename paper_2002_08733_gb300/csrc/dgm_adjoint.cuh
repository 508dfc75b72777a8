// Adjoint stage kernel: the transpose of the fused right-hand side, plus the
// material-gradient terms, for the discrete adjoint of LSRK4 time stepping.
//
// Forward (per element T, stage input u, see dgm_stage.cuh):
//   F_E = B_eps [ s curl_S(u_H) + sum_f R_f^T g_E,f + src ] - A^T eta A^-T u_E - p / eps
//   F_H = B_mu  [-s curl_S(u_E) + sum_f R_f^T g_H,f ]       - A^T eta A^-T u_H - q / mu
//   F_p = -A^T Sigma A^-T p + eps A^T xi A^-T u_E   (likewise q)
// with g_E = 2|F| A^-1 [c_E n x dH - b_E n x (n x dE)],
//      g_H = -2|F| A^-1 [c_H n x dE + b_H n x (n x dH)], dX = X+ - X-.
//
// Transpose applied to an adjoint vector lam (this kernel: lam = lr, the
// adjoint stage residual), rho = B lam per mode:
//   volume: (F^T lam)_E += s curl_{S^T}(rho_H), (F^T lam)_H -= s curl_{S^T}(rho_E)
//           (curl_S^T = -curl_{S^T}; S^T via the generated DerivTOp)
//   faces:  gamma = R_f rho (own), phi_E = 2|F| A^-T gamma_E, phi_H = -2|F| A^-T gamma_H;
//           adj(dH) = -c_E n x phi_E + b_H n x (n x phi_H),
//           adj(dE) = -b_E n x (n x phi_E) - c_H n x phi_H    (T as the "-" side),
//           the same from the neighbour's face with n -> -n, coefficients
//           of that face (c_E <-> c_H), and its own rho, gamma, phi; the
//           element's face-trace adjoint is A^-1 (adj(d)_nbr - adj(d)_own)
//           (PEC: A^-1 (-2 adj(dE)_own), nothing for H), lifted with R_f^T.
//   PML:    (F^T lam)_E -= (A^T eta A^-T)^T lam_E - eps (A^T xi A^-T)^T lam_p,
//           (F^T lam)_p  = -lam_E / eps - (A^T Sigma A^-T)^T lam_p.
// Gradient terms (per column; partial sums over a work item in the kernel's
// precision, their sum over items, stages and steps in FP64), dt times:
//   d/d eps_T: -(1/eps) rho_E . rhs_E(T) + lam_E . p / eps^2 + lam_p . (A^T xi A^-T u_E)
//              - Z/(2 eps) dJ/dZ_T
//   d/d mu_T:  -(1/mu) rho_H . rhs_H(T) + lam_H . q / mu^2 + lam_q . (A^T xi A^-T u_H)
//              + Z/(2 mu) dJ/dZ_T
// where dJ/dZ_T collects phi . d(flux)/dZ over the element's faces (its own
// face equations, Z = Z^-) and over its neighbours' equations on the shared
// faces (Z = Z^+ there), evaluated with the forward jumps d of this face,
// which the neighbour sees as -d.
#pragma once

#include <cstdint>

#include "dgm_stage.cuh"

namespace dgm {

constexpr int FGA = 21;   // face constants of the adjoint: FG + neighbour det, eps, mu
enum AdjFaceConst { FA_DETN = 18, FA_EPSN = 19, FA_MUN = 20 };

// B = A^T A / (mat |det|) from A^-T (row major) and det A: b[3][3]
template <typename R>
__device__ __forceinline__ void mass_block(const R (&ait)[9], R det, R mat, R (&b)[3][3], R (&AT)[3][3]) {
    AT[0][0] = ait[4] * ait[8] - ait[5] * ait[7];
    AT[0][1] = ait[2] * ait[7] - ait[1] * ait[8];
    AT[0][2] = ait[1] * ait[5] - ait[2] * ait[4];
    AT[1][0] = ait[5] * ait[6] - ait[3] * ait[8];
    AT[1][1] = ait[0] * ait[8] - ait[2] * ait[6];
    AT[1][2] = ait[2] * ait[3] - ait[0] * ait[5];
    AT[2][0] = ait[3] * ait[7] - ait[4] * ait[6];
    AT[2][1] = ait[1] * ait[6] - ait[0] * ait[7];
    AT[2][2] = ait[0] * ait[4] - ait[1] * ait[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) AT[a][c] *= det;
    const R inv = R(1) / (mat * fabs(det));
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            b[j][k] = inv * (AT[j][0] * AT[k][0] + AT[j][1] * AT[k][1] + AT[j][2] * AT[k][2]);
}

template <typename R>
__device__ __forceinline__ void matvec3(const R (&m)[3][3], const R (&v)[3], R (&o)[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) o[r] = m[r][0] * v[0] + m[r][1] * v[1] + m[r][2] * v[2];
}

// A^-T v (ait row major) and A^-1 v
template <typename R>
__device__ __forceinline__ void ait_mul(const R (&a)[9], const R (&v)[3], R (&o)[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) o[r] = a[3 * r] * v[0] + a[3 * r + 1] * v[1] + a[3 * r + 2] * v[2];
}
template <typename R>
__device__ __forceinline__ void ai_mul(const R (&a)[9], const R (&v)[3], R (&o)[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) o[r] = a[r] * v[0] + a[3 + r] * v[1] + a[6 + r] * v[2];
}

// adjoint volume term rows [LO, HI) of component comp plus the lift of zeta
template <int P, typename R, int TE, int LO, int HI>
__device__ __forceinline__ void adj_rows(int comp, int c, const R* rs, const R* trO, R sgn,
                                         R (&acc)[nmodes(P)]) {
    constexpr int N = nmodes(P);
    constexpr int NF = nfmodes(P);
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l] = R(0);
    const int j = comp % 3;
    const int srcf = comp < 3 ? 3 : 0;
    const R sg = comp < 3 ? sgn : -sgn;
    const R* base = rs + c;
    switch (j) {
        case 0:
            DerivTOp<P, 1>::template apply<R, LO, HI>(base + (srcf + 2) * N * TE, TE, sg, acc);
            DerivTOp<P, 2>::template apply<R, LO, HI>(base + (srcf + 1) * N * TE, TE, -sg, acc);
            break;
        case 1:
            DerivTOp<P, 2>::template apply<R, LO, HI>(base + (srcf + 0) * N * TE, TE, sg, acc);
            DerivTOp<P, 0>::template apply<R, LO, HI>(base + (srcf + 2) * N * TE, TE, -sg, acc);
            break;
        default:
            DerivTOp<P, 0>::template apply<R, LO, HI>(base + (srcf + 1) * N * TE, TE, sg, acc);
            DerivTOp<P, 1>::template apply<R, LO, HI>(base + (srcf + 0) * N * TE, TE, -sg, acc);
            break;
    }
    LiftOp<P, 0>::template apply<R, LO, HI>(trO + ((0 * 6 + comp) * NF) * TE + c, TE, acc);
    LiftOp<P, 1>::template apply<R, LO, HI>(trO + ((1 * 6 + comp) * NF) * TE + c, TE, acc);
    LiftOp<P, 2>::template apply<R, LO, HI>(trO + ((2 * 6 + comp) * NF) * TE + c, TE, acc);
    LiftOp<P, 3>::template apply<R, LO, HI>(trO + ((3 * 6 + comp) * NF) * TE + c, TE, acc);
}

template <int P, typename R, int TE, int NPART>
__device__ __forceinline__ void adj_part(int part, int comp, int c, const R* rs, const R* trO,
                                         R sgn, R (&acc)[nmodes(P)]) {
    constexpr int N = nmodes(P);
    switch (part) {
        case 0: adj_rows<P, R, TE, 0, (NPART == 1 ? N : N / NPART)>(comp, c, rs, trO, sgn, acc); break;
        case 1: adj_rows<P, R, TE, N / NPART, (NPART == 2 ? N : 2 * N / NPART)>(comp, c, rs, trO, sgn, acc); break;
        case 2: adj_rows<P, R, TE, 2 * N / NPART, (NPART == 3 ? N : 3 * N / NPART)>(comp, c, rs, trO, sgn, acc); break;
        default: adj_rows<P, R, TE, 3 * N / NPART, N>(comp, c, rs, trO, sgn, acc); break;
    }
}

template <int P, typename R, int TE, int NT>
__device__ __host__ constexpr size_t adjoint_smem_bytes() {
    constexpr int NG = NT / TE;
    constexpr int NPART = NG >= 24 ? 4 : (NG >= 12 ? 2 : 1);
    constexpr int CH = NG >= 12 ? NG / 4 : 1;
    return sizeof(R) * size_t(TE) * (12 * nmodes(P) + 48 * nfmodes(P) + 4 * FGA + EG) +
           sizeof(double) * size_t(TE) * (4 * CH + 2 * 6 * NPART);
}

// IX: index type (uint32_t when every index of the plan fits, else int64_t)
template <int P, typename R, int TE, int NT, typename IX = int64_t>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 && P <= 3 ? 2 : 1) adjoint_kernel(const AdjParams prm) {
    constexpr int N = nmodes(P);
    constexpr int NF = nfmodes(P);
    constexpr int NG = NT / TE;
    constexpr int NPART = NG >= 24 ? 4 : (NG >= 12 ? 2 : 1);
    constexpr int CH = NG >= 12 ? NG / 4 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* us = reinterpret_cast<R*>(smem_raw);      // [6N][TE]  lam
    R* rs = us + 6 * N * TE;                     // [6N][TE]  rho = B lam
    R* trO = rs + 6 * N * TE;                    // [4][6][NF][TE] gamma -> zeta
    R* trN = trO + 24 * NF * TE;                 // [4][6][NF][TE] nbr lam traces -> F^T lam
    R* fg = trN + 24 * NF * TE;                  // [4][FGA][TE]
    R* eg = fg + 4 * FGA * TE;                   // [EG][TE]
    double* zs = reinterpret_cast<double*>(eg + EG * TE);   // [4 CH][TE]   dJ/dZ partials
    double* gp = zs + 4 * CH * TE;                           // [2][6 NPART][TE] gradient partials

    const int c = threadIdx.x % TE;
    const int grp = threadIdx.x / TE;
    const IX K = prm.K;
    const int S = prm.S;
    const IX C = K * S;
    const IX col = IX(tile_index(prm.tile_groups)) * TE + c;
    const bool active = col < C;
    const IX e = active ? col / S : 0;
    const int s = active ? int(col - e * S) : 0;
    const R* lam = static_cast<const R*>(prm.lr);

    // ---- 1: adjoint residual tile, element and face constants -------------------
    // Groups 0..3: face constants of face f = group from the element's geometry
    // and the per-face neighbour table.  Other groups: the tile of lam and the
    // element constants (all loads of a thread in flight before its first
    // shared-memory store) and the neighbour lam of their first phase-2 item.
    const R* gr = static_cast<const R*>(prm.geo_r);
    constexpr int FACE_GROUPS = NG > 4 ? 4 : 0;
    constexpr int LG = NG - FACE_GROUPS;
    R vn[N];
    bool vn_ready = false;
    auto face_consts = [&](int f) {
        R ait[9], aitn[9];
        const R* fn = static_cast<const R*>(prm.fnb_r) + IX(f * FNB_COUNT) * K + e;
        const int32_t code = active ? prm.nbr[IX(f) * K + e] : -1;
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = active ? gr[IX(G_AIT + k) * K + e] : R(k % 4 == 0);
#pragma unroll
        for (int k = 0; k < 9; ++k) aitn[k] = active ? fn[IX(FNB_AIT + k) * K] : ait[k];
        const R det = active ? gr[IX(G_DET) * K + e] : R(1);
        const R epsm = active ? gr[IX(G_EPS) * K + e] : R(1);
        const R mum = active ? gr[IX(G_MU) * K + e] : R(1);
        const R zn = active ? fn[IX(FNB_Z) * K] : R(1);
        const bool has = code >= 0 && (code >> 2) < K;
        R* fc = fg + f * FGA * TE + c;
        face_constants_tab<R, TE>(f, ait, det, epsm, mum, has, aitn, zn, prm.upwind, fc);
        fc[FA_DETN * TE] = has ? fn[IX(FNB_DET) * K] : det;
        fc[FA_EPSN * TE] = has ? fn[IX(FNB_EPS) * K] : epsm;
        fc[FA_MUN * TE] = has ? fn[IX(FNB_MU) * K] : mum;
    };
    if (grp < FACE_GROUPS) {
        face_consts(grp);
    } else {
        const int lg = grp - FACE_GROUPS;
        constexpr int UR = (6 * N + LG - 1) / LG;
        constexpr int ER = (EG + LG - 1) / LG;
        constexpr int BATCH = 16;
        R tmp[BATCH];
#pragma unroll
        for (int i = 0; i < BATCH; ++i) {
            const int r = lg + i * LG;
            tmp[i] = (i < UR && r < 6 * N && active) ? lam[IX(r) * C + col] : R(0);
        }
        if (grp < 24 && active) {   // round-0 item of phase 2: face grp / 6, component grp % 6
            const int32_t code = prm.nbr[IX(grp / 6) * K + e];
            const IX ne = code >> 2;
            if (code >= 0 && ne < K) {
                const IX ncol = ne * S + s;
#pragma unroll
                for (int l = 0; l < N; ++l) vn[l] = lam[IX((grp % 6) * N + l) * C + ncol];
                vn_ready = true;
            }
        }
#pragma unroll
        for (int i0 = 0; i0 < UR; i0 += BATCH) {
            if (i0 > 0) {
#pragma unroll
                for (int i = 0; i < BATCH; ++i) {
                    const int r = lg + (i0 + i) * LG;
                    tmp[i] = (i0 + i < UR && r < 6 * N && active) ? lam[IX(r) * C + col] : R(0);
                }
            }
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int r = lg + (i0 + i) * LG;
                if (i0 + i < UR && r < 6 * N) us[r * TE + c] = tmp[i];
            }
        }
        R tmpe[ER];
#pragma unroll
        for (int i = 0; i < ER; ++i) {
            const int k = lg + i * LG;
            tmpe[i] = (k < EG && active) ? gr[IX(k) * K + e]
                                         : R(k == G_DET || k == G_EPS || k == G_MU ? 1 : 0);
        }
#pragma unroll
        for (int i = 0; i < ER; ++i) {
            const int k = lg + i * LG;
            if (k < EG) eg[k * TE + c] = tmpe[i];
        }
        for (int i = lg; i < 4 * CH; i += LG) zs[i * TE + c] = 0.0;
        for (int i = lg; i < 2 * 6 * NPART; i += LG) gp[i * TE + c] = 0.0;
    }
    if (FACE_GROUPS == 0) {
        for (int f = grp; f < 4; f += NG) face_consts(f);
    }
    __syncthreads();
    // rho = B lam per mode (field fb, rows [lo, hi))
    for (int it = grp; it < 2 * NPART; it += NG) {
        const int fb = (it / NPART) * 3;
        const int part = it % NPART;
        R ait[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = eg[(G_AIT + k) * TE + c];
        R b[3][3], AT[3][3];
        mass_block(ait, eg[G_DET * TE + c], fb == 0 ? eg[G_EPS * TE + c] : eg[G_MU * TE + c], b, AT);
        for (int l = part * N / NPART; l < (part + 1) * N / NPART; ++l) {
            R v[3], o[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = us[((fb + k) * N + l) * TE + c];
            matvec3(b, v, o);
#pragma unroll
            for (int k = 0; k < 3; ++k) rs[((fb + k) * N + l) * TE + c] = o[k];
        }
    }
    __syncthreads();

    // ---- 2: traces: own of rho (= gamma), neighbour of lam ------------------------
    for (int r = grp; r < 24; r += NG) {
        const int f = r / 6, comp = r % 6;
        const int32_t code = active ? prm.nbr[IX(f) * K + e] : -1;
        const IX ne = code >> 2;
        const bool has_nbr = code >= 0 && ne < K;
        if (code >= 0 && ne >= K) atomicOr(prm.status, ST_BAD_NEIGHBOUR);
        if (has_nbr && !(r == grp && vn_ready)) {
            const IX ncol = ne * S + s;
#pragma unroll
            for (int l = 0; l < N; ++l) vn[l] = lam[IX(comp * N + l) * C + ncol];
        }
        R v[N], acc[NF];
#pragma unroll
        for (int l = 0; l < N; ++l) v[l] = rs[(comp * N + l) * TE + c];
        trace_any<P, R>(f, v, acc);
        R* dst = trO + ((f * 6 + comp) * NF) * TE + c;
#pragma unroll
        for (int m = 0; m < NF; ++m) dst[m * TE] = acc[m];
        if (has_nbr) {
            trace_any<P, R>(code & 3, vn, acc);
        } else {
#pragma unroll
            for (int m = 0; m < NF; ++m) acc[m] = R(0);
        }
        dst = trN + ((f * 6 + comp) * NF) * TE + c;
#pragma unroll
        for (int m = 0; m < NF; ++m) dst[m * TE] = acc[m];
    }
    __syncthreads();

    // ---- 3: transposed flux per (face, chunk of face modes) + dJ/dZ ---------------
    for (int it = grp; it < 4 * CH; it += NG) {
        const int f = it / CH;
        const int ch = it % CH;
        const R* d = fg + f * FGA * TE + c;
        R ait[9], aitn[9], n[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            ait[k] = eg[(G_AIT + k) * TE + c];
            aitn[k] = d[(FC_AITN + k) * TE];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) n[r] = d[(FC_N + r) * TE];
        const bool bnd = d[FC_BND * TE] != R(0);
        const R twoF = d[FC_TWOF * TE];
        const R ce = d[FC_CE * TE], be = d[FC_BE * TE], chh = d[FC_CH * TE], bh = d[FC_BH * TE];
        // phi of the neighbour's side = +-2|F| A_n^-T B_n t: the two 3x3 products
        // formed once per item (fewer live values across the mode loop)
        R ME[3][3], MH[3][3];
        {
            R bNe[3][3], bNh[3][3], ATn[3][3];
            mass_block(aitn, d[FA_DETN * TE], d[FA_EPSN * TE], bNe, ATn);
            mass_block(aitn, d[FA_DETN * TE], d[FA_MUN * TE], bNh, ATn);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ME[r][k] = twoF * (aitn[3 * r] * bNe[0][k] + aitn[3 * r + 1] * bNe[1][k] + aitn[3 * r + 2] * bNe[2][k]);
                    MH[r][k] = -twoF * (aitn[3 * r] * bNh[0][k] + aitn[3 * r + 1] * bNh[1][k] + aitn[3 * r + 2] * bNh[2][k]);
                }
        }
        // impedances for dJ/dZ (upwind only)
        const R zm = sqrt(eg[G_MU * TE + c] / eg[G_EPS * TE + c]);
        const R zp = bnd ? zm : sqrt(d[FA_MUN * TE] / d[FA_EPSN * TE]);
        const R D = (zm + zp) * (zm + zp);
        const R* jp = static_cast<const R*>(prm.jumps);
        R zacc = R(0);   // partial sums in the kernel's precision, FP64 from phase 6 on
        for (int m = ch * NF / CH; m < (ch + 1) * NF / CH; ++m) {
            R* own = trO + (f * 6 * NF + m) * TE + c;
            const R* nbt = trN + (f * 6 * NF + m) * TE + c;
            R gE[3], gH[3], phiE[3], phiH[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gE[k] = own[k * NF * TE];
                gH[k] = own[(3 + k) * NF * TE];
            }
            ait_mul(ait, gE, phiE);
            ait_mul(ait, gH, phiH);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                phiE[k] *= twoF;
                phiH[k] *= -twoF;
            }
            R t1[3], t2[3], aE[3], aH[3];
            // own face: adj(dH) = -cE n x phiE + bH n x (n x phiH); adj(dE) = -bE n x (n x phiE) - cH n x phiH
            cross3(n, phiE, t1);
            cross3(n, t1, t2);   // n x (n x phiE)
            R nxphH[3], nnxphH[3];
            cross3(n, phiH, nxphH);
            cross3(n, nxphH, nnxphH);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                aH[r] = -ce * t1[r] + bh * nnxphH[r];
                aE[r] = -be * t2[r] - chh * nxphH[r];
            }
            R zE[3], zH[3], vE[3], vH[3];
            R phiEn[3] = {0, 0, 0}, phiHn[3] = {0, 0, 0};
            if (bnd) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    vE[r] = R(-2) * aE[r];
                    vH[r] = R(0);
                }
            } else {
                R tn[3], tnh[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    tn[k] = nbt[k * NF * TE];
                    tnh[k] = nbt[(3 + k) * NF * TE];
                }
                matvec3(ME, tn, phiEn);
                matvec3(MH, tnh, phiHn);
                // neighbour's face (normal -n, c_E <-> c_H):
                // adj(dH)_N = cH n x phiE_N + bH n x (n x phiH_N); adj(dE)_N = -bE n x (n x phiE_N) + cE n x phiH_N
                R a1[3], a2[3], b1[3], b2[3];
                cross3(n, phiEn, a1);
                cross3(n, a1, a2);
                cross3(n, phiHn, b1);
                cross3(n, b1, b2);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    vH[r] = (chh * a1[r] + bh * b2[r]) - aH[r];
                    vE[r] = (-be * a2[r] + ce * b1[r]) - aE[r];
                }
            }
            ai_mul(ait, vE, zE);
            ai_mul(ait, vH, zH);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                own[k * NF * TE] = zE[k];
                own[(3 + k) * NF * TE] = zH[k];
            }
            if (prm.upwind && active) {
                R dE[3], dH[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    dE[r] = jp[IX((f * 6 + r) * NF + m) * C + col];
                    dH[r] = jp[IX((f * 6 + 3 + r) * NF + m) * C + col];
                }
                R nxdE[3], nnxdE[3], nxdH[3], nnxdH[3];
                cross3(n, dE, nxdE);
                cross3(n, nxdE, nnxdE);
                cross3(n, dH, nxdH);
                cross3(n, nxdH, nnxdH);
                R z = R(0);
                if (bnd) {
                    // Z+ = Z- = Z: d b_E/dZ = -1/(2 Z^2) on the -b_E n x (n x dE) term
                    const R ib = R(1) / (R(2) * zm * zm);
#pragma unroll
                    for (int r = 0; r < 3; ++r) z += phiE[r] * nnxdE[r] * ib;
                } else {
                    const R iD = R(1) / D;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        // own equations (derivative in Z-)
                        z += phiE[r] * (-zp * iD * nxdH[r] + iD * nnxdE[r]) +
                             phiH[r] * (zp * iD * nxdE[r] + zp * zp * iD * nnxdH[r]);
                        // neighbour's equations (derivative in its Z+ = this element's Z)
                        z += phiEn[r] * (zp * iD * nxdH[r] - iD * nnxdE[r]) +
                             phiHn[r] * (-zp * iD * nxdE[r] - zp * zp * iD * nnxdH[r]);
                    }
                }
                zacc += z;
            }
        }
        zs[it * TE + c] = double(zacc);
    }
    __syncthreads();

    // ---- 4: transposed volume term + lift per (component, row part) ---------------
    R* rh = trN;   // [6][N][TE]
    for (int it = grp; it < 6 * NPART; it += NG) {
        const int comp = it / NPART;
        const int part = it % NPART;
        const R sgn = eg[G_DET * TE + c] < R(0) ? R(-1) : R(1);
        R acc[N];
        adj_part<P, R, TE, NPART>(part, comp, c, rs, trO, sgn, acc);
        const int lo = part * N / NPART, hi = (part + 1) * N / NPART;
#pragma unroll
        for (int l = 0; l < N; ++l)
            if (l >= lo && l < hi) rh[(comp * N + l) * TE + c] = acc[l];
    }
    __syncthreads();

    // ---- 5: PML transposes, adjoint update, gradient partials -----------------------
    for (int it = grp; it < 6 * NPART; it += NG) {
        const int comp = it / NPART;
        const int part = it % NPART;
        if (!active) continue;
        const int j = comp % 3;
        const int fb = comp < 3 ? 0 : 3;
        R ait[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = eg[(G_AIT + k) * TE + c];
        const R det = eg[G_DET * TE + c];
        const R mat = comp < 3 ? eg[G_EPS * TE + c] : eg[G_MU * TE + c];
        R bb[3][3], AT[3][3];
        mass_block(ait, det, mat, bb, AT);
        int32_t pi = -1;
        if (prm.pml != nullptr) pi = prm.pml[e];
        // columns j of A^T D A^-T (transposed rows): (A^T D A^-T)[k][j] = sum_a AT[k][a] D_a Ait[a][j]
        R etaT[3] = {0, 0, 0}, sigT[3] = {0, 0, 0}, xiT[3] = {0, 0, 0}, xiR[3] = {0, 0, 0};
        if (pi >= 0) {
            const R sx = eg[(G_SIG + 0) * TE + c], sy = eg[(G_SIG + 1) * TE + c], sz = eg[(G_SIG + 2) * TE + c];
            const R sg3[3] = {sx, sy, sz};
            const R et3[3] = {sy + sz - sx, sz + sx - sy, sx + sy - sz};
            const R xi3[3] = {(sx - sy) * (sx - sz), (sy - sz) * (sy - sx), (sz - sx) * (sz - sy)};
            const R aj[3] = {ait[j], ait[3 + j], ait[6 + j]};     // column j of A^-T
            R atj[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) atj[b] = j == 0 ? AT[0][b] : (j == 1 ? AT[1][b] : AT[2][b]);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const R w = AT[k][a] * aj[a];        // transposed: row k, column j
                    etaT[k] += w * et3[a];
                    sigT[k] += w * sg3[a];
                    xiT[k] += w * xi3[a];
                    xiR[k] += atj[a] * xi3[a] * ait[3 * a + k];   // row j (forward) for the gradient
                }
        }
        const IX C2 = IX(prm.npml) * S;
        const IX acol = IX(pi) * S + s;
        R* lu = static_cast<R*>(prm.lu);
        const R* lra = static_cast<const R*>(prm.lr_aux);
        R* lua = static_cast<R*>(prm.lu_aux);
        const R* uf = static_cast<const R*>(prm.u);
        const R* af = static_cast<const R*>(prm.aux);
        const R* raw = static_cast<const R*>(prm.raw);
        const R dt = R(prm.dt);
        R gmass = R(0), gpml = R(0);   // partial sums in the kernel's precision
        const int lo = part * N / NPART, hi = (part + 1) * N / NPART;
        // the item's forward right-hand-side and adjoint rows, all requested
        // before the arithmetic so that their round trips overlap
        constexpr int RP = (N + NPART - 1) / NPART;
        R rawv[RP], luv[RP];
#pragma unroll
        for (int i = 0; i < RP; ++i) {
            const bool ok = lo + i < hi;
            const IX gi = IX(comp * N + lo + i) * C + col;
            rawv[i] = ok ? raw[gi] : R(0);
            luv[i] = ok ? lu[gi] : R(0);
        }
#pragma unroll
        for (int i = 0; i < RP; ++i) {
            const int l = lo + i;
            if (l >= hi) break;
            R w = rh[(comp * N + l) * TE + c];
            const IX gi = IX(comp * N + l) * C + col;
            // mass term of the gradient: -(1/mat) rho_c . rhs_c
            gmass += rs[(comp * N + l) * TE + c] * rawv[i];
            if (pi >= 0) {
                const R l0 = us[((fb + 0) * N + l) * TE + c];
                const R l1 = us[((fb + 1) * N + l) * TE + c];
                const R l2 = us[((fb + 2) * N + l) * TE + c];
                const IX ai = IX(fb * N + l) * C2 + acol;
                const R p0 = lra[ai], p1 = lra[ai + IX(N) * C2], p2 = lra[ai + 2 * IX(N) * C2];
                w -= etaT[0] * l0 + etaT[1] * l1 + etaT[2] * l2;
                w += mat * (xiT[0] * p0 + xiT[1] * p1 + xiT[2] * p2);
                const R lj = j == 0 ? l0 : (j == 1 ? l1 : l2);
                const R pj = j == 0 ? p0 : (j == 1 ? p1 : p2);
                const R wa = -lj / mat - (sigT[0] * p0 + sigT[1] * p1 + sigT[2] * p2);
                const IX aj2 = IX(comp * N + l) * C2 + acol;
                lua[aj2] += dt * wa;
                // PML gradient terms: lam_j p_j / mat^2 + lam_aux_j (A^T xi A^-T u)_j
                const R apj = af[aj2];
                const R u0 = uf[IX((fb + 0) * N + l) * C + col];
                const R u1 = uf[IX((fb + 1) * N + l) * C + col];
                const R u2 = uf[IX((fb + 2) * N + l) * C + col];
                gpml += lj * apj / (mat * mat) + pj * (xiR[0] * u0 + xiR[1] * u1 + xiR[2] * u2);
            }
            lu[gi] = luv[i] + dt * w;
        }
        const int slot = comp < 3 ? 0 : 1;
        gp[(slot * 6 * NPART + it) * TE + c] = double(-gmass / mat + gpml);
    }
    __syncthreads();

    // ---- 6: per-column gradient (one owner thread per column, fixed order) --------
    if (grp == 0 && active) {
        const double eps = prm.geo[IX(G_EPS) * K + e], mu = prm.geo[IX(G_MU) * K + e];
        const double Z = sqrt(mu / eps);
        double dz = 0.0, ge = 0.0, gm = 0.0;
        for (int i = 0; i < 4 * CH; ++i) dz += zs[i * TE + c];
        for (int i = 0; i < 6 * NPART; ++i) {
            ge += gp[(0 * 6 * NPART + i) * TE + c];
            gm += gp[(1 * 6 * NPART + i) * TE + c];
        }
        ge += -Z / (2.0 * eps) * dz;
        gm += Z / (2.0 * mu) * dz;
        prm.grad[col] += prm.dt * ge;
        prm.grad[C + col] += prm.dt * gm;
    }
}

}  // namespace dgm
