// Fused DG right-hand-side / stage-update kernel (SIMT, FP64 or FP32).
//
// One CTA owns a tile of TE consecutive columns (column = element * S +
// source) and evaluates, for each of them, the whole semi-discrete right-hand
// side of Secs. III-IV in the strong form
//
//   d u_E/dt = B_eps [ s_T curl_ref(u_H) + sum_f R_f^T g_E,f - w_src g(t) ]
//              - A^T eta A^-T u_E - p / eps
//   d u_H/dt = B_mu  [-s_T curl_ref(u_E) + sum_f R_f^T g_H,f ]
//              - A^T eta A^-T u_H - q / mu
//   d p/dt   = -A^T Sigma A^-T p + eps A^T xi A^-T u_E   (likewise q)
//
// where u are covariant modal coefficients (Eq. (mapped_eh)),
// curl_ref uses the geometry-free derivative matrices S_a (Eq.
// (matrix_free_curl); the Piola map, Eq. (piola_transf), leaves only the
// orientation sign s_T = sign det A), B = (A^T A) / (material |det A|) is the
// inverse of the at-most 3x3 block mass matrix (Sec. II), R_f are the
// geometry-free trace matrices onto face f, and g_f = 2|F| A^-1 flux_f are the
// face-mode coefficients of the numerical flux pulled back to the element:
//   flux_E = c_E n x dH - b_E n x (n x dE),  flux_H = c_H n x dE + b_H n x (n x dH)
// with dX = X+ - X- the jump of the physical traces (X = A^-T x_ref per side),
// central (c = 1/2, b = 0, Eqs. (uwc)/(cwc)) or upwind coefficients, and the
// PEC ghost state e+ = -e-, h+ = h- on boundary faces.
//
// Phases (separated by __syncthreads):
//   1 load the tile's coefficients into shared memory, element geometry
//   2 own traces (4 faces x 6 components) from shared memory, neighbour traces
//     from global memory (the neighbour's coefficients are usually L2 hits),
//     face constants (normal, neighbour map, flux coefficients)
//   3 numerical flux per (face, face mode), pulled back to the element
//   4 right-hand side per component: volume curl + lift (+ source)
//   5 3x3 mass-block inverse, PML terms, and the stage update
// The reference operators are straight-line code with literal coefficients
// (generated at build time, dgm_refgen.cpp) that visits only the non-zero
// entries: S_a[l][m] = 0 unless deg(l) < deg(m), R_f[m][l] = 0 unless
// deg(m) <= deg(l) (hierarchical orthonormal bases), and many more entries
// vanish exactly for the collapsed basis (e.g. on the face x = 0 each mode
// has a single face mode).
#pragma once

#include <cstdint>

#include "dgm_internal.h"
#include "dgm_ops_gen.cuh"

namespace dgm {

// offset of the first mode of total degree d (3-D) and (2-D)
__host__ __device__ constexpr int off3(int d) { return d <= 0 ? 0 : nmodes(d - 1); }
__host__ __device__ constexpr int off2(int d) { return d <= 0 ? 0 : nfmodes(d - 1); }

constexpr int FG = 18;   // face constants per (face, column)
enum FaceConst {
    FC_N = 0,     // unit outward normal (3)
    FC_AITN = 3,  // neighbour A^-T (9), own A^-T on PEC faces
    FC_CE = 12, FC_BE = 13, FC_CH = 14, FC_BH = 15,
    FC_TWOF = 16, // 2 |F|
    FC_BND = 17   // 1 on a PEC face
};
constexpr int EG = 16;   // element constants per column (same slots as G_*)

template <int P, typename R, int TE>
__host__ __device__ constexpr size_t stage_smem_bytes() {
    return sizeof(R) * size_t(TE) *
           (6 * nmodes(P) + 48 * nfmodes(P) + 4 * FG + EG);
}

// Reference operators: straight-line code with literal coefficients generated
// at build time from the library's own reference matrices (dgm_refgen.cpp),
// visiting only the entries that are not zero.
template <int P, typename R, int F>
__device__ __forceinline__ void trace_face(const R (&v)[nmodes(P)], R (&acc)[nfmodes(P)]) {
    TraceOp<P, F>::template apply<R>(v, acc);
}

template <int P, typename R>
__device__ __forceinline__ void trace_any(int f, const R (&v)[nmodes(P)], R (&acc)[nfmodes(P)]) {
    switch (f) {
        case 0: trace_face<P, R, 0>(v, acc); break;
        case 1: trace_face<P, R, 1>(v, acc); break;
        case 2: trace_face<P, R, 2>(v, acc); break;
        default: trace_face<P, R, 3>(v, acc); break;
    }
}

// acc[l] += sign * sum_m S[a][l][m] v[m]
template <int P, typename R, int A>
__device__ __forceinline__ void deriv_acc(const R* vs, int stride, R sign, R (&acc)[nmodes(P)]) {
    DerivOp<P, A>::template apply<R>(vs, stride, sign, acc);
}

// acc[l] += sum_m R[f][m][l] g[m]
template <int P, typename R, int F>
__device__ __forceinline__ void lift_face(const R* gs, int stride, R (&acc)[nmodes(P)]) {
    LiftOp<P, F>::template apply<R>(gs, stride, acc);
}

template <typename R>
__device__ __forceinline__ void cross3(const R a[3], const R b[3], R o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// source time function g(t) = sin(2 pi f0 (t - t0)) exp(-(t - t0)^2 / (2 s^2)), s = 1/(2 pi bw)
__device__ __forceinline__ double source_time(double t, double f0, double bw, double t0) {
    const double twopi = 6.283185307179586476925286766559;
    const double s = 1.0 / (twopi * bw);
    const double tau = t - t0;
    return sin(twopi * f0 * tau) * exp(-tau * tau / (2.0 * s * s));
}

template <int P, typename R, int TE, int NT, int MODE>
__global__ void __launch_bounds__(NT) stage_kernel(const StageParams prm) {
    constexpr int N = nmodes(P);
    constexpr int NF = nfmodes(P);
    constexpr int NG = NT / TE;
    constexpr bool DO_E = (MODE != MODE_LF_H);   // E equation updated
    constexpr bool DO_H = (MODE != MODE_LF_E);   // H equation updated
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* us = reinterpret_cast<R*>(smem_raw);      // [6N][TE]
    R* trO = us + 6 * N * TE;                    // [4][6][NF][TE]  own traces -> g
    R* trN = trO + 24 * NF * TE;                 // [4][6][NF][TE]  nbr traces -> rhs [6][N][TE]
    R* fg = trN + 24 * NF * TE;                  // [4][FG][TE]
    R* eg = fg + 4 * FG * TE;                    // [EG][TE]

    const int c = threadIdx.x % TE;
    const int grp = threadIdx.x / TE;
    const int64_t K = prm.K;
    const int S = prm.S;
    const int64_t C = K * S;
    const int64_t col = int64_t(blockIdx.x) * TE + c;
    const bool active = col < C;
    const int64_t e = active ? col / S : 0;
    const int s = active ? int(col - e * S) : 0;
    const R* u = static_cast<const R*>(prm.u);   // may alias u_out (leapfrog)

    // ---- phase 1: tile coefficients and element constants -------------------
    for (int r = grp; r < 6 * N; r += NG) us[r * TE + c] = active ? u[int64_t(r) * C + col] : R(0);
    for (int k = grp; k < EG; k += NG)
        eg[k * TE + c] = active ? R(prm.geo[int64_t(k) * K + e]) : R(k == G_DET || k == G_EPS || k == G_MU ? 1 : 0);
    __syncthreads();

    // ---- phase 2: traces and face constants ---------------------------------
    // items 0..23: own traces (f, comp); 24..47: neighbour traces; 48..51: face constants
    for (int it = grp; it < 52; it += NG) {
        if (it < 48) {
            const int side = it / 24;
            const int f = (it / 6) % 4;
            const int comp = it % 6;
            // a leapfrog half step only needs the traces of the other field
            if (MODE == MODE_LF_E && comp < 3) continue;
            if (MODE == MODE_LF_H && comp >= 3) continue;
            R v[N];
            R acc[NF];
            R* dst = (side == 0 ? trO : trN) + ((f * 6 + comp) * NF) * TE + c;
            if (side == 0) {
#pragma unroll
                for (int l = 0; l < N; ++l) v[l] = us[(comp * N + l) * TE + c];
                trace_any<P, R>(f, v, acc);
            } else {
                const int32_t code = active ? prm.nbr[int64_t(f) * K + e] : -1;
                if (code < 0) {
#pragma unroll
                    for (int m = 0; m < NF; ++m) acc[m] = R(0);
                } else {
                    const int64_t ne = code >> 2;
                    const int fp = code & 3;
                    const int64_t ncol = ne * S + s;
                    if (ne >= K) {
                        atomicOr(prm.status, ST_BAD_NEIGHBOUR);
#pragma unroll
                        for (int m = 0; m < NF; ++m) acc[m] = R(0);
                    } else {
#pragma unroll
                        for (int l = 0; l < N; ++l) v[l] = u[int64_t(comp * N + l) * C + ncol];
                        trace_any<P, R>(fp, v, acc);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < NF; ++m) dst[m * TE] = acc[m];
        } else {
            const int f = it - 48;
            R ait[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) ait[k] = eg[(G_AIT + k) * TE + c];
            const R det = eg[G_DET * TE + c];
            // 2|F_hat| n_hat of reference face f: (1,1,1), (-1,0,0), (0,-1,0), (0,0,-1)
            R mref[3] = {R(f == 0 ? 1 : (f == 1 ? -1 : 0)), R(f == 0 ? 1 : (f == 2 ? -1 : 0)),
                         R(f == 0 ? 1 : (f == 3 ? -1 : 0))};
            R vn[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                vn[r] = ait[3 * r + 0] * mref[0] + ait[3 * r + 1] * mref[1] + ait[3 * r + 2] * mref[2];
            const R fs = sqrt(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
            R* d = fg + f * FG * TE + c;
#pragma unroll
            for (int r = 0; r < 3; ++r) d[(FC_N + r) * TE] = vn[r] / fs;
            d[FC_TWOF * TE] = fabs(det) * fs;
            const R epsm = eg[G_EPS * TE + c], mum = eg[G_MU * TE + c];
            const R zm = sqrt(mum / epsm);
            const int32_t code = active ? prm.nbr[int64_t(f) * K + e] : -1;
            R zp = zm;
            if (code >= 0 && (code >> 2) < K) {
                const int64_t ne = code >> 2;
#pragma unroll
                for (int k = 0; k < 9; ++k) d[(FC_AITN + k) * TE] = R(prm.geo[int64_t(G_AIT + k) * K + ne]);
                zp = sqrt(R(prm.geo[int64_t(G_MU) * K + ne]) / R(prm.geo[int64_t(G_EPS) * K + ne]));
                d[FC_BND * TE] = R(0);
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) d[(FC_AITN + k) * TE] = ait[k];
                d[FC_BND * TE] = R(1);
            }
            if (prm.upwind) {
                const R ym = R(1) / zm, yp = R(1) / zp;
                d[FC_CE * TE] = zp / (zm + zp);
                d[FC_BE * TE] = R(1) / (zm + zp);
                d[FC_CH * TE] = yp / (ym + yp);
                d[FC_BH * TE] = R(1) / (ym + yp);
            } else {
                d[FC_CE * TE] = R(0.5);
                d[FC_BE * TE] = R(0);
                d[FC_CH * TE] = R(0.5);
                d[FC_BH * TE] = R(0);
            }
        }
    }
    __syncthreads();

    // ---- phase 3: numerical flux per (face, face mode) ----------------------
    for (int it = grp; it < 4 * NF; it += NG) {
        const int f = it / NF;
        const int m = it % NF;
        const R* d = fg + f * FG * TE + c;
        R ait[9], aitn[9], n[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            ait[k] = eg[(G_AIT + k) * TE + c];
            aitn[k] = d[(FC_AITN + k) * TE];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) n[r] = d[(FC_N + r) * TE];
        const bool bnd = d[FC_BND * TE] != R(0);
        R* own = trO + (f * 6 * NF + m) * TE + c;
        const R* nbt = trN + (f * 6 * NF + m) * TE + c;
        R dE[3] = {0, 0, 0}, dH[3] = {0, 0, 0};
        // physical traces X = A^-T x_ref on each side
        if (DO_H || MODE == MODE_RHS || MODE == MODE_LSRK) {   // E traces needed by flux_H and upwind flux_E
            R em[3], ep[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                em[r] = R(0);
                ep[r] = R(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    em[r] += ait[3 * r + k] * own[k * NF * TE];
                    ep[r] += aitn[3 * r + k] * nbt[k * NF * TE];
                }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) dE[r] = bnd ? R(-2) * em[r] : ep[r] - em[r];
        }
        if (DO_E) {
            R hm[3], hp[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                hm[r] = R(0);
                hp[r] = R(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    hm[r] += ait[3 * r + k] * own[(3 + k) * NF * TE];
                    hp[r] += aitn[3 * r + k] * nbt[(3 + k) * NF * TE];
                }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) dH[r] = bnd ? R(0) : hp[r] - hm[r];
        }
        const R twoF = d[FC_TWOF * TE];
        R nxdE[3], nxdH[3], nnxdE[3], nnxdH[3];
        cross3(n, dE, nxdE);
        cross3(n, dH, nxdH);
        cross3(n, nxdE, nnxdE);
        cross3(n, nxdH, nnxdH);
        if (DO_E) {
            const R ce = d[FC_CE * TE], be = d[FC_BE * TE];
            R fl[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) fl[r] = ce * nxdH[r] - be * nnxdE[r];
            // g = 2|F| A^-1 flux, A^-1 = (A^-T)^T
#pragma unroll
            for (int j = 0; j < 3; ++j)
                own[j * NF * TE] = twoF * (ait[j] * fl[0] + ait[3 + j] * fl[1] + ait[6 + j] * fl[2]);
        }
        if (DO_H) {
            const R ch = d[FC_CH * TE], bh = d[FC_BH * TE];
            R fl[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) fl[r] = ch * nxdE[r] + bh * nnxdH[r];
#pragma unroll
            for (int j = 0; j < 3; ++j)
                own[(3 + j) * NF * TE] = -twoF * (ait[j] * fl[0] + ait[3 + j] * fl[1] + ait[6 + j] * fl[2]);
        }
    }
    __syncthreads();

    // ---- phase 4: volume curl + lift per component ---------------------------
    R* rh = trN;   // [6][N][TE], the neighbour traces are dead now
    for (int comp = grp; comp < 6; comp += NG) {
        if (!DO_E && comp < 3) continue;
        if (!DO_H && comp >= 3) continue;
        R acc[N];
#pragma unroll
        for (int l = 0; l < N; ++l) acc[l] = R(0);
        const R sgn = eg[G_DET * TE + c] < R(0) ? R(-1) : R(1);
        // curl_x = d_y v_z - d_z v_y, curl_y = d_z v_x - d_x v_z, curl_z = d_x v_y - d_y v_x,
        // applied to H for the E equation (+s) and to E for the H equation (-s)
        const int j = comp % 3;
        const int srcf = comp < 3 ? 3 : 0;
        const R sg = comp < 3 ? sgn : -sgn;
        const R* base = us + c;
        switch (j) {
            case 0:
                deriv_acc<P, R, 1>(base + (srcf + 2) * N * TE, TE, sg, acc);
                deriv_acc<P, R, 2>(base + (srcf + 1) * N * TE, TE, -sg, acc);
                break;
            case 1:
                deriv_acc<P, R, 2>(base + (srcf + 0) * N * TE, TE, sg, acc);
                deriv_acc<P, R, 0>(base + (srcf + 2) * N * TE, TE, -sg, acc);
                break;
            default:
                deriv_acc<P, R, 0>(base + (srcf + 1) * N * TE, TE, sg, acc);
                deriv_acc<P, R, 1>(base + (srcf + 0) * N * TE, TE, -sg, acc);
                break;
        }
        lift_face<P, R, 0>(trO + ((0 * 6 + comp) * NF) * TE + c, TE, acc);
        lift_face<P, R, 1>(trO + ((1 * 6 + comp) * NF) * TE + c, TE, acc);
        lift_face<P, R, 2>(trO + ((2 * 6 + comp) * NF) * TE + c, TE, acc);
        lift_face<P, R, 3>(trO + ((3 * 6 + comp) * NF) * TE + c, TE, acc);
        if (comp < 3 && prm.src != nullptr && active) {
            const double* rec = prm.src + int64_t(s) * (SRC_HDR + 3 * N);
            if (int64_t(rec[0]) == e) {
                const R g = R(source_time(prm.t, rec[1], rec[2], rec[3]));
#pragma unroll
                for (int l = 0; l < N; ++l) acc[l] -= g * R(rec[SRC_HDR + j * N + l]);
            }
        }
#pragma unroll
        for (int l = 0; l < N; ++l) rh[(comp * N + l) * TE + c] = acc[l];
    }
    __syncthreads();

    // ---- phase 5: mass-block inverse, PML, update ------------------------------
    for (int comp = grp; comp < 6; comp += NG) {
        if (!DO_E && comp < 3) continue;
        if (!DO_H && comp >= 3) continue;
        if (!active) continue;
        const int j = comp % 3;
        const int fb = comp < 3 ? 0 : 3;   // first component of this field
        R ait[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = eg[(G_AIT + k) * TE + c];
        const R det = eg[G_DET * TE + c];
        const R mat = comp < 3 ? eg[G_EPS * TE + c] : eg[G_MU * TE + c];
        // A^T = adj(A^-T) det A
        R AT[3][3];
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
            for (int b = 0; b < 3; ++b) AT[a][b] *= det;
        R brow[3];
        const R inv = R(1) / (mat * fabs(det));
#pragma unroll
        for (int k = 0; k < 3; ++k)
            brow[k] = inv * (AT[j][0] * AT[k][0] + AT[j][1] * AT[k][1] + AT[j][2] * AT[k][2]);
        // PML rows: (A^T D A^-T)[j][k] = sum_a A^T[j][a] D_a A^-T[a][k]
        int32_t pi = -1;
        if (prm.pml != nullptr) pi = prm.pml[e];
        R eta_row[3] = {0, 0, 0}, sig_row[3] = {0, 0, 0}, xi_row[3] = {0, 0, 0};
        if (pi >= 0) {
            const R sx = eg[(G_SIG + 0) * TE + c], sy = eg[(G_SIG + 1) * TE + c],
                    sz = eg[(G_SIG + 2) * TE + c];
            const R sg3[3] = {sx, sy, sz};
            const R et3[3] = {sy + sz - sx, sz + sx - sy, sx + sy - sz};
            const R xi3[3] = {(sx - sy) * (sx - sz), (sy - sz) * (sy - sx), (sz - sx) * (sz - sy)};
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const R w = AT[j][a] * ait[3 * a + k];
                    eta_row[k] += w * et3[a];
                    sig_row[k] += w * sg3[a];
                    xi_row[k] += w * xi3[a];
                }
        }
        const int64_t C2 = int64_t(prm.npml) * S;
        const int64_t acol = int64_t(pi) * S + s;
        R* uo = static_cast<R*>(prm.u_out);
        R* __restrict__ res = static_cast<R*>(prm.res);
        const R* __restrict__ aux = static_cast<const R*>(prm.aux);
        R* __restrict__ auxo = static_cast<R*>(prm.aux_out);
        R* __restrict__ auxr = static_cast<R*>(prm.aux_res);
        const R dt = R(prm.dt), ca = R(prm.a), cb = R(prm.b);
#pragma unroll 4
        for (int l = 0; l < N; ++l) {
            const R r0 = rh[((fb + 0) * N + l) * TE + c];
            const R r1 = rh[((fb + 1) * N + l) * TE + c];
            const R r2 = rh[((fb + 2) * N + l) * TE + c];
            R du = brow[0] * r0 + brow[1] * r1 + brow[2] * r2;
            const R uv = us[(comp * N + l) * TE + c];
            const int64_t gi = int64_t(comp * N + l) * C + col;
            if (pi >= 0) {
                const R u0 = us[((fb + 0) * N + l) * TE + c];
                const R u1 = us[((fb + 1) * N + l) * TE + c];
                const R u2 = us[((fb + 2) * N + l) * TE + c];
                const int64_t ai = int64_t(fb * N + l) * C2 + acol;
                const R a0 = aux[ai], a1 = aux[ai + int64_t(N) * C2], a2 = aux[ai + 2 * int64_t(N) * C2];
                const R av = j == 0 ? a0 : (j == 1 ? a1 : a2);
                du -= eta_row[0] * u0 + eta_row[1] * u1 + eta_row[2] * u2 + av / mat;
                const R da = -(sig_row[0] * a0 + sig_row[1] * a1 + sig_row[2] * a2) +
                             mat * (xi_row[0] * u0 + xi_row[1] * u1 + xi_row[2] * u2);
                const int64_t aj = int64_t(comp * N + l) * C2 + acol;
                if (MODE == MODE_RHS) {
                    auxo[aj] = da;
                } else if (MODE == MODE_LSRK) {
                    const R rr = (ca == R(0) ? R(0) : ca * auxr[aj]) + dt * da;
                    auxr[aj] = rr;
                    auxo[aj] = av + cb * rr;
                }
            }
            if (MODE == MODE_RHS) {
                uo[gi] = du;
            } else if (MODE == MODE_LSRK) {
                const R rr = (ca == R(0) ? R(0) : ca * res[gi]) + dt * du;
                res[gi] = rr;
                uo[gi] = uv + cb * rr;
            } else {
                uo[gi] = uv + dt * du;
            }
        }
    }
}

}  // namespace dgm
