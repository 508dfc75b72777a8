// Paired stage kernel (LSRK4 stages, FP32 fields): the algorithm of
// dgm_stage.cuh with every thread carrying two columns (col and col + 32) in
// a pair type PR (dgm_pair.cuh).  A CTA owns 64 columns.  Each literal
// coefficient of the generated reference operators, each shared-memory
// address and each branch now serves two elements, and with PR = F2x the
// arithmetic issues as packed FP32x2 instructions.  Phases and data layout
// (shared memory holds one PR per column pair) are those of stage_kernel.
#pragma once

#include <cstdint>

#include "dgm_pair.cuh"
#include "dgm_stage.cuh"

namespace dgm {

template <typename PR>
__device__ __forceinline__ void face_constants2(int f, const PR (&ait)[9], PR det, PR epsm, PR mum,
                                                bool hA, bool hB, const PR (&aitn)[9], PR zn,
                                                int upwind, PR* fc) {
    constexpr int TE = 32;
    const PR m0 = PR(f == 0 ? 1.0 : (f == 1 ? -1.0 : 0.0));
    const PR m1 = PR(f == 0 ? 1.0 : (f == 2 ? -1.0 : 0.0));
    const PR m2 = PR(f == 0 ? 1.0 : (f == 3 ? -1.0 : 0.0));
    PR vn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) vn[r] = ait[3 * r + 0] * m0 + ait[3 * r + 1] * m1 + ait[3 * r + 2] * m2;
    const PR fs = psqrt(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
    const PR ifs = prcp(fs);
#pragma unroll
    for (int r = 0; r < 3; ++r) fc[(FC_N + r) * TE] = vn[r] * ifs;
    fc[FC_TWOF * TE] = pabs(det) * fs;
    const PR zm = psqrt(mum * prcp(epsm));
#pragma unroll
    for (int k = 0; k < 9; ++k) fc[(FC_AITN + k) * TE] = aitn[k];
    const PR zp = psel(hA, hB, zn, zm);
    fc[FC_BND * TE] = PR(hA ? 0.f : 1.f, hB ? 0.f : 1.f);
    if (upwind) {
        const PR isum = prcp(zm + zp);
        fc[FC_CE * TE] = zp * isum;
        fc[FC_BE * TE] = isum;
        fc[FC_CH * TE] = zm * isum;          // Y+/(Y- + Y+) = Z-/(Z- + Z+)
        fc[FC_BH * TE] = zm * zp * isum;     // 1/(Y- + Y+)  = Z- Z+/(Z- + Z+)
    } else {
        fc[FC_CE * TE] = PR(0.5);
        fc[FC_BE * TE] = PR(0.0);
        fc[FC_CH * TE] = PR(0.5);
        fc[FC_BH * TE] = PR(0.0);
    }
}

template <typename PR>
__device__ __forceinline__ void cross3p(const PR a[3], const PR b[3], PR o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

template <int P, typename PR>
__host__ __device__ constexpr size_t stage2_smem_bytes() {
    return sizeof(PR) * size_t(32) * (6 * nmodes(P) + 48 * nfmodes(P) + 4 * FG + EG) +
           sizeof(int2) * 4 * 32;
}

template <int P, typename PR, int NT, typename IX = int64_t>
__global__ void __launch_bounds__(NT, 1) stage2_kernel(const StageParams prm) {
    constexpr int TE = 32;
    constexpr int N = nmodes(P);
    constexpr int NF = nfmodes(P);
    constexpr int NG = NT / TE;
    constexpr int NPART = NG >= 24 ? 4 : (NG >= 12 ? 2 : 1);
    static_assert(NG > 4, "groups 0..3 compute the face constants");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PR* us = reinterpret_cast<PR*>(smem_raw);     // [6N][32]
    PR* trO = us + 6 * N * TE;                    // [4][6][NF][32]
    PR* trN = trO + 24 * NF * TE;                 // [4][6][NF][32]
    PR* fg = trN + 24 * NF * TE;                  // [4][FG][32]
    PR* eg = fg + 4 * FG * TE;                    // [EG][32]
    int2* nbs = reinterpret_cast<int2*>(eg + EG * TE);   // [4][32]

    const int c = threadIdx.x % TE;
    const int grp = threadIdx.x / TE;
    const IX K = prm.K;
    const int S = prm.S;
    const IX C = K * S;
    const IX colA = IX(tile_index(prm.tile_groups)) * 64 + c, colB = colA + 32;
    const IX Cact = IX(prm.K_active) * IX(S);     // columns updated (the rest: halo copies)
    const bool actA = colA < Cact, actB = colB < Cact;
    const IX eA = actA ? colA / S : 0, eB = actB ? colB / S : 0;
    const int sA = actA ? int(colA - eA * S) : 0, sB = actB ? int(colB - eB * S) : 0;
    const float* u = static_cast<const float*>(prm.u);
    const float* gr = static_cast<const float*>(prm.geo_r);
    if (grp < 4)
        nbs[grp * TE + c] = make_int2(actA ? prm.nbr[IX(grp) * K + eA] : -1,
                                      actB ? prm.nbr[IX(grp) * K + eB] : -1);

    // ---- phase 1 -------------------------------------------------------------------
    auto geo2 = [&](int k, float dflt) {
        return PR(actA ? gr[IX(k) * K + eA] : dflt, actB ? gr[IX(k) * K + eB] : dflt);
    };
    constexpr int FACE_GROUPS = NG > 4 ? 4 : 0;
    if (grp < FACE_GROUPS) {
        const int f = grp;
        const float* fn = static_cast<const float*>(prm.fnb_r) + IX(f * FNB_COUNT) * K;
        const int32_t ca = actA ? prm.nbr[IX(f) * K + eA] : -1;
        const int32_t cb = actB ? prm.nbr[IX(f) * K + eB] : -1;
        PR ait[9], aitn[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = geo2(G_AIT + k, k % 4 == 0 ? 1.f : 0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            aitn[k] = PR(actA ? fn[IX(FNB_AIT + k) * K + eA] : ait[k].a(),
                         actB ? fn[IX(FNB_AIT + k) * K + eB] : ait[k].b());
        const PR zn(actA ? fn[IX(FNB_Z) * K + eA] : 1.f, actB ? fn[IX(FNB_Z) * K + eB] : 1.f);
        face_constants2<PR>(f, ait, geo2(G_DET, 1.f), geo2(G_EPS, 1.f), geo2(G_MU, 1.f),
                            ca >= 0 && (ca >> 2) < K, cb >= 0 && (cb >> 2) < K, aitn, zn, prm.upwind,
                            fg + f * FG * TE + c);
    }
    if (grp >= FACE_GROUPS) {
        // all loads of a thread in flight before its first shared-memory store
        constexpr int LG = NG - FACE_GROUPS;
        constexpr int UR = (6 * N + LG - 1) / LG;
        constexpr int ER = (EG + LG - 1) / LG;
        const int lg = grp - FACE_GROUPS;
        constexpr int BATCH = 8;
#pragma unroll
        for (int i0 = 0; i0 < UR; i0 += BATCH) {
            PR tmp[BATCH];
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int r = lg + (i0 + i) * LG;
                const bool ok = i0 + i < UR && r < 6 * N;
                tmp[i] = PR(ok && actA ? u[IX(r) * C + colA] : 0.f, ok && actB ? u[IX(r) * C + colB] : 0.f);
            }
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int r = lg + (i0 + i) * LG;
                if (i0 + i < UR && r < 6 * N) us[r * TE + c] = tmp[i];
            }
        }
#pragma unroll
        for (int i = 0; i < ER; ++i) {
            const int k = lg + i * LG;
            if (k < EG) eg[k * TE + c] = geo2(k, (k == G_DET || k == G_EPS || k == G_MU) ? 1.f : 0.f);
        }
    }
    __syncthreads();

    // ---- phase 2: traces -------------------------------------------------------------
    {
        constexpr int NOWN = 12, NNBR = 24;
        constexpr int ROUNDS = (NNBR + NG - 1) / NG;
#pragma unroll 1
        for (int rr = 0; rr < ROUNDS; ++rr) {
            const int ni = grp + rr * NG;
            const bool do_nbr = ni < NNBR;
            const int nf = ni / 6, ncomp = ni % 6;
            int2 code = make_int2(-1, -1);
            if (do_nbr) code = nbs[nf * TE + c];
            const bool hA = do_nbr && code.x >= 0 && (code.x >> 2) < K;
            const bool hB = do_nbr && code.y >= 0 && (code.y >> 2) < K;
            if (do_nbr && ((code.x >= 0 && (code.x >> 2) >= K) || (code.y >= 0 && (code.y >> 2) >= K)))
                atomicOr(prm.status, ST_BAD_NEIGHBOUR);
            PR vn[N];
            if (hA || hB) {
                const IX na = hA ? (IX(code.x >> 2) * S + sA) : 0;
                const IX nb = hB ? (IX(code.y >> 2) * S + sB) : 0;
#pragma unroll
                for (int l = 0; l < N; ++l)
                    vn[l] = PR(hA ? u[IX(ncomp * N + l) * C + na] : 0.f,
                               hB ? u[IX(ncomp * N + l) * C + nb] : 0.f);
            }
            if (ni < NOWN) {
                const int ocomp = ni % 6, fp = ni / 6;
                PR v[N];
                PR acc[NF];
#pragma unroll
                for (int l = 0; l < N; ++l) v[l] = us[(ocomp * N + l) * TE + c];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int f = 2 * fp + h;
                    trace_any<P, PR>(f, v, acc);
                    PR* dst = trO + ((f * 6 + ocomp) * NF) * TE + c;
#pragma unroll
                    for (int m = 0; m < NF; ++m) dst[m * TE] = acc[m];
                }
            }
            if (do_nbr) {
                PR acc[NF];
                const int fa = code.x & 3, fb = code.y & 3;
                if (hA && hB && fa == fb) {
                    trace_any<P, PR>(fa, vn, acc);
                } else {
                    PR t1[NF], t2[NF];
                    if (hA) trace_any<P, PR>(fa, vn, t1);
                    if (hB) trace_any<P, PR>(fb, vn, t2);
#pragma unroll
                    for (int m = 0; m < NF; ++m) acc[m] = PR(hA ? t1[m].a() : 0.f, hB ? t2[m].b() : 0.f);
                }
                PR* dst = trN + ((nf * 6 + ncomp) * NF) * TE + c;
#pragma unroll
                for (int m = 0; m < NF; ++m) dst[m * TE] = acc[m];
            }
        }
    }
    __syncthreads();

    // ---- phase 3: flux ---------------------------------------------------------------
    {
        constexpr int CHUNKS = NG >= 12 ? (NG / 4) : 1;
        for (int it = grp; it < 4 * CHUNKS; it += NG) {
            const int f = it / CHUNKS;
            const int ch = it % CHUNKS;
            const PR* d = fg + f * FG * TE + c;
            PR ait[9], aitn[9], n[3];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                ait[k] = eg[(G_AIT + k) * TE + c];
                aitn[k] = d[(FC_AITN + k) * TE];
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) n[r] = d[(FC_N + r) * TE];
            const PR bndv = d[FC_BND * TE];
            const bool bA = bndv.a() != 0.f, bB = bndv.b() != 0.f;
            const PR twoF = d[FC_TWOF * TE];
            const PR ce = d[FC_CE * TE], be = d[FC_BE * TE], chc = d[FC_CH * TE], bh = d[FC_BH * TE];
            const PR mtwo = PR(-2.0), zero = PR(0.0);
            for (int m = ch * NF / CHUNKS; m < (ch + 1) * NF / CHUNKS; ++m) {
                PR* own = trO + (f * 6 * NF + m) * TE + c;
                const PR* nbt = trN + (f * 6 * NF + m) * TE + c;
                PR dE[3], dH[3];
                {
                    PR tm[3], tp[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        tm[k] = own[k * NF * TE];
                        tp[k] = nbt[k * NF * TE];
                    }
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const PR em = ait[3 * r] * tm[0] + ait[3 * r + 1] * tm[1] + ait[3 * r + 2] * tm[2];
                        const PR ep = aitn[3 * r] * tp[0] + aitn[3 * r + 1] * tp[1] + aitn[3 * r + 2] * tp[2];
                        dE[r] = psel(bA, bB, mtwo * em, ep - em);
                    }
                }
                {
                    PR tm[3], tp[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        tm[k] = own[(3 + k) * NF * TE];
                        tp[k] = nbt[(3 + k) * NF * TE];
                    }
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const PR hm = ait[3 * r] * tm[0] + ait[3 * r + 1] * tm[1] + ait[3 * r + 2] * tm[2];
                        const PR hp = aitn[3 * r] * tp[0] + aitn[3 * r + 1] * tp[1] + aitn[3 * r + 2] * tp[2];
                        dH[r] = psel(bA, bB, zero, hp - hm);
                    }
                }
                PR nxdE[3], nxdH[3], nnxdE[3], nnxdH[3];
                cross3p(n, dE, nxdE);
                cross3p(n, dH, nxdH);
                cross3p(n, nxdE, nnxdE);
                cross3p(n, nxdH, nnxdH);
                PR fe[3], fh[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    fe[r] = ce * nxdH[r] - be * nnxdE[r];
                    fh[r] = chc * nxdE[r] + bh * nnxdH[r];
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    own[j * NF * TE] = twoF * (ait[j] * fe[0] + ait[3 + j] * fe[1] + ait[6 + j] * fe[2]);
                    own[(3 + j) * NF * TE] = -(twoF * (ait[j] * fh[0] + ait[3 + j] * fh[1] + ait[6 + j] * fh[2]));
                }
            }
        }
    }
    __syncthreads();

    // ---- phase 4: curl + lift ------------------------------------------------------
    PR* rh = trN;
    constexpr int RPF = (N + NPART - 1) / NPART;
    constexpr bool PREFETCH_RES = 6 * NPART <= NG;
    PR resv[PREFETCH_RES ? RPF : 1];
    const float* resg = static_cast<const float*>(prm.res);
    if (PREFETCH_RES && grp < 6 * NPART && prm.a_f != 0.f) {
        const int comp = grp / NPART, part = grp % NPART;
        const int lo = part * N / NPART, hi = (part + 1) * N / NPART;
#pragma unroll
        for (int i = 0; i < RPF; ++i)
            if (lo + i < hi)
                resv[i] = PR(actA ? resg[IX(comp * N + lo + i) * C + colA] : 0.f,
                             actB ? resg[IX(comp * N + lo + i) * C + colB] : 0.f);
    }
    for (int it = grp; it < 6 * NPART; it += NG) {
        const int comp = it / NPART;
        const int part = it % NPART;
        const PR dt_ = eg[G_DET * TE + c];
        const PR sgn = PR(dt_.a() < 0.f ? -1.f : 1.f, dt_.b() < 0.f ? -1.f : 1.f);
        PR acc[N];
        rhs_part<P, PR, TE, NPART>(part, comp, c, us, trO, sgn, acc);
        const int lo = part * N / NPART, hi = (part + 1) * N / NPART;
        if (comp < 3 && prm.src != nullptr) {
            const double* ra = prm.src + IX(sA) * (SRC_HDR + 3 * N);
            const double* rb = prm.src + IX(sB) * (SRC_HDR + 3 * N);
            const bool hitA = actA && ra[0] >= 0.0 && IX(ra[0]) == eA, hitB = actB && rb[0] >= 0.0 && IX(rb[0]) == eB;
            if (hitA || hitB) {
                const double tt = prm.tdev ? *prm.tdev + prm.t : prm.t;
                const float ga = hitA ? float(source_time(tt, ra[1], ra[2], ra[3])) : 0.f;
                const float gb = hitB ? float(source_time(tt, rb[1], rb[2], rb[3])) : 0.f;
#pragma unroll
                for (int l = 0; l < N; ++l)
                    if (l >= lo && l < hi)
                        acc[l] -= PR(hitA ? ga * float(ra[SRC_HDR + (comp % 3) * N + l]) : 0.f,
                                     hitB ? gb * float(rb[SRC_HDR + (comp % 3) * N + l]) : 0.f);
            }
        }
#pragma unroll
        for (int l = 0; l < N; ++l)
            if (l >= lo && l < hi) rh[(comp * N + l) * TE + c] = acc[l];
    }
    __syncthreads();

    // ---- phase 5: mass inverse, PML, LSRK update --------------------------------------
    for (int it = grp; it < 6 * NPART; it += NG) {
        const int comp = it / NPART;
        const int part = it % NPART;
        const int j = comp % 3;
        const int fb = comp < 3 ? 0 : 3;
        PR ait[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) ait[k] = eg[(G_AIT + k) * TE + c];
        const PR det = eg[G_DET * TE + c];
        const PR mat = comp < 3 ? eg[G_EPS * TE + c] : eg[G_MU * TE + c];
        PR AT[3][3];
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
            for (int b = 0; b < 3; ++b) AT[a][b] = AT[a][b] * det;
        PR atj[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) atj[b] = j == 0 ? AT[0][b] : (j == 1 ? AT[1][b] : AT[2][b]);
        const PR inv = prcp(mat * pabs(det));
        PR brow[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) brow[k] = inv * (atj[0] * AT[k][0] + atj[1] * AT[k][1] + atj[2] * AT[k][2]);
        const int32_t piA = (prm.pml != nullptr && actA) ? prm.pml[eA] : -1;
        const int32_t piB = (prm.pml != nullptr && actB) ? prm.pml[eB] : -1;
        const bool any_pml = piA >= 0 || piB >= 0;
        PR eta_row[3] = {PR(0.0), PR(0.0), PR(0.0)}, sig_row[3] = {PR(0.0), PR(0.0), PR(0.0)},
           xi_row[3] = {PR(0.0), PR(0.0), PR(0.0)};
        if (any_pml) {
            const PR sx = eg[(G_SIG + 0) * TE + c], sy = eg[(G_SIG + 1) * TE + c], sz = eg[(G_SIG + 2) * TE + c];
            const PR sg3[3] = {sx, sy, sz};
            const PR et3[3] = {sy + sz - sx, sz + sx - sy, sx + sy - sz};
            const PR xi3[3] = {(sx - sy) * (sx - sz), (sy - sz) * (sy - sx), (sz - sx) * (sz - sy)};
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const PR w = atj[a] * ait[3 * a + k];
                    eta_row[k] += w * et3[a];
                    sig_row[k] += w * sg3[a];
                    xi_row[k] += w * xi3[a];
                }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                eta_row[k] = psel(piA >= 0, piB >= 0, eta_row[k], PR(0.0));
                sig_row[k] = psel(piA >= 0, piB >= 0, sig_row[k], PR(0.0));
                xi_row[k] = psel(piA >= 0, piB >= 0, xi_row[k], PR(0.0));
            }
        }
        const IX C2 = IX(prm.npml) * S;
        const IX acA = IX(piA) * S + sA, acB = IX(piB) * S + sB;
        float* uo = static_cast<float*>(prm.u_out);
        float* res = static_cast<float*>(prm.res);
        const float* aux = static_cast<const float*>(prm.aux);
        float* auxo = static_cast<float*>(prm.aux_out);
        float* auxr = static_cast<float*>(prm.aux_res);
        const PR dt = PR(prm.dt_f, prm.dt_f), cb = PR(prm.b_f, prm.b_f);
        const float ca = prm.a_f;
        const int lo = part * N / NPART, hi = (part + 1) * N / NPART;
#pragma unroll
        for (int i = 0; i < RPF; ++i) {
            const int l = lo + i;
            if (l >= hi) break;
            const PR r0 = rh[((fb + 0) * N + l) * TE + c];
            const PR r1 = rh[((fb + 1) * N + l) * TE + c];
            const PR r2 = rh[((fb + 2) * N + l) * TE + c];
            PR du = brow[0] * r0 + brow[1] * r1 + brow[2] * r2;
            const PR uv = us[(comp * N + l) * TE + c];
            const IX row = IX(comp * N + l) * C;
            if (any_pml) {
                const PR u0 = us[((fb + 0) * N + l) * TE + c];
                const PR u1 = us[((fb + 1) * N + l) * TE + c];
                const PR u2 = us[((fb + 2) * N + l) * TE + c];
                auto ld = [&](int cc) {
                    const IX rw = IX(cc * N + l) * C2;
                    return PR(piA >= 0 ? aux[rw + acA] : 0.f, piB >= 0 ? aux[rw + acB] : 0.f);
                };
                const PR a0 = ld(fb), a1 = ld(fb + 1), a2 = ld(fb + 2);
                const PR av = j == 0 ? a0 : (j == 1 ? a1 : a2);
                du = du - (eta_row[0] * u0 + eta_row[1] * u1 + eta_row[2] * u2 + av * prcp(mat));
                const PR da = mat * (xi_row[0] * u0 + xi_row[1] * u1 + xi_row[2] * u2) -
                              (sig_row[0] * a0 + sig_row[1] * a1 + sig_row[2] * a2);
                const IX rw = IX(comp * N + l) * C2;
                if (piA >= 0) {
                    const float rr = (ca == 0.f ? 0.f : ca * auxr[rw + acA]) + prm.dt_f * da.a();
                    auxr[rw + acA] = rr;
                    auxo[rw + acA] = av.a() + prm.b_f * rr;
                }
                if (piB >= 0) {
                    const float rr = (ca == 0.f ? 0.f : ca * auxr[rw + acB]) + prm.dt_f * da.b();
                    auxr[rw + acB] = rr;
                    auxo[rw + acB] = av.b() + prm.b_f * rr;
                }
            }
            PR rold = PR(0.0);
            if (ca != 0.f)
                rold = PREFETCH_RES ? resv[PREFETCH_RES ? i : 0]
                                    : PR(actA ? res[row + colA] : 0.f, actB ? res[row + colB] : 0.f);
            const PR rr = PR(ca) * rold + dt * du;
            const PR un = uv + cb * rr;
            if (actA) {
                res[row + colA] = rr.a();
                uo[row + colA] = un.a();
            }
            if (actB) {
                res[row + colB] = rr.b();
                uo[row + colB] = un.b();
            }
        }
    }
}

}  // namespace dgm
