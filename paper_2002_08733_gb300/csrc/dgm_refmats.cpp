// Reference-element operators of the matrix-free method (host, FP64).
//
// Basis (Sec. II, Eq. (dubiner_functions) with the standard collapsed
// exponents): phi_ijk = nu_ijk * Q_i^(0)(z, 1-x-y) * Q_j^(2i+1)(y, 1-x)
// * Q_k^(2i+2j+2)(x, 1), where Q_n^(a)(y, w) = w^n P_n^(a,0)(2y/w - 1) is the
// "scaled" Jacobi polynomial, a polynomial in (y, w) evaluated by a
// division-free recurrence, and nu_ijk = sqrt(2 (2i+1)(i+j+1)(2n+3)),
// n = i+j+k, is the closed-form L2 normalisation that makes the set
// orthonormal on the reference tetrahedron (Eq. (ortho_cond)).  Gradients are
// carried alongside in forward mode (dual numbers).
//
// Face basis: psi_ij(s, t) = sqrt(2 (2i+1)(i+j+1)) Q_i^(0)(t, 1-s) Q_j^(2i+1)(s, 1),
// orthonormal on the reference triangle {s, t >= 0, s + t <= 1}.  Face f of
// the reference tetrahedron is the face opposite local vertex f, parametrised
// as V_a + s (V_b - V_a) + t (V_c - V_a) with a < b < c its other vertices.
// Because every element orders its vertices by ascending global id, the two
// elements sharing a face parametrise it identically, so face-mode
// coefficients of both sides are directly comparable.
//
// Geometry-free operators (Sec. III, Eq. (matrix_free_curl)):
//   S[a][l][m] = int_T phi_l d_a phi_m           (volume derivative, a = x,y,z)
//   R[f][m][l] = int_{T2} psi_m phi_l(x_f(s, t))  (trace onto face f; its
//                transpose is the lift back from the face)
// integrated with collapsed Gauss-Legendre rules that are exact for the
// polynomial degrees involved.  The basis orthonormality is re-checked here.
#include <cmath>
#include <string>
#include <vector>

#include "dgm_internal.h"

namespace dgm {

namespace {

struct Dual {
    double v, g[3];
};

inline Dual dconst(double c) { return Dual{c, {0, 0, 0}}; }
inline Dual dvar(double c, int i) {
    Dual d{c, {0, 0, 0}};
    d.g[i] = 1.0;
    return d;
}
inline Dual operator+(Dual a, Dual b) {
    return Dual{a.v + b.v, {a.g[0] + b.g[0], a.g[1] + b.g[1], a.g[2] + b.g[2]}};
}
inline Dual operator-(Dual a, Dual b) {
    return Dual{a.v - b.v, {a.g[0] - b.g[0], a.g[1] - b.g[1], a.g[2] - b.g[2]}};
}
inline Dual operator*(Dual a, Dual b) {
    return Dual{a.v * b.v,
                {a.g[0] * b.v + a.v * b.g[0], a.g[1] * b.v + a.v * b.g[1],
                 a.g[2] * b.v + a.v * b.g[2]}};
}
inline Dual operator*(double c, Dual a) { return Dual{c * a.v, {c * a.g[0], c * a.g[1], c * a.g[2]}}; }

// Q_0..Q_nmax of the scaled Jacobi family with parameter alpha (beta = 0):
// Q_0 = 1, Q_1 = (alpha+2) y - w, and for n >= 2
// 2n(n+a)(2n+a-2) Q_n = (2n+a-1)[(2n+a)(2n+a-2)(2y-w) + a^2 w] Q_{n-1}
//                       - 2(n+a-1)(n-1)(2n+a) w^2 Q_{n-2}.
void scaled_jacobi(int nmax, double alpha, Dual y, Dual w, Dual* Q) {
    Q[0] = dconst(1.0);
    if (nmax < 1) return;
    Q[1] = (alpha + 2.0) * y - w;
    Dual w2 = w * w;
    Dual ym = 2.0 * y - w;
    for (int n = 2; n <= nmax; ++n) {
        double a = alpha;
        double c0 = 2.0 * n * (n + a) * (2.0 * n + a - 2.0);
        double c1 = (2.0 * n + a - 1.0) * (2.0 * n + a) * (2.0 * n + a - 2.0);
        double c2 = (2.0 * n + a - 1.0) * a * a;
        double c3 = 2.0 * (n + a - 1.0) * (n - 1.0) * (2.0 * n + a);
        Q[n] = (1.0 / c0) * ((c1 * ym + c2 * w) * Q[n - 1] - c3 * (w2 * Q[n - 2]));
    }
}

// All N basis functions (with gradients) at one reference point.
void basis_dual(int p, const double xr[3], Dual* out) {
    Dual x = dvar(xr[0], 0), y = dvar(xr[1], 1), z = dvar(xr[2], 2);
    Dual one = dconst(1.0);
    Dual Qi[PMAX + 1], Qj[PMAX + 1], Qk[PMAX + 1];
    scaled_jacobi(p, 0.0, z, one - x - y, Qi);
    int l = 0;
    for (int n = 0; n <= p; ++n)
        for (int i = 0; i <= n; ++i) {
            scaled_jacobi(n - i, 2.0 * i + 1.0, y, one - x, Qj);
            for (int j = 0; j <= n - i; ++j) {
                int k = n - i - j;
                scaled_jacobi(k, 2.0 * i + 2.0 * j + 2.0, x, one, Qk);
                double nu = std::sqrt(2.0 * (2 * i + 1) * (i + j + 1) * (2 * n + 3));
                out[l++] = nu * (Qi[i] * (Qj[j] * Qk[k]));
            }
        }
}

void face_basis(int p, double s, double t, double* out) {
    Dual Qi[PMAX + 1], Qj[PMAX + 1];
    Dual one = dconst(1.0);
    scaled_jacobi(p, 0.0, dconst(t), one - dconst(s), Qi);
    int m = 0;
    for (int n = 0; n <= p; ++n)
        for (int i = 0; i <= n; ++i) {
            int j = n - i;
            scaled_jacobi(j, 2.0 * i + 1.0, dconst(s), one, Qj);
            out[m++] = std::sqrt(2.0 * (2 * i + 1) * (i + j + 1)) * (Qi[i] * Qj[j]).v;
        }
}

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int n = 2; n <= q; ++n) {
                double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1.0; }
            double dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int n = 2; n <= q; ++n) {
            double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        if (q == 1) { p1 = z; p0 = 1.0; }
        double dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void tri_rule(int q, std::vector<double>& pts, std::vector<double>& w) {
    std::vector<double> g, wg;
    gauss_legendre(q, g, wg);
    pts.clear();
    w.clear();
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            double s = 0.5 * (1.0 + g[b]);
            double t = 0.5 * (1.0 + g[a]) * (1.0 - s);
            pts.push_back(s);
            pts.push_back(t);
            w.push_back(wg[a] * wg[b] * (1.0 - s) * 0.25);
        }
}

const double REF_V[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

}  // namespace

void tet_rule(int q, std::vector<double>& pts, std::vector<double>& w) {
    std::vector<double> g, wg;
    gauss_legendre(q, g, wg);
    pts.clear();
    w.clear();
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b)
            for (int c = 0; c < q; ++c) {
                double x = 0.5 * (1.0 + g[c]);
                double y = 0.5 * (1.0 + g[b]) * (1.0 - x);
                double z = 0.5 * (1.0 + g[a]) * (1.0 - x - y);
                pts.push_back(x);
                pts.push_back(y);
                pts.push_back(z);
                w.push_back(wg[a] * wg[b] * wg[c] * (1.0 - x) * (1.0 - x - y) / 8.0);
            }
}

void face_rule(int p, int q, std::vector<double>& pts, std::vector<double>& w,
               std::vector<double>& psi) {
    tri_rule(q, pts, w);
    const int NF = nfmodes(p);
    psi.assign(w.size() * NF, 0.0);
    for (size_t i = 0; i < w.size(); ++i) face_basis(p, pts[2 * i], pts[2 * i + 1], &psi[i * NF]);
}

void ref_basis_values(int p, const double xr[3], double* out) {
    Dual d[nmodes(PMAX)];
    basis_dual(p, xr, d);
    for (int l = 0; l < nmodes(p); ++l) out[l] = d[l].v;
}

int build_refmats(int p, std::vector<double>& S, std::vector<double>& R, std::string& err) {
    if (p < 0 || p > PMAX) {
        err = "unsupported polynomial degree";
        return 1;
    }
    const int N = nmodes(p), NF = nfmodes(p);
    std::vector<double> pts, w;
    tet_rule(p + 3, pts, w);
    const size_t nq = w.size();
    S.assign(3 * N * N, 0.0);
    std::vector<double> gram(N * N, 0.0);
    std::vector<Dual> phi(N);
    for (size_t q = 0; q < nq; ++q) {
        basis_dual(p, &pts[3 * q], phi.data());
        for (int l = 0; l < N; ++l)
            for (int m = 0; m < N; ++m) {
                gram[l * N + m] += w[q] * phi[l].v * phi[m].v;
                for (int a = 0; a < 3; ++a) S[(a * N + l) * N + m] += w[q] * phi[l].v * phi[m].g[a];
            }
    }
    double worst = 0.0;
    for (int l = 0; l < N; ++l)
        for (int m = 0; m < N; ++m)
            worst = std::fmax(worst, std::fabs(gram[l * N + m] - (l == m ? 1.0 : 0.0)));
    if (worst > 1e-12) {
        err = "reference basis failed its orthonormality check";
        return 1;
    }
    std::vector<double> fp, fw;
    tri_rule(p + 2, fp, fw);
    R.assign(4 * NF * N, 0.0);
    std::vector<double> psi(NF), fgram(NF * NF, 0.0), val(N);
    for (int f = 0; f < 4; ++f) {
        int vv[3], c = 0;
        for (int v = 0; v < 4; ++v)
            if (v != f) vv[c++] = v;
        for (size_t q = 0; q < fw.size(); ++q) {
            double s = fp[2 * q], t = fp[2 * q + 1];
            double xr[3];
            for (int i = 0; i < 3; ++i)
                xr[i] = REF_V[vv[0]][i] + s * (REF_V[vv[1]][i] - REF_V[vv[0]][i]) +
                        t * (REF_V[vv[2]][i] - REF_V[vv[0]][i]);
            face_basis(p, s, t, psi.data());
            ref_basis_values(p, xr, val.data());
            for (int m = 0; m < NF; ++m) {
                for (int l = 0; l < N; ++l) R[(f * NF + m) * N + l] += fw[q] * psi[m] * val[l];
                if (f == 0)
                    for (int m2 = 0; m2 < NF; ++m2) fgram[m * NF + m2] += fw[q] * psi[m] * psi[m2];
            }
        }
    }
    for (int m = 0; m < NF; ++m)
        for (int m2 = 0; m2 < NF; ++m2)
            worst = std::fmax(worst, std::fabs(fgram[m * NF + m2] - (m == m2 ? 1.0 : 0.0)));
    if (worst > 1e-12) {
        err = "face basis failed its orthonormality check";
        return 1;
    }
    return 0;
}

}  // namespace dgm
