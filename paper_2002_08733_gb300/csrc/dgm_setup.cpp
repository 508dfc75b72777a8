// Host-side mesh setup (FP64): element maps, face-neighbour table, PML profile.
//
// Element map (Eq. (mapping_template)): r = A r_hat + b with the columns of A
// the edges v1-v0, v2-v0, v3-v0 of the element's vertices sorted by global
// id.  Stored per element: A^-T (the covariant map of Eq. (cov_transf)),
// the signed det A (its sign orients the Piola-mapped curl, Eq.
// (piola_transf)), eps, mu and the PML damping triple.
//
// Face f of an element is the face opposite its local vertex f.  Faces are
// matched by their sorted vertex-id triples; the neighbour table stores
// (neighbour << 2) | (neighbour's local index of the shared face), or -1 for
// a boundary face (PEC wall).
//
// PML (Sec. IV): sigma_a = sigma_max (d_a / L)^order at the element centroid,
// d_a the depth into the layer outside the box [lo, hi] along axis a, so the
// damping is constant per element as Sec. V motivates.
#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "dgm_internal.h"
#include "dgmax.h"

namespace dgm {

int build_mesh(int64_t nv, const double* xyz, int64_t nt, const int64_t* tets, const double* eps,
               const double* mu, const double* pml_lo, const double* pml_hi, double pml_L,
               double pml_smax, int pml_order, bool has_pml, HostMesh& out, std::string& err) {
    if (nv < 4 || nt < 1 || !xyz || !tets || !eps || !mu) {
        err = "empty mesh or null input";
        return DGM_EINVAL;
    }
    if (nt >= (int64_t(1) << 29)) {
        err = "too many elements for the 29-bit neighbour encoding";
        return DGM_EUNSUP;
    }
    const int64_t K = nt;
    out.K = K;
    out.geo.assign(size_t(G_COUNT) * K, 0.0);
    out.nbr.assign(size_t(4) * K, -1);
    out.pml_idx.assign(size_t(K), -1);
    out.verts.assign(size_t(12) * K, 0.0);
    out.vid.assign(size_t(4) * K, 0);
    std::vector<std::array<int64_t, 4>> sv(K);
    for (int64_t e = 0; e < K; ++e) {
        std::array<int64_t, 4> v;
        for (int i = 0; i < 4; ++i) {
            v[i] = tets[4 * e + i];
            if (v[i] < 0 || v[i] >= nv) {
                err = "vertex id out of range in element " + std::to_string(e);
                return DGM_EMESH;
            }
        }
        std::sort(v.begin(), v.end());
        for (int i = 0; i < 3; ++i)
            if (v[i] == v[i + 1]) {
                err = "repeated vertex in element " + std::to_string(e);
                return DGM_EMESH;
            }
        sv[e] = v;
        for (int i = 0; i < 4; ++i) out.vid[4 * e + i] = v[i];
        if (!(eps[e] > 0.0) || !(mu[e] > 0.0) || !std::isfinite(eps[e]) || !std::isfinite(mu[e])) {
            err = "eps and mu must be positive and finite (element " + std::to_string(e) + ")";
            return DGM_EINVAL;
        }
        double P[4][3];
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) {
                P[i][c] = xyz[3 * v[i] + c];
                out.verts[12 * e + 3 * i + c] = P[i][c];
            }
        double A[3][3];  // columns are edges
        double hmax = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                A[r][c] = P[c + 1][r] - P[0][r];
                hmax = std::fmax(hmax, std::fabs(A[r][c]));
            }
        double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        if (!std::isfinite(det) || std::fabs(det) <= 1e-13 * hmax * hmax * hmax) {
            err = "degenerate element " + std::to_string(e);
            return DGM_EMESH;
        }
        // A^-1 = adj(A) / det; A^-T[r][c] = A^-1[c][r]
        double adj[3][3] = {
            {A[1][1] * A[2][2] - A[1][2] * A[2][1], A[0][2] * A[2][1] - A[0][1] * A[2][2],
             A[0][1] * A[1][2] - A[0][2] * A[1][1]},
            {A[1][2] * A[2][0] - A[1][0] * A[2][2], A[0][0] * A[2][2] - A[0][2] * A[2][0],
             A[0][2] * A[1][0] - A[0][0] * A[1][2]},
            {A[1][0] * A[2][1] - A[1][1] * A[2][0], A[0][1] * A[2][0] - A[0][0] * A[2][1],
             A[0][0] * A[1][1] - A[0][1] * A[1][0]}};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) out.geo[(G_AIT + 3 * r + c) * K + e] = adj[c][r] / det;
        out.geo[G_DET * K + e] = det;
        out.geo[G_EPS * K + e] = eps[e];
        out.geo[G_MU * K + e] = mu[e];
        if (has_pml) {
            bool any = false;
            for (int a = 0; a < 3; ++a) {
                double c = 0.25 * (P[0][a] + P[1][a] + P[2][a] + P[3][a]);
                double d = std::fmax(0.0, std::fmax(pml_lo[a] - c, c - pml_hi[a]));
                double s = pml_smax * std::pow(d / pml_L, double(pml_order));
                out.geo[(G_SIG + a) * K + e] = s;
                any = any || s > 0.0;
            }
            if (any) out.pml_idx[e] = int32_t(out.npml++);
        }
    }
    // face matching by sorted vertex triples
    struct FaceKey {
        int64_t a, b, c;
        int64_t id;  // 4 * element + local face
    };
    std::vector<FaceKey> faces(size_t(4) * K);
    for (int64_t e = 0; e < K; ++e)
        for (int f = 0; f < 4; ++f) {
            int64_t t[3];
            int c = 0;
            for (int i = 0; i < 4; ++i)
                if (i != f) t[c++] = sv[e][i];
            faces[4 * e + f] = FaceKey{t[0], t[1], t[2], 4 * e + f};
        }
    std::sort(faces.begin(), faces.end(), [](const FaceKey& x, const FaceKey& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        if (x.c != y.c) return x.c < y.c;
        return x.id < y.id;
    });
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j].a == faces[i].a && faces[j].b == faces[i].b &&
               faces[j].c == faces[i].c)
            ++j;
        if (j - i > 2) {
            err = "non-manifold face shared by more than two elements";
            return DGM_EMESH;
        }
        if (j - i == 2) {
            int64_t e1 = faces[i].id / 4, f1 = faces[i].id % 4;
            int64_t e2 = faces[i + 1].id / 4, f2 = faces[i + 1].id % 4;
            if (e1 == e2) {
                err = "element shares a face with itself";
                return DGM_EMESH;
            }
            out.nbr[f1 * K + e1] = int32_t((e2 << 2) | f2);
            out.nbr[f2 * K + e2] = int32_t((e1 << 2) | f1);
        }
        i = j;
    }
    return 0;
}

}  // namespace dgm
