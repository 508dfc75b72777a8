"""Element and global matrices of the oracle (test infrastructure only).

Everything is integrated by quadrature at *physical* points: reference
quadrature points are mapped to the element, basis functions are evaluated
there through the inverse map of whichever element they belong to (own or
neighbour), and the integrands are formed from physical vectors.

Basis, Eq. (mapped_eh): phi_{j,l}(r) = A^-T e_j phihat_l(A^-1 (r - b)).
Curl by the chain rule: curl phi_{j,l} = (A^-T gradhat phihat_l) x (A^-T e_j).

Semi-discrete system (Sec. III; PML terms of Sec. IV):

  E equation, weak form of Eq. (uwc):
    (eps de/dt, phi)_T = (h, curl phi)_T + sum_F (phi, n x h*)_F
                         - (eps eta e, phi)_T - (p, phi)_T - (j, phi)_T
  H equation, strong form of Eq. (cwc):
    (mu dh/dt, phi)_T = -(curl e, phi)_T - sum_F (phi, n x (e* - e^-))_F
                        - (mu eta h, phi)_T - (q, phi)_T
  PML auxiliaries, Eqs. (p_variable), (q_variable), one pole per Cartesian
  component:
    (dp/dt + Sigma p, phi)_T = (xi eps e, phi)_T,  likewise q with mu, h.

Face states h*, e*: central flux of Eq. (uwc)/(cwc), h* = {{h}}, e* = {{e}};
upwind flux (exact Riemann solution of the 1-D interface problem):
    n x h* = [Z- n x h- + Z+ n x h+ + n x (n x (e- - e+))] / (Z- + Z+)
    n x e* = [Y- n x e- + Y+ n x e+ - n x (n x (h- - h+))] / (Y- + Y+)
with Z = sqrt(mu/eps), Y = 1/Z.  PEC wall (Sec. IV, closing the PML): ghost
state e+ = -e-, h+ = h-, Z+ = Z-.

Global vector layout (per batch column): [E; H; P; Q], each block element
major with entry (T, j, l) at T*3N + j*N + l.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import RefBasis, tet_quadrature, tri_quadrature


def pml_sigma(centroids, lo, hi, thickness, sigma_max, order=2):
    """Per-element damping triple sigma_a = sigma_max (d_a / L)^order at the centroid.

    d_a is the depth of the centroid into the layer along axis a (0 inside the
    box [lo, hi]).  Piecewise constant per element, as Sec. V requires for
    constant-coefficient element operators.
    """
    c = np.asarray(centroids, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = np.maximum(0.0, np.maximum(lo[None, :] - c, c - hi[None, :]))
    return sigma_max * (d / thickness) ** order


def pml_eta_xi(sigma):
    """Diagonals of eta and xi for stretching factors sigma [..., 3].

    Partial fractions of the stretched tensor of Sec. IV: with lambda = -i omega,
      lambda eps~_aa / eps = (lambda + s_b)(lambda + s_c) / (lambda + s_a)
                           = lambda + eta_aa + xi_aa / (lambda + s_a),
      eta_aa = s_b + s_c - s_a,  xi_aa = (s_a - s_b)(s_a - s_c).
    """
    s = np.asarray(sigma, dtype=np.float64)
    sa, sb, sc = s[..., 0], s[..., 1], s[..., 2]
    eta = np.stack([sb + sc - sa, sc + sa - sb, sa + sb - sc], axis=-1)
    xi = np.stack([(sa - sb) * (sa - sc), (sb - sc) * (sb - sa), (sc - sa) * (sc - sb)],
                  axis=-1)
    return eta, xi


class Assembly:
    """Assembled semi-discrete operator of one mesh.

    mesh:  oracle.mesh.Mesh
    eps, mu: per-element scalars [K]
    flux: "central" or "upwind"
    sigma: per-element PML damping triples [K, 3] or None
    rows: elements whose equations are assembled (default: all).  With a
        subset, the operator maps the full state to those elements' rows
        only, which lets the oracle evaluate the right-hand side of sampled
        elements of a mesh too large to assemble whole.
    incident: boundary faces through which an incident field enters, as a
        list of vertex-id triples, or None.  On those faces the exterior
        state is e+ = e- + 2 E_inc, h+ = -h-, Z+ = Z-: the listing of Appendix A
        sets the boundary value of e to 2 E_inc + e and builds the E equation as
        the transpose of the H equation's operator, which leaves no E-equation
        boundary term, i.e. tangential h* = 0 (a magnetic wall radiating the
        incident field).  Operator terms: only the upwind H-H term
        Z (phi, n x (n x h)); the rest is a forcing (Solver.incident_vector).
    """

    def __init__(self, mesh, p, eps, mu, flux="central", sigma=None, rows=None, incident=None):
        self.mesh = mesh
        self.rows = np.arange(mesh.K) if rows is None else np.asarray(rows, dtype=np.int64)
        self.R = self.rows.size
        self.pos = -np.ones(mesh.K, dtype=np.int64)
        self.pos[self.rows] = np.arange(self.R)
        self.p = p
        self.basis = RefBasis(p)
        self.N = self.basis.N
        self.K = mesh.K
        self.n3 = 3 * self.N
        # eps/mu may be complex (complex-step derivatives in oracle.adjoint)
        self.eps = np.asarray(eps) * np.ones(self.K)
        self.mu = np.asarray(mu) * np.ones(self.K)
        if flux not in ("central", "upwind"):
            raise ValueError(flux)
        self.flux = flux
        self.has_pml = sigma is not None
        self.sigma = None if sigma is None else np.asarray(sigma, dtype=np.float64)
        self.incident = set()
        if incident is not None:
            keys = {}
            for T in range(mesh.K):
                for f in range(4):
                    keys[tuple(np.delete(mesh.tets[T], f))] = (T, f)
            for tri in incident:
                T, f = keys[tuple(sorted(int(v) for v in tri))]
                if mesh.nbr[T, f] >= 0:
                    raise ValueError("incident face %s is not a boundary face" % (tri,))
                self.incident.add((T, f))
        self._volume()
        self._faces()
        self._global()

    # -- basis vectors at physical points ---------------------------------
    def _basis_vectors(self, T, r, with_curl=False):
        """phi_{j,l}(r) for points r [n,3] of element T -> [n, 3, 3N] (+ curls)."""
        out = self._basis_vectors_many(np.array([T]), r[None], with_curl)
        return tuple(o[0] for o in out) if with_curl else out[0]

    def _basis_vectors_many(self, Ts, r, with_curl=False):
        """Batched over elements: Ts [E], r [E, n, 3] -> [E, n, 3, 3N] (+ curls)."""
        m = self.mesh
        E, n = r.shape[0], r.shape[1]
        rh = np.einsum("eaj,enj->ena", m.Ainv[Ts], r - m.b[Ts][:, None, :])
        V = self.basis.values(rh.reshape(-1, 3)).reshape(E, n, self.N)
        Ait = np.transpose(m.Ainv[Ts], (0, 2, 1))               # A^-T per element
        B = np.einsum("ecj,eql->eqcjl", Ait, V).reshape(E, n, 3, self.n3)
        if not with_curl:
            return B
        G = self.basis.gradients(rh.reshape(-1, 3)).reshape(E, n, self.N, 3)
        gphys = np.einsum("eca,eqla->eqlc", Ait, G)              # physical gradients
        vj = np.transpose(Ait, (0, 2, 1))                       # vj[e, j, :] = A^-T e_j
        C = np.cross(gphys[:, :, None, :, :], vj[:, None, :, None, :], axis=-1)
        C = np.transpose(C, (0, 1, 4, 2, 3)).reshape(E, n, 3, self.n3)
        return B, C

    # -- element volume matrices ------------------------------------------
    def _volume(self, chunk=64):
        m, n3 = self.mesh, self.n3
        rq, wq = tet_quadrature(self.p + 3)
        self.M1 = np.empty((self.R, n3, n3))
        self.C_eh = np.empty((self.R, n3, n3))   # (curl phi_test, phi_trial)
        self.pml_blocks = {}
        if self.has_pml:
            eta, xi = pml_eta_xi(self.sigma)
            self._eta, self._xi = eta, xi
            for key in ("eta", "sig", "xi"):
                self.pml_blocks[key] = np.zeros((self.R, n3, n3))
        for i0 in range(0, self.R, chunk):
            Ts = self.rows[i0:i0 + chunk]
            r = np.einsum("eij,qj->eqi", m.A[Ts], rq) + m.b[Ts][:, None, :]
            w = wq[None, :] * np.abs(m.det[Ts])[:, None]
            B, C = self._basis_vectors_many(Ts, r, with_curl=True)
            self.M1[i0:i0 + len(Ts)] = np.einsum("eq,eqci,eqcj->eij", w, B, B)
            self.C_eh[i0:i0 + len(Ts)] = np.einsum("eq,eqci,eqcj->eij", w, C, B)
            if self.has_pml:
                for key, d in (("eta", self._eta[Ts]), ("sig", self.sigma[Ts]),
                               ("xi", self._xi[Ts])):
                    self.pml_blocks[key][i0:i0 + len(Ts)] = np.einsum(
                        "eq,eqci,ec,eqcj->eij", w, B, d, B)

    # -- face matrices ------------------------------------------------------
    def _faces(self, chunk=64):
        m = self.mesh
        st, wst = tri_quadrature(self.p + 2)
        self.face = []   # list of dicts per (T, f)
        for i0 in range(0, self.R, chunk):
            Ts = self.rows[i0:i0 + chunk]
            for f in range(4):
                frames = [m.face_frame(T, f) for T in Ts]
                P = np.stack([fr[0] for fr in frames])             # [E, 3, 3]
                nrm = np.stack([fr[1] for fr in frames])           # [E, 3]
                area = np.array([fr[2] for fr in frames])
                r = P[:, None, 0, :] + st[None, :, :1] * (P[:, None, 1, :] - P[:, None, 0, :]) \
                    + st[None, :, 1:2] * (P[:, None, 2, :] - P[:, None, 0, :])
                w = wst[None, :] * 2.0 * area[:, None]
                Bo = self._basis_vectors_many(Ts, r)
                nb = m.nbr[Ts, f]
                has = nb >= 0
                Bn = np.zeros_like(Bo)
                if np.any(has):
                    Bn[has] = self._basis_vectors_many(nb[has], r[has])

                def cross_n(B):
                    return np.cross(nrm[:, None, :, None], B, axis=2)

                x_own = np.einsum("eq,eqci,eqcj->eij", w, Bo, cross_n(Bo))
                xx_own = np.einsum("eq,eqci,eqcj->eij", w, Bo, cross_n(cross_n(Bo)))
                x_nbr = np.einsum("eq,eqci,eqcj->eij", w, Bo, cross_n(Bn))
                xx_nbr = np.einsum("eq,eqci,eqcj->eij", w, Bo, cross_n(cross_n(Bn)))
                for e, T in enumerate(Ts):
                    ent = dict(T=T, f=f, nb=nb[e], x_own=x_own[e], xx_own=xx_own[e])
                    if nb[e] >= 0:
                        ent["x_nbr"] = x_nbr[e]
                        ent["xx_nbr"] = xx_nbr[e]
                    self.face.append(ent)

    # -- global operator -----------------------------------------------------
    def _global(self):
        K, R, n3 = self.K, self.R, self.n3
        nblk = 4 if self.has_pml else 2
        self.nblk = nblk
        self.ndof = nblk * K * n3
        rows, cols, vals = [], [], []

        def put(bi, T, bj, T2, blk):
            r0 = bi * R * n3 + self.pos[T] * n3
            c0 = bj * K * n3 + T2 * n3
            ii, jj = np.nonzero(blk)
            rows.append(ii + r0)
            cols.append(jj + c0)
            vals.append(blk[ii, jj])

        E, H, P, Q = 0, 1, 2, 3
        Z = np.sqrt(self.mu / self.eps)
        upwind = self.flux == "upwind"
        for i, T in enumerate(self.rows):
            # volume: E eq weak form (h, curl phi); H eq strong form -(curl e, phi)
            put(E, T, H, T, self.C_eh[i])
            put(H, T, E, T, -self.C_eh[i].T)
        for ent in self.face:
            T, nb = ent["T"], ent["nb"]
            if nb < 0 and (T, ent["f"]) in self.incident:   # e+ = e- + 2 E_inc, h+ = -h-
                if upwind:   # n x (e* - e-) = n x E_inc - Z n x (n x h-)
                    put(H, T, H, T, Z[T] * ent["xx_own"])
                continue
            if nb < 0:   # PEC wall: e+ = -e-, h+ = h-
                put(E, T, H, T, ent["x_own"])
                if upwind:
                    put(E, T, E, T, ent["xx_own"] / Z[T])
                put(H, T, E, T, ent["x_own"])
                continue
            Zm, Zp = Z[T], Z[nb]
            Ym, Yp = 1.0 / Zm, 1.0 / Zp
            if upwind:
                cm, cp, be = Zm / (Zm + Zp), Zp / (Zm + Zp), 1.0 / (Zm + Zp)
                dp, bh = Yp / (Ym + Yp), 1.0 / (Ym + Yp)
            else:
                cm, cp, be, dp, bh = 0.5, 0.5, 0.0, 0.5, 0.0
            # E eq: + (phi, n x h*)
            put(E, T, H, T, cm * ent["x_own"])
            put(E, T, H, nb, cp * ent["x_nbr"])
            if be:
                put(E, T, E, T, be * ent["xx_own"])
                put(E, T, E, nb, -be * ent["xx_nbr"])
            # H eq: - (phi, n x (e* - e-))
            put(H, T, E, T, dp * ent["x_own"])
            put(H, T, E, nb, -dp * ent["x_nbr"])
            if bh:
                put(H, T, H, T, bh * ent["xx_own"])
                put(H, T, H, nb, -bh * ent["xx_nbr"])
        if self.has_pml:
            for i, T in enumerate(self.rows):
                if not np.any(self.sigma[T] != 0.0):
                    continue
                pb = self.pml_blocks
                put(E, T, E, T, -self.eps[T] * pb["eta"][i])
                put(E, T, P, T, -self.M1[i])
                put(H, T, H, T, -self.mu[T] * pb["eta"][i])
                put(H, T, Q, T, -self.M1[i])
                put(P, T, P, T, -pb["sig"][i])
                put(P, T, E, T, self.eps[T] * pb["xi"][i])
                put(Q, T, Q, T, -pb["sig"][i])
                put(Q, T, H, T, self.mu[T] * pb["xi"][i])
        self.Kmat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                                           np.concatenate(cols))),
                                  shape=(nblk * R * n3, self.ndof))
        self.Kmat.sum_duplicates()
        # element mass blocks per field block: eps M1, mu M1, M1, M1 (dense inverses)
        er, mr = self.eps[self.rows], self.mu[self.rows]
        scale = [er, mr, np.ones(R), np.ones(R)][:nblk]
        self.Minv = [np.linalg.inv(s[:, None, None] * self.M1) for s in scale]

    # -- application -----------------------------------------------------------
    def apply_minv(self, y):
        """Block-diagonal mass inverse on row-space vectors y [nblk*R*3N, S]."""
        R, n3 = self.R, self.n3
        out = np.empty_like(y)
        for bi in range(self.nblk):
            blk = y[bi * R * n3:(bi + 1) * R * n3].reshape(R, n3, -1)
            out[bi * R * n3:(bi + 1) * R * n3] = np.matmul(self.Minv[bi], blk).reshape(R * n3, -1)
        return out

    def energy(self, x):
        """Discrete energy 1/2 (e^T M_eps e + h^T M_mu h) per column (full assembly)."""
        K, n3 = self.K, self.n3
        assert self.R == K
        e = x[:K * n3].reshape(K, n3, -1)
        h = x[K * n3:2 * K * n3].reshape(K, n3, -1)
        we = np.einsum("kis,kij,kjs->s", e, self.eps[:, None, None] * self.M1, e)
        wh = np.einsum("kis,kij,kjs->s", h, self.mu[:, None, None] * self.M1, h)
        return 0.5 * (we + wh)
