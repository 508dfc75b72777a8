"""Mixed-order oracle: E of degree pE, H of degree pH (test infrastructure only).

Sec. III, Eqs. (triale)/(trialh) discretise e in the covariant space of degree
p+1 and h in that of degree p.  The weak forms are those of oracle.assemble --
E equation (uwc) in weak form, H equation (cwc) in strong form, central or
upwind face states, PEC ghost states -- with the test and trial functions of
each field taken from that field's own space, so the volume-curl and face
blocks are rectangular.  Everything is again integrated by quadrature at
physical points; no PML.

Global vector layout (per batch column): [E; H], E element-major with entry
(T, j, l) at T 3 N_E + j N_E + l, H likewise with N_H.
State convention shared with the tests: (K, S, 6, N_E) with the H modes
l >= N_H zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import RefBasis, tet_quadrature, tri_quadrature
from .solver import LSRK4_A, LSRK4_B, LSRK4_C, source_time


def _vectors(mesh, basis, Ts, r, with_curl=False):
    """phi_{j,l}(r) = A^-T e_j phihat_l(A^-1 (r - b)) for points r [E, n, 3] of
    elements Ts -> [E, n, 3, 3N] (+ curls by the chain rule)."""
    E, n = r.shape[0], r.shape[1]
    N = basis.N
    rh = np.einsum("eaj,enj->ena", mesh.Ainv[Ts], r - mesh.b[Ts][:, None, :])
    V = basis.values(rh.reshape(-1, 3)).reshape(E, n, N)
    Ait = np.transpose(mesh.Ainv[Ts], (0, 2, 1))
    B = np.einsum("ecj,eql->eqcjl", Ait, V).reshape(E, n, 3, 3 * N)
    if not with_curl:
        return B
    G = basis.gradients(rh.reshape(-1, 3)).reshape(E, n, N, 3)
    gphys = np.einsum("eca,eqla->eqlc", Ait, G)
    vj = np.transpose(Ait, (0, 2, 1))
    C = np.cross(gphys[:, :, None, :, :], vj[:, None, :, None, :], axis=-1)
    C = np.transpose(C, (0, 1, 4, 2, 3)).reshape(E, n, 3, 3 * N)
    return B, C


class MixedAssembly:
    """Assembled semi-discrete operator with E of degree pE and H of degree pH."""

    def __init__(self, mesh, pE, pH, eps, mu, flux="central"):
        if flux not in ("central", "upwind"):
            raise ValueError(flux)
        self.mesh, self.pE, self.pH, self.flux = mesh, pE, pH, flux
        self.bE, self.bH = RefBasis(pE), RefBasis(pH)
        self.NE, self.NH = self.bE.N, self.bH.N
        self.nE, self.nH = 3 * self.NE, 3 * self.NH
        self.K = mesh.K
        self.eps = np.asarray(eps, dtype=np.float64) * np.ones(self.K)
        self.mu = np.asarray(mu, dtype=np.float64) * np.ones(self.K)
        self._volume()
        self._faces()
        self._global()

    def _volume(self, chunk=64):
        m = self.mesh
        q = max(self.pE, self.pH) + 3
        rq, wq = tet_quadrature(q)
        K = self.K
        self.ME = np.empty((K, self.nE, self.nE))
        self.MH = np.empty((K, self.nH, self.nH))
        self.C_eh = np.empty((K, self.nE, self.nH))   # (curl phi^E_test, phi^H_trial)
        for i0 in range(0, K, chunk):
            Ts = np.arange(i0, min(K, i0 + chunk))
            r = np.einsum("eij,qj->eqi", m.A[Ts], rq) + m.b[Ts][:, None, :]
            w = wq[None, :] * np.abs(m.det[Ts])[:, None]
            BE, CE = _vectors(m, self.bE, Ts, r, with_curl=True)
            BH = _vectors(m, self.bH, Ts, r)
            self.ME[Ts] = np.einsum("eq,eqci,eqcj->eij", w, BE, BE)
            self.MH[Ts] = np.einsum("eq,eqci,eqcj->eij", w, BH, BH)
            self.C_eh[Ts] = np.einsum("eq,eqci,eqcj->eij", w, CE, BH)

    def _faces(self, chunk=64):
        m = self.mesh
        st, wst = tri_quadrature(max(self.pE, self.pH) + 2)
        self.face = []
        K = self.K
        for i0 in range(0, K, chunk):
            Ts = np.arange(i0, min(K, i0 + chunk))
            for f in range(4):
                frames = [m.face_frame(T, f) for T in Ts]
                P = np.stack([fr[0] for fr in frames])
                nrm = np.stack([fr[1] for fr in frames])
                area = np.array([fr[2] for fr in frames])
                r = P[:, None, 0, :] + st[None, :, :1] * (P[:, None, 1, :] - P[:, None, 0, :]) \
                    + st[None, :, 1:2] * (P[:, None, 2, :] - P[:, None, 0, :])
                w = wst[None, :] * 2.0 * area[:, None]
                nb = m.nbr[Ts, f]
                has = nb >= 0
                own = {"E": _vectors(m, self.bE, Ts, r), "H": _vectors(m, self.bH, Ts, r)}
                nbr = {}
                for key, basis in (("E", self.bE), ("H", self.bH)):
                    Bn = np.zeros_like(own[key])
                    if np.any(has):
                        Bn[has] = _vectors(m, basis, nb[has], r[has])
                    nbr[key] = Bn
                cross = lambda B: np.cross(nrm[:, None, :, None], B, axis=2)
                blk = lambda test, trial: np.einsum("eq,eqci,eqcj->eij", w, test, trial)
                x = {}
                for a in "EH":
                    for b in "EH":
                        x[("x", a, b, "own")] = blk(own[a], cross(own[b]))
                        x[("x", a, b, "nbr")] = blk(own[a], cross(nbr[b]))
                        x[("xx", a, b, "own")] = blk(own[a], cross(cross(own[b])))
                        x[("xx", a, b, "nbr")] = blk(own[a], cross(cross(nbr[b])))
                for e, T in enumerate(Ts):
                    ent = {"T": T, "f": f, "nb": nb[e]}
                    for k, v in x.items():
                        ent[k] = v[e]
                    self.face.append(ent)

    def _global(self):
        K, nE, nH = self.K, self.nE, self.nH
        off = {"E": 0, "H": K * nE}
        size = {"E": nE, "H": nH}
        rows, cols, vals = [], [], []

        def put(a, T, b, T2, blk):
            ii, jj = np.nonzero(blk)
            rows.append(ii + off[a] + T * size[a])
            cols.append(jj + off[b] + T2 * size[b])
            vals.append(blk[ii, jj])

        Z = np.sqrt(self.mu / self.eps)
        up = self.flux == "upwind"
        for T in range(K):
            put("E", T, "H", T, self.C_eh[T])
            put("H", T, "E", T, -self.C_eh[T].T)
        for ent in self.face:
            T, nb = ent["T"], ent["nb"]
            if nb < 0:   # PEC: e+ = -e-, h+ = h-
                put("E", T, "H", T, ent[("x", "E", "H", "own")])
                if up:
                    put("E", T, "E", T, ent[("xx", "E", "E", "own")] / Z[T])
                put("H", T, "E", T, ent[("x", "H", "E", "own")])
                continue
            Zm, Zp = Z[T], Z[nb]
            Ym, Yp = 1.0 / Zm, 1.0 / Zp
            if up:
                cm, cp, be = Zm / (Zm + Zp), Zp / (Zm + Zp), 1.0 / (Zm + Zp)
                dp, bh = Yp / (Ym + Yp), 1.0 / (Ym + Yp)
            else:
                cm, cp, be, dp, bh = 0.5, 0.5, 0.0, 0.5, 0.0
            put("E", T, "H", T, cm * ent[("x", "E", "H", "own")])
            put("E", T, "H", nb, cp * ent[("x", "E", "H", "nbr")])
            if be:
                put("E", T, "E", T, be * ent[("xx", "E", "E", "own")])
                put("E", T, "E", nb, -be * ent[("xx", "E", "E", "nbr")])
            put("H", T, "E", T, dp * ent[("x", "H", "E", "own")])
            put("H", T, "E", nb, -dp * ent[("x", "H", "E", "nbr")])
            if bh:
                put("H", T, "H", T, bh * ent[("xx", "H", "H", "own")])
                put("H", T, "H", nb, -bh * ent[("xx", "H", "H", "nbr")])
        n = K * (nE + nH)
        self.Kmat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(n, n))
        self.Kmat.sum_duplicates()
        self.MinvE = np.linalg.inv(self.eps[:, None, None] * self.ME)
        self.MinvH = np.linalg.inv(self.mu[:, None, None] * self.MH)

    def apply_minv(self, y):
        K, nE, nH = self.K, self.nE, self.nH
        out = np.empty_like(y)
        out[:K * nE] = np.matmul(self.MinvE, y[:K * nE].reshape(K, nE, -1)).reshape(K * nE, -1)
        out[K * nE:] = np.matmul(self.MinvH, y[K * nE:].reshape(K, nH, -1)).reshape(K * nH, -1)
        return out


class MixedSolver:
    """Right-hand side, LSRK4, sources, projection and energy over a MixedAssembly."""

    def __init__(self, asm, S=1, sources=None):
        self.asm, self.S = asm, S
        self.src = []
        for s, rec in enumerate(sources or []):
            if rec is None:
                continue
            pos = np.asarray(rec["pos"], dtype=np.float64)
            T = asm.mesh.locate(pos)
            B = _vectors(asm.mesh, asm.bE, np.array([T]), pos[None, None, :])[0, 0]
            self.src.append((s, T, np.asarray(rec["dir"], dtype=np.float64) @ B, rec))

    def pack(self, u):
        a = self.asm
        K, NE, NH, S = a.K, a.NE, a.NH, u.shape[1]
        x = np.zeros((K * (a.nE + a.nH), S))
        x[:K * a.nE] = u[:, :, 0:3, :NE].transpose(0, 2, 3, 1).reshape(K * a.nE, S)
        x[K * a.nE:] = u[:, :, 3:6, :NH].transpose(0, 2, 3, 1).reshape(K * a.nH, S)
        return x

    def unpack(self, x):
        a = self.asm
        K, NE, NH, S = a.K, a.NE, a.NH, x.shape[1]
        u = np.zeros((K, S, 6, NE))
        u[:, :, 0:3, :] = x[:K * a.nE].reshape(K, 3, NE, S).transpose(0, 3, 1, 2)
        u[:, :, 3:6, :NH] = x[K * a.nE:].reshape(K, 3, NH, S).transpose(0, 3, 1, 2)
        return u

    def rhs(self, x, t=0.0):
        a = self.asm
        y = a.Kmat @ x
        for s, T, w, rec in self.src:
            y[T * a.nE:(T + 1) * a.nE, s] -= source_time(t, rec["f0"], rec["bw"], rec["t0"]) * w
        return a.apply_minv(y)

    def lsrk4(self, x, t0, dt, steps):
        res = np.zeros_like(x)
        t = t0
        for _ in range(steps):
            for k in range(5):
                res = LSRK4_A[k] * res + dt * self.rhs(x, t + LSRK4_C[k] * dt)
                x = x + LSRK4_B[k] * res
            t += dt
        return x

    def project(self, fn, field):
        """L2 projection of fn(r) -> [n, 3] onto field 'E' (degree pE) or 'H' (pH):
        coefficients (K, 3, N_field)."""
        a, m = self.asm, self.asm.mesh
        basis = a.bE if field == "E" else a.bH
        rq, wq = tet_quadrature(max(a.pE, a.pH) + 4)
        out = np.empty((a.K, 3, basis.N))
        for T in range(a.K):
            r = rq @ m.A[T].T + m.b[T][None, :]
            w = wq * abs(m.det[T])
            B = _vectors(m, basis, np.array([T]), r[None])[0]
            out[T] = np.linalg.solve(np.einsum("q,qci,qcj->ij", w, B, B),
                                     np.einsum("q,qc,qci->i", w, fn(r), B)).reshape(3, basis.N)
        return out

    def evaluate_e(self, coef, T, r):
        """E of element T with coefficients coef (3 N_E,) at points r [n, 3]."""
        B = _vectors(self.asm.mesh, self.asm.bE, np.array([T]), r[None])[0]
        return np.einsum("qci,i->qc", B, coef)

    def energy(self, x):
        a = self.asm
        K = a.K
        e = x[:K * a.nE].reshape(K, a.nE, -1)
        h = x[K * a.nE:].reshape(K, a.nH, -1)
        we = np.einsum("kis,kij,kjs->s", e, a.eps[:, None, None] * a.ME, e)
        wh = np.einsum("kis,kij,kjs->s", h, a.mu[:, None, None] * a.MH, h)
        return 0.5 * (we + wh)
