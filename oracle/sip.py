"""Symmetric interior penalty with a facet field (Sec. III, Eqs. (jmp_var_def),
(1st_weak_equation), (weak_penalty)) -- test infrastructure only.

On every interior facet F a tangential field h_s of degree p evolves with the
tangential jump of e and feeds back into the E equation.  With T- the element
of lower index at F, n- its outward normal and [[e]] = e- - e+:

  E equation of T (both sides of F), Eq. (1st_weak_equation):
      (eps de/dt, phi)_T  +=  -(h_s x n_T, phi)_F
  facet equation, Eq. (weak_penalty) in the matrix form printed after it,
  whose blocks are C_F and -C_F^T (so that the extended system stays skew):
      (mu_F / alpha) (dh_s/dt, psi)_F  =  (n- x [[e]], psi)_F

Reading of the printed facet equation: its right-hand side, written with
the half jump and the opposite sign, would make the facet energy negative
(alpha effectively -alpha/2); the matrix form fixes the coupling as above.
mu_F is the mean of the two sides' mu; alpha > 0 is given.  Boundary facets
carry no h_s.  Central flux only (the penalty is the paper's cure for the
central flux's spurious modes); no PML.

Facet basis (the oracle's own; any basis of the same space gives the same e,
h): orthonormal tangents t1 = edge / |edge|, t2 = n- x t1, times scalar
polynomials of degree <= p in the facet parameters (s, t) of the sorted
vertices, orthonormalised in the facet's L2 product, so that the facet mass
is (mu_F / alpha) I.  Unknown (F, d, a) at offset F * 2 NFp + d * NFp + a.

Extended state (per column): [E; H; S], E and H as in oracle.assemble.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import tri_quadrature


def _monomials(p, st):
    """s^i t^j, i + j <= p, at points st [q, 2] -> [q, NFp]."""
    s, t = st[:, 0], st[:, 1]
    return np.stack([s ** i * t ** j for d in range(p + 1) for i in range(d, -1, -1)
                     for j in [d - i]], axis=1)


class SipAssembly:
    """Facet field h_s on the interior facets of an oracle Assembly."""

    def __init__(self, asm, alpha):
        if asm.flux != "central" or asm.has_pml or asm.R != asm.K:
            raise ValueError("the penalty is built for the central flux, no PML, full assembly")
        if not alpha > 0.0:
            raise ValueError("alpha must be positive")
        self.asm = asm
        self.alpha = float(alpha)
        m = asm.mesh
        p = asm.p
        self.NFp = (p + 1) * (p + 2) // 2
        self.facets = [(T, f, int(m.nbr[T, f])) for T in range(m.K) for f in range(4)
                       if m.nbr[T, f] > T]
        self.nF = len(self.facets)
        self.ns = self.nF * 2 * self.NFp
        self._build()

    def _facet_frame(self, T, f):
        """Vertices (sorted ids), unit normal n- (outward of T), area, tangents t1, t2."""
        P, opp = self.asm.mesh.face_vertices(T, f)
        c = np.cross(P[1] - P[0], P[2] - P[0])
        area = 0.5 * np.linalg.norm(c)
        n = c / np.linalg.norm(c)
        if np.dot(n, P[0] - opp) < 0:
            n = -n
        t1 = (P[1] - P[0]) / np.linalg.norm(P[1] - P[0])
        t2 = np.cross(n, t1)
        return P, n, area, np.stack([t1, t2])

    def _build(self):
        a, m = self.asm, self.asm.mesh
        n3, NFp, p = a.n3, self.NFp, a.p
        st, wst = tri_quadrature(p + 2)          # exact for the degree-2p integrands
        rows, cols, vals = [], [], []
        self.mu_F = np.empty(self.nF)
        self.frames = []
        self.coef = []                            # scalar basis: monomials @ coef
        for i, (Tm, f, Tp) in enumerate(self.facets):
            P, n, area, tang = self._facet_frame(Tm, f)
            self.frames.append((P, n, area, tang))
            self.mu_F[i] = 0.5 * (a.mu[Tm] + a.mu[Tp])
            r = P[0] + st[:, :1] * (P[1] - P[0]) + st[:, 1:2] * (P[2] - P[0])
            w = wst * 2.0 * area
            mono = _monomials(p, st)
            G = np.einsum("q,qa,qb->ab", w, mono, mono)
            L = np.linalg.cholesky(G)
            cf = np.linalg.inv(L).T                # psi = mono @ cf, orthonormal on F
            self.coef.append(cf)
            psi = mono @ cf                        # [q, NFp]
            trial = np.einsum("dc,qa->qdac", tang, psi).reshape(len(w), 2 * NFp, 3)
            for T, sgn in ((Tm, 1.0), (Tp, -1.0)):
                B = a._basis_vectors(T, r)        # [q, 3, 3N]
                nT = sgn * n
                # C_F[(T, j, l), (F, d, a)] = -(psi_da x n_T, phi_jl)_F
                X = -np.cross(trial, nT[None, None, :])        # [q, 2NFp, 3]
                blk = np.einsum("q,qci,qkc->ik", w, B, X)      # [3N, 2NFp]
                ii, kk = np.nonzero(np.abs(blk) > 0)
                rows.append(T * n3 + ii)
                cols.append(i * 2 * NFp + kk)
                vals.append(blk[ii, kk])
        self.C_F = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                 shape=(a.K * n3, self.ns))
        nE = a.K * n3
        top = sp.hstack([a.Kmat, sp.vstack([self.C_F, sp.csr_matrix((nE, self.ns))])])
        bottom = sp.hstack([-self.C_F.T, sp.csr_matrix((self.ns, nE + self.ns))])
        self.Kmat = sp.vstack([top, bottom]).tocsr()
        self.ndof = 2 * nE + self.ns
        self.minv_s = np.repeat(self.alpha / self.mu_F, 2 * NFp)   # facet mass inverse

    def apply_minv(self, y):
        nEH = 2 * self.asm.K * self.asm.n3
        out = np.empty_like(y)
        out[:nEH] = self.asm.apply_minv(y[:nEH])
        out[nEH:] = self.minv_s[:, None] * y[nEH:]
        return out

    def energy(self, x):
        """1/2 (e^T M_eps e + h^T M_mu h + sum_F (mu_F / alpha) |h_s|_F^2) per column."""
        nEH = 2 * self.asm.K * self.asm.n3
        s = x[nEH:]
        return self.asm.energy(x[:nEH]) + 0.5 * np.sum(s * s / self.minv_s[:, None], axis=0)

    def facet_moments(self, x):
        """Per facet and column: the L2 norm squared of h_s on F and its integral
        over F (a physical vector) -> ([nF, S], [nF, S, 3])."""
        nEH = 2 * self.asm.K * self.asm.n3
        NFp = self.NFp
        S = x.shape[1]
        s = x[nEH:].reshape(self.nF, 2, NFp, S)
        st, wst = tri_quadrature(self.asm.p + 2)
        norm2 = np.sum(s * s, axis=(1, 2))
        mean = np.empty((self.nF, S, 3))
        mono = _monomials(self.asm.p, st)
        for i, (P, n, area, tang) in enumerate(self.frames):
            ipsi = (wst * 2.0 * area) @ (mono @ self.coef[i])      # int_F psi_a
            mean[i] = np.einsum("das,a,dc->sc", s[i], ipsi, tang)
        return norm2, mean


class SipSolver:
    """LSRK4 stepping and right-hand side of the extended system [E; H; S]."""

    def __init__(self, solver, alpha):
        self.base = solver
        self.sip = SipAssembly(solver.asm, alpha)
        self.S = solver.S

    def pack(self, u, hs=None):
        x0 = self.base.pack(u)
        x = np.zeros((self.sip.ndof, x0.shape[1]))
        x[:x0.shape[0]] = x0
        if hs is not None:
            x[x0.shape[0]:] = hs
        return x

    def unpack(self, x):
        nEH = 2 * self.sip.asm.K * self.sip.asm.n3
        u, _ = self.base.unpack(x[:nEH])
        return u, x[nEH:]

    def rhs(self, x, t=0.0):
        y = self.sip.Kmat @ x
        nEH = 2 * self.sip.asm.K * self.sip.asm.n3
        if self.base.src:
            y[:nEH] += self.base.source_vector(t)
        if getattr(self.base, "inc", None) is not None and self.sip.asm.incident:
            y[:nEH] += self.base.incident_vector(t)
        return self.sip.apply_minv(y)

    def lsrk4(self, x, t0, dt, steps):
        from .solver import LSRK4_A, LSRK4_B, LSRK4_C
        res = np.zeros_like(x)
        t = t0
        for _ in range(steps):
            for k in range(5):
                res = LSRK4_A[k] * res + dt * self.rhs(x, t + LSRK4_C[k] * dt)
                x = x + LSRK4_B[k] * res
            t += dt
        return x
