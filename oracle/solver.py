"""Right-hand side, time stepping, projection, sources and receivers of the oracle.

Test infrastructure only (see the package docstring).

Time integrators
----------------
* Leapfrog (Sec. V: "classic leap-frog"), staggered E/H.  Reading for the
  start: H is given at t = 0 and advanced half a step with the H equation,
  H^{1/2} = H^0 + dt/2 L_H(E^0); then E^{n+1} = E^n + dt L_E(H^{n+1/2}),
  H^{n+3/2} = H^{n+1/2} + dt L_H(E^{n+1}).  Needs a flux whose E equation
  depends on H only (central).
* Low-storage RK4, five stages, 2N storage (Carpenter & Kennedy 1994):
  res = a_k res + dt L(u, t + c_k dt);  u = u + b_k res.

Point dipole source: j = d delta(r - r_s) g(t), entering the E equation as
-(j, phi)_T = -g(t) d . phi(r_s) in the element containing r_s, with the
Gaussian-modulated sine g(t) = sin(2 pi f0 (t - t0)) exp(-(t - t0)^2 / (2 s^2)),
s = 1/(2 pi bw).
"""
from __future__ import annotations

import math

import numpy as np

from .basis import tet_quadrature

# Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage Runge-Kutta.
LSRK4_A = (0.0,
           -567301805773.0 / 1357537059087.0,
           -2404267990393.0 / 2016746695238.0,
           -3550918686646.0 / 2091501179385.0,
           -1275806237668.0 / 842570457699.0)
LSRK4_B = (1432997174477.0 / 9575080441755.0,
           5161836677717.0 / 13612068292357.0,
           1720146321549.0 / 2090206949498.0,
           3134564353537.0 / 4481467310338.0,
           2277821191437.0 / 14882151754819.0)
LSRK4_C = (0.0,
           1432997174477.0 / 9575080441755.0,
           2526269341429.0 / 6820363962896.0,
           2006345519317.0 / 3224310063776.0,
           2802321613138.0 / 2924317926251.0)


def source_time(t, f0, bw, t0):
    s = 1.0 / (2.0 * math.pi * bw)
    return math.sin(2.0 * math.pi * f0 * (t - t0)) * math.exp(-(t - t0) ** 2 / (2.0 * s * s))


class Solver:
    """Time stepper over an oracle Assembly with batch columns S.

    sources: list (length S or empty) of None or dict(pos, dir, f0, bw, t0);
    column s is driven by sources[s].
    """

    def __init__(self, asm, S=1, sources=None):
        self.asm = asm
        self.S = S
        self.src = []
        sources = sources or []
        for s, rec in enumerate(sources):
            if rec is None:
                continue
            T = asm.mesh.locate(np.asarray(rec["pos"], dtype=np.float64))
            B = asm._basis_vectors(T, np.asarray(rec["pos"], dtype=np.float64)[None, :])[0]
            w = np.asarray(rec["dir"], dtype=np.float64) @ B      # d . phi_{j,l}(r_s)
            self.src.append((s, T, w, rec))

    # -- conversion from the shared (K, S, 6, N) state convention ------------
    def pack(self, u, aux=None):
        a = self.asm
        K, N, S = a.K, a.N, u.shape[1]
        x = np.zeros((a.ndof, S))
        x[:K * 3 * N] = u[:, :, 0:3, :].transpose(0, 2, 3, 1).reshape(K * 3 * N, S)
        x[K * 3 * N:2 * K * 3 * N] = u[:, :, 3:6, :].transpose(0, 2, 3, 1).reshape(K * 3 * N, S)
        if a.nblk == 4 and aux is not None:
            x[2 * K * 3 * N:3 * K * 3 * N] = aux[:, :, 0:3, :].transpose(0, 2, 3, 1).reshape(-1, S)
            x[3 * K * 3 * N:] = aux[:, :, 3:6, :].transpose(0, 2, 3, 1).reshape(-1, S)
        return x

    def unpack(self, y, nelem=None):
        """Row-space vector -> (fields (R, S, 6, N), aux or None)."""
        a = self.asm
        R = a.R if nelem is None else nelem
        N, S = a.N, y.shape[1]
        blocks = [y[b * R * 3 * N:(b + 1) * R * 3 * N].reshape(R, 3, N, S).transpose(0, 3, 1, 2)
                  for b in range(a.nblk)]
        u = np.concatenate(blocks[:2], axis=2)
        aux = np.concatenate(blocks[2:], axis=2) if a.nblk == 4 else None
        return u, aux

    # -- operator --------------------------------------------------------------
    def apply_k(self, x):
        """K x with the assembled sparse operator (scipy's CSR product)."""
        return self.asm.Kmat @ x

    def source_vector(self, t):
        a = self.asm
        f = np.zeros((a.Kmat.shape[0], self.S), dtype=np.result_type(a.Kmat.dtype, np.float64))
        for s, T, w, rec in self.src:
            if a.pos[T] < 0:
                continue
            g = source_time(t, rec["f0"], rec["bw"], rec["t0"])
            r0 = a.pos[T] * a.n3
            f[r0:r0 + a.n3, s] -= g * w
        return f

    def set_incident(self, E0, direction, speed, f0, bw, t0, quad=None):
        """Incident plane wave E_inc(r, t) = E0 g(t - t0 - d . r / speed),
        g(tau) = cos(2 pi f0 tau) exp(-tau^2 / (2 s^2)), s = 1/(2 pi bw), on the
        assembly's incident faces; its face integrals use a collapsed Gauss
        rule with `quad` points per direction (default p + 4)."""
        self.inc = dict(E0=np.asarray(E0, np.float64), d=np.asarray(direction, np.float64),
                        c=float(speed), f0=float(f0), bw=float(bw), t0=float(t0),
                        quad=int(quad) if quad else self.asm.p + 4)

    def incident_vector(self, t):
        """Forcing of the incident faces (e+ - e- = 2 E_inc, h+ = -h-, Z+ = Z-):
        H rows -(phi, n x E_inc)_F (central and upwind alike), E rows
        -(1/Z) (phi, n x (n x E_inc))_F for the upwind flux; by quadrature on
        each face at physical points."""
        from .basis import tri_quadrature
        a, m = self.asm, self.asm.mesh
        f = np.zeros((a.Kmat.shape[0], self.S))
        inc = getattr(self, "inc", None)
        if inc is None or not a.incident:
            return f
        st, wst = tri_quadrature(inc["quad"])
        s = 1.0 / (2.0 * math.pi * inc["bw"])
        Z = np.sqrt(a.mu / a.eps)
        for (T, fc) in a.incident:
            if a.pos[T] < 0:
                continue
            P, nrm, area = m.face_frame(T, fc)
            r = P[0] + st[:, :1] * (P[1] - P[0]) + st[:, 1:2] * (P[2] - P[0])
            w = wst * 2.0 * area
            tau = t - inc["t0"] - r @ inc["d"] / inc["c"]
            g = np.cos(2.0 * math.pi * inc["f0"] * tau) * np.exp(-tau ** 2 / (2.0 * s * s))
            Einc = g[:, None] * inc["E0"][None, :]
            B = a._basis_vectors(T, r)                                   # [q, 3, 3N]
            nE = np.cross(nrm[None, :], Einc)
            nnE = np.cross(nrm[None, :], nE)
            r0 = a.pos[T] * a.n3
            hoff = a.R * a.n3
            f[hoff + r0:hoff + r0 + a.n3, :] -= np.einsum("q,qc,qci->i", w, nE, B)[:, None]
            if a.flux == "upwind":
                f[r0:r0 + a.n3, :] -= (np.einsum("q,qc,qci->i", w, nnE, B) / Z[T])[:, None]
        return f

    def rhs(self, x, t=0.0):
        """du/dt for the assembled rows: M^-1 (K x + f(t))."""
        y = self.apply_k(x)
        if self.src:
            y = y + self.source_vector(t)
        if getattr(self, "inc", None) is not None and self.asm.incident:
            y = y + self.incident_vector(t)
        return self.asm.apply_minv(y)

    def lsrk4(self, x, t0, dt, steps, callback=None):
        res = np.zeros_like(x)
        t = t0
        for n in range(steps):
            for k in range(5):
                res = LSRK4_A[k] * res + dt * self.rhs(x, t + LSRK4_C[k] * dt)
                x = x + LSRK4_B[k] * res
            t += dt
            if callback is not None:
                callback(n + 1, t, x)
        return x

    def leapfrog(self, x, t0, dt, steps, callback=None):
        """Staggered leapfrog; on return E is at t0 + steps dt, H half a step later."""
        a = self.asm
        nE = a.K * a.n3
        assert a.nblk == 2 and a.flux == "central"
        x = x.copy()
        x[nE:] += 0.5 * dt * self.rhs(x, t0)[nE:]
        t = t0
        for n in range(steps):
            x[:nE] += dt * self.rhs(x, t + 0.5 * dt)[:nE]
            x[nE:] += dt * self.rhs(x, t + dt)[nE:]
            t += dt
            if callback is not None:
                callback(n + 1, t, x)
        return x

    def leapfrog_pml(self, x, t0, dt, steps, callback=None):
        """Staggered leapfrog with the PML's dissipative terms taken by the
        trapezoid rule (Sec. V: leap-frog, dissipative terms by the trapezoid
        rule, explicit because every such term is element-local).

        Unknowns: e at integer steps, h at half steps; the auxiliaries p (of the
        E equation) at half steps and q (of the H equation) at integer steps, so
        that every equation is centred.  With the element mass M1, the PML
        matrices M_eta, M_Sigma, M_xi of Sec. IV and the curl/flux blocks K_EH,
        K_HE of the central flux, one step from (e^n, h^{n+1/2}, p^{n+1/2}, q^n):

          (M1 + dt/2 M_Sigma) q^{n+1}   = (M1 - dt/2 M_Sigma) q^n + dt mu M_xi h^{n+1/2}
          eps (M1 + dt/2 M_eta) e^{n+1} = eps (M1 - dt/2 M_eta) e^n
                                          + dt (K_EH h^{n+1/2} - M1 p^{n+1/2} - (j, phi)(t + dt/2))
          (M1 + dt/2 M_Sigma) p^{n+3/2} = (M1 - dt/2 M_Sigma) p^{n+1/2} + dt eps M_xi e^{n+1}
          mu (M1 + dt/2 M_eta) h^{n+3/2} = mu (M1 - dt/2 M_eta) h^{n+1/2}
                                          + dt (K_HE e^{n+1} - M1 q^{n+1})

        Start (h, q and p given at t0): h and p advance half a step with the
        same updates over dt/2 from e^0, q^0.  On return e is at t0 + steps dt
        and h, p half a step later.  Without a PML (or with sigma = 0) this is
        the plain staggered leapfrog."""
        a = self.asm
        K, n3 = a.K, a.n3
        assert a.flux == "central" and a.R == K
        nE = K * n3
        Keh = a.Kmat[:nE, nE:2 * nE]
        Khe = a.Kmat[nE:2 * nE, :nE]
        M1 = a.M1
        eps = a.eps[:, None, None]
        mu = a.mu[:, None, None]
        if a.has_pml:
            Eta, Sig, Xi = a.pml_blocks["eta"], a.pml_blocks["sig"], a.pml_blocks["xi"]
            # auxiliaries exist only in elements with a damping (elsewhere they
            # are not coupled, as in the assembled operator)
            M1aux = M1 * np.any(a.sigma[a.rows] != 0.0, axis=1)[:, None, None]
        else:
            Eta = Sig = Xi = np.zeros_like(M1)
            M1aux = np.zeros_like(M1)
        blk = lambda v, b: v[b * nE:(b + 1) * nE].reshape(K, n3, -1)
        mv = lambda Mats, v: np.matmul(Mats, v)

        def field_update(v, mat, rhs_vec, h):
            """mat (M1 + h/2 M_eta) v_new = mat (M1 - h/2 M_eta) v + h rhs."""
            A = mat * (M1 + 0.5 * h * Eta)
            B = mat * (M1 - 0.5 * h * Eta)
            return np.linalg.solve(A, mv(B, v) + h * rhs_vec)

        def aux_update(v, drive, h):
            """(M1 + h/2 M_Sigma) v_new = (M1 - h/2 M_Sigma) v + h drive."""
            return np.linalg.solve(M1 + 0.5 * h * Sig, mv(M1 - 0.5 * h * Sig, v) + h * drive)

        x = x.copy()
        S = x.shape[1]
        e, hf = blk(x, 0).copy(), blk(x, 1).copy()
        p = blk(x, 2).copy() if a.nblk == 4 else np.zeros_like(e)
        q = blk(x, 3).copy() if a.nblk == 4 else np.zeros_like(e)

        def src(t):
            if not self.src:
                return 0.0
            return self.source_vector(t)[:nE].reshape(K, n3, S)

        def h_step(e_, h_, q_, h):
            curl = (Khe @ e_.reshape(nE, S)).reshape(K, n3, S)
            return field_update(h_, mu, curl - mv(M1aux, q_), h)

        def e_step(e_, h_, p_, t, h):
            curl = (Keh @ h_.reshape(nE, S)).reshape(K, n3, S)
            return field_update(e_, eps, curl - mv(M1aux, p_) + src(t), h)

        hf = h_step(e, hf, q, 0.5 * dt)
        p = aux_update(p, eps * mv(Xi, e), 0.5 * dt)
        t = t0
        for n in range(steps):
            q = aux_update(q, mu * mv(Xi, hf), dt)
            e = e_step(e, hf, p, t + 0.5 * dt, dt)
            p = aux_update(p, eps * mv(Xi, e), dt)
            hf = h_step(e, hf, q, dt)
            t += dt
            if callback is not None:
                out = np.concatenate([e.reshape(nE, S), hf.reshape(nE, S)] +
                                     ([p.reshape(nE, S), q.reshape(nE, S)] if a.nblk == 4 else []))
                callback(n + 1, t, out)
        parts = [e.reshape(nE, S), hf.reshape(nE, S)]
        if a.nblk == 4:
            parts += [p.reshape(nE, S), q.reshape(nE, S)]
        return np.concatenate(parts)

    # -- projection and sampling --------------------------------------------------
    def project(self, fn, field):
        """L2 projection of a vector function fn(r [n,3]) -> [n,3] onto field 'E' or 'H'.

        Returns coefficients (K, 3, N) solving M1 c = (fn, phi)_T per element.
        """
        a, m = self.asm, self.asm.mesh
        rq, wq = tet_quadrature(a.p + 4)
        out = np.empty((a.K, 3, a.N))
        for T in range(a.K):
            r = rq @ m.A[T].T + m.b[T][None, :]
            w = wq * abs(m.det[T])
            B = a._basis_vectors(T, r)
            rhs = np.einsum("q,qc,qci->i", w, fn(r), B)
            out[T] = np.linalg.solve(np.einsum("q,qci,qcj->ij", w, B, B), rhs).reshape(3, a.N)
        return out

    def evaluate(self, coef, T, r):
        """Field of element T with coefficients coef (3N,) at points r [n,3] -> [n,3]."""
        B = self.asm._basis_vectors(T, r)
        return np.einsum("qci,i->qc", B, coef)

    def l2_error(self, coef, fn, q=None):
        """L2 norm over the mesh of (field with coefficients coef (K,3,N)) - fn."""
        a, m = self.asm, self.asm.mesh
        rq, wq = tet_quadrature(q or a.p + 4)
        err = 0.0
        for T in range(a.K):
            r = rq @ m.A[T].T + m.b[T][None, :]
            w = wq * abs(m.det[T])
            v = self.evaluate(coef[T].reshape(-1), T, r) - fn(r)
            err += float(np.einsum("q,qc,qc->", w, v, v))
        return math.sqrt(err)
