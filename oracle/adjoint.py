"""Discrete adjoint of the oracle's LSRK4 stepping (test infrastructure only).

The one-step map of the low-storage RK4 scheme (Carpenter & Kennedy) is
affine in the state; its adjoint is obtained by transposing the assembled
operator explicitly.  Stage k: r_k = a_k r_{k-1} + dt F(u_{k-1}, t_k),
u_k = u_{k-1} + b_k r_k, with F(u, t) = M^-1 (K u + f(t)).  Reverse:
  lr += b_k lu;  lu += dt F_u^T lr;  grad += dt (dF/dtheta)^T lr;  lr *= a_k
with F_u^T = K^T M^-T.  dF/dtheta for theta = eps_T or mu_T is taken by a
complex step on the element-local reassembly of the rows that depend on the
element's material (its own and its face neighbours'), which makes it exact
to rounding.

Receivers: E(r) = sum_{j,l} u_{T,j,l} phi_{j,l}(r) (Eq. (mapped_eh)) in the
lowest-index element containing r; the loss gradient with respect to the
records is injected through the transpose of that evaluation.
"""
from __future__ import annotations

import numpy as np

from .assemble import Assembly
from .solver import LSRK4_A, LSRK4_B, LSRK4_C, Solver


class Receivers:
    def __init__(self, asm, positions):
        self.asm = asm
        self.items = []
        for r in np.asarray(positions, dtype=np.float64):
            T = asm.mesh.locate(r)
            B = asm._basis_vectors(T, r[None, :])[0]     # [3, 3N]
            self.items.append((T, B))

    def sample(self, x):
        """x [ndof, S] -> E at the receivers [S, R, 3]."""
        a = self.asm
        out = np.zeros((x.shape[1], len(self.items), 3))
        for r, (T, B) in enumerate(self.items):
            out[:, r, :] = (B @ x[T * a.n3:(T + 1) * a.n3, :]).T
        return out

    def inject(self, g, shape):
        """Transpose of sample: g [S, R, 3] -> vector [ndof, S]."""
        a = self.asm
        v = np.zeros(shape)
        for r, (T, B) in enumerate(self.items):
            v[T * a.n3:(T + 1) * a.n3, :] += B.T @ g[:, r, :].T
        return v


def forward(solver, x0, t0, dt, steps, rec):
    """LSRK4 from x0; returns (final state, stage inputs per step, records [steps, S, R, 3])."""
    x = x0.copy()
    res = np.zeros_like(x)
    stages, records = [], []
    t = t0
    for n in range(steps):
        ins = []
        for k in range(5):
            ins.append(x.copy())
            res = LSRK4_A[k] * res + dt * solver.rhs(x, t + LSRK4_C[k] * dt)
            x = x + LSRK4_B[k] * res
        stages.append(ins)
        records.append(rec.sample(x))
        t += dt
    return x, stages, np.array(records)


def apply_transpose(solver, v):
    """F_u^T v = K^T (M^-1)^T v (assembled operator, explicitly transposed)."""
    a = solver.asm
    R, n3 = a.R, a.n3
    w = np.empty_like(v)
    for bi in range(a.nblk):
        blk = v[bi * R * n3:(bi + 1) * R * n3].reshape(R, n3, -1)
        w[bi * R * n3:(bi + 1) * R * n3] = np.einsum("kji,kjs->kis", a.Minv[bi], blk).reshape(R * n3, -1)
    return a.Kmat.T @ w


class MaterialDerivative:
    """dF/dtheta_T u for theta in {eps, mu}, by complex step on the reassembled rows."""

    def __init__(self, mesh, p, eps, mu, flux, sigma, S, sources, which, T, h=1e-20):
        K = mesh.K
        nb = [int(n) for n in mesh.nbr[T] if n >= 0]
        self.rows = np.array(sorted(set([T] + nb)))
        eps_c = np.asarray(eps, dtype=np.complex128) * np.ones(K)
        mu_c = np.asarray(mu, dtype=np.complex128) * np.ones(K)
        scale = (eps_c if which == "eps" else mu_c)[T].real
        self.h = h * scale
        if which == "eps":
            eps_c[T] += 1j * self.h
        else:
            mu_c[T] += 1j * self.h
        asm = Assembly(mesh, p, eps_c, mu_c, flux, sigma=sigma, rows=self.rows)
        self.solver = Solver(asm, S=S, sources=sources)
        a = asm
        self.idx = np.concatenate([(b * K + self.rows)[:, None] * a.n3 + np.arange(a.n3)[None, :]
                                   for b in range(a.nblk)]).ravel()

    def dot(self, lr, x, t):
        """sum over rows of lr . (dF/dtheta_T x) at time t."""
        dF = self.solver.rhs(x.astype(np.complex128), t).imag / self.h
        return float(np.sum(lr[self.idx] * dF))


def gradient(mesh, p, eps, mu, flux, sigma, S, sources, x0, t0, dt, steps, rec_pos, drec_fn,
             elements=None, which=("eps", "mu")):
    """Discrete-adjoint gradient of a loss of the receiver records.

    drec_fn(records [steps, S, R, 3]) -> dL/drecords (same shape).
    Returns dict which -> array over `elements` (default: all)."""
    asm = Assembly(mesh, p, eps, mu, flux, sigma=sigma)
    solver = Solver(asm, S=S, sources=sources)
    rec = Receivers(asm, rec_pos)
    _, stages, records = forward(solver, x0, t0, dt, steps, rec)
    drec = drec_fn(records)
    elements = np.arange(mesh.K) if elements is None else np.asarray(elements)
    derivs = {w: [MaterialDerivative(mesh, p, eps, mu, flux, sigma, S, sources, w, int(T))
                  for T in elements] for w in which}
    grads = {w: np.zeros(len(elements)) for w in which}
    lam = np.zeros_like(x0)
    for n in reversed(range(steps)):
        lam = lam + rec.inject(drec[n], lam.shape)
        lu, lr = lam, np.zeros_like(lam)
        t = t0 + n * dt
        for k in reversed(range(5)):
            lr = lr + LSRK4_B[k] * lu
            xk, tk = stages[n][k], t + LSRK4_C[k] * dt
            for w in which:
                for i, d in enumerate(derivs[w]):
                    grads[w][i] += dt * d.dot(lr, xk, tk)
            lu = lu + dt * apply_transpose(solver, lr)
            lr = LSRK4_A[k] * lr
        lam = lu
    return grads, records


def loss_records(mesh, p, eps, mu, flux, sigma, S, sources, x0, t0, dt, steps, rec_pos):
    asm = Assembly(mesh, p, eps, mu, flux, sigma=sigma)
    solver = Solver(asm, S=S, sources=sources)
    rec = Receivers(asm, rec_pos)
    return forward(solver, x0, t0, dt, steps, rec)[2]
