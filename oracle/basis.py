"""Reference-element basis and quadrature of the oracle (test infrastructure only).

Follows Sec. II of Kapidani & Schoeberl: the modal basis on the reference
tetrahedron T = {x, y, z >= 0, x + y + z <= 1} built from Jacobi polynomials
in collapsed (Duffy) coordinates, Eq. (dubiner_functions), normalised so that
it is orthonormal in L2(T), Eq. (ortho_cond).

Reading of the printed formula (it is garbled): the standard collapsed form
  phi_ijk = P_i^(0,0)(2z/(1-x-y) - 1) (1-x-y)^i
          * P_j^(2i+1,0)(2y/(1-x) - 1) (1-x)^j
          * P_k^(2i+2j+2,0)(2x - 1),
which is a polynomial of total degree i+j+k and orthogonal; the printed one
lacks the (1-x)^j factor and uses (2i+1,0) in the last factor, which is not
orthogonal.  Normalisation is numerical (quadrature), sign positive.

Mode order: graded by total degree n = i+j+k, then by i, then by j.

Gradients are taken by complex-step differentiation of the same formula, so
no separate derivative formula needs checking.
"""
from __future__ import annotations

import numpy as np


def jacobi(n: int, alpha: float, beta: float, w):
    """Jacobi polynomial P_n^(alpha,beta)(w) by the classical three-term recurrence.

    Works for real or complex arrays w.  Normalisation P_n(1) = binom(n+alpha, n).
    """
    w = np.asarray(w)
    p0 = np.ones_like(w)
    if n == 0:
        return p0
    p1 = 0.5 * ((alpha + beta + 2.0) * w + (alpha - beta))
    for m in range(2, n + 1):
        a = alpha + beta
        c1 = 2.0 * m * (m + a) * (2.0 * m + a - 2.0)
        c2 = (2.0 * m + a - 1.0) * (alpha * alpha - beta * beta)
        c3 = (2.0 * m + a - 2.0) * (2.0 * m + a - 1.0) * (2.0 * m + a)
        c4 = 2.0 * (m + alpha - 1.0) * (m + beta - 1.0) * (2.0 * m + a)
        p0, p1 = p1, ((c2 + c3 * w) * p1 - c4 * p0) / c1
    return p1


def modes(p: int):
    """List of (i, j, k) with i+j+k <= p in graded order (degree, then i, then j)."""
    out = []
    for n in range(p + 1):
        for i in range(n + 1):
            for j in range(n - i + 1):
                out.append((i, j, n - i - j))
    return out


def degrees(p: int):
    return np.array([sum(m) for m in modes(p)])


def _phi_raw(i, j, k, x, y, z):
    """Unnormalised collapsed-coordinate Dubiner function (see module docstring)."""
    s1 = 1.0 - x - y
    s2 = 1.0 - x
    a = 2.0 * z / s1 - 1.0
    b = 2.0 * y / s2 - 1.0
    c = 2.0 * x - 1.0
    return (jacobi(i, 0.0, 0.0, a) * s1 ** i
            * jacobi(j, 2.0 * i + 1.0, 0.0, b) * s2 ** j
            * jacobi(k, 2.0 * i + 2.0 * j + 2.0, 0.0, c))


def tet_quadrature(q: int):
    """Collapsed Gauss-Legendre rule on the reference tetrahedron.

    q points per collapsed direction; exact for polynomials of total degree
    <= 2q - 3.  Returns (points [q^3, 3], weights [q^3]).
    """
    g, wg = np.polynomial.legendre.leggauss(q)
    A, B, C = np.meshgrid(g, g, g, indexing="ij")
    WA, WB, WC = np.meshgrid(wg, wg, wg, indexing="ij")
    x = 0.5 * (1.0 + C)
    y = 0.5 * (1.0 + B) * (1.0 - x)
    z = 0.5 * (1.0 + A) * (1.0 - x - y)
    jac = (1.0 - x) * (1.0 - x - y) / 8.0
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return pts, (WA * WB * WC * jac).ravel()


def tri_quadrature(q: int):
    """Collapsed Gauss-Legendre rule on the reference triangle {s,t>=0, s+t<=1}.

    Exact for total degree <= 2q - 2.  Returns (points [q^2, 2], weights [q^2]).
    """
    g, wg = np.polynomial.legendre.leggauss(q)
    A, B = np.meshgrid(g, g, indexing="ij")
    WA, WB = np.meshgrid(wg, wg, indexing="ij")
    s = 0.5 * (1.0 + B)
    t = 0.5 * (1.0 + A) * (1.0 - s)
    jac = (1.0 - s) / 4.0
    return np.stack([s.ravel(), t.ravel()], axis=1), (WA * WB * jac).ravel()


class RefBasis:
    """Orthonormal Dubiner basis of degree p on the reference tetrahedron."""

    def __init__(self, p: int):
        self.p = p
        self.modes = modes(p)
        self.N = len(self.modes)
        pts, w = tet_quadrature(p + 3)
        raw = self._raw(pts)
        # numerical normalisation, Eq. (ortho_cond)
        self.scale = 1.0 / np.sqrt((raw ** 2 * w[:, None]).sum(axis=0))

    def _raw(self, pts):
        x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
        return np.stack([_phi_raw(i, j, k, x, y, z) for (i, j, k) in self.modes], axis=1)

    def values(self, pts):
        """phi_l at reference points [n, 3] -> [n, N]."""
        return self._raw(np.asarray(pts, dtype=np.float64)) * self.scale[None, :]

    def gradients(self, pts):
        """Reference gradients of phi_l at points [n, 3] -> [n, N, 3] (complex step)."""
        pts = np.asarray(pts, dtype=np.float64)
        hstep = 1e-30
        out = np.empty((pts.shape[0], self.N, 3))
        for a in range(3):
            zp = pts.astype(np.complex128)
            zp[:, a] += 1j * hstep
            out[:, :, a] = (self._raw(zp).imag / hstep) * self.scale[None, :]
        return out
