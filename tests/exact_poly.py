"""Exact rational polynomial arithmetic for brute-force pins of the oracle.

Polynomials in (x, y, z) with fractions.Fraction coefficients, stored as
{(a, b, c): coeff}.  Used by tests only: the Dubiner functions of Sec. II are
expanded into monomials through the explicit finite-sum form of the Jacobi
polynomials (not the recurrence the oracle uses), composed exactly with
rational affine element maps, differentiated exactly, and integrated exactly
with  int_T x^a y^b z^c = a! b! c! / (a+b+c+3)!  on the reference
tetrahedron and  int s^a t^b = a! b! / (a+b+2)!  on the reference triangle.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial


class Poly:
    __slots__ = ("c",)

    def __init__(self, c=None):
        self.c = {k: v for k, v in (c or {}).items() if v != 0}

    @staticmethod
    def const(v):
        return Poly({(0, 0, 0): Fraction(v)})

    @staticmethod
    def var(i):
        e = [0, 0, 0]
        e[i] = 1
        return Poly({tuple(e): Fraction(1)})

    def __add__(self, o):
        if not isinstance(o, Poly):
            o = Poly.const(o)
        out = dict(self.c)
        for k, v in o.c.items():
            out[k] = out.get(k, 0) + v
        return Poly(out)

    __radd__ = __add__

    def __neg__(self):
        return Poly({k: -v for k, v in self.c.items()})

    def __sub__(self, o):
        return self + (-o if isinstance(o, Poly) else Poly.const(-Fraction(o)))

    def __rsub__(self, o):
        return Poly.const(o) - self

    def __mul__(self, o):
        if not isinstance(o, Poly):
            o = Fraction(o)
            return Poly({k: v * o for k, v in self.c.items()})
        out = {}
        for k1, v1 in self.c.items():
            for k2, v2 in o.c.items():
                k = (k1[0] + k2[0], k1[1] + k2[1], k1[2] + k2[2])
                out[k] = out.get(k, 0) + v1 * v2
        return Poly(out)

    __rmul__ = __mul__

    def __pow__(self, n):
        out = Poly.const(1)
        for _ in range(n):
            out = out * self
        return out

    def diff(self, i):
        out = {}
        for k, v in self.c.items():
            if k[i] == 0:
                continue
            e = list(k)
            e[i] -= 1
            out[tuple(e)] = out.get(tuple(e), 0) + v * k[i]
        return Poly(out)

    def compose(self, lin):
        """Substitute x_i -> lin[i] (three Polys)."""
        out = Poly()
        cache = {}
        for k, v in self.c.items():
            term = Poly.const(v)
            for i in range(3):
                if k[i]:
                    key = (i, k[i])
                    if key not in cache:
                        cache[key] = lin[i] ** k[i]
                    term = term * cache[key]
            out = out + term
        return out

    def int_tet(self):
        """Exact integral over the reference tetrahedron."""
        s = Fraction(0)
        for (a, b, c), v in self.c.items():
            s += v * Fraction(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))
        return s

    def int_tri(self):
        """Exact integral over the reference triangle in the first two variables
        (the third must not appear)."""
        s = Fraction(0)
        for (a, b, c), v in self.c.items():
            assert c == 0
            s += v * Fraction(factorial(a) * factorial(b), factorial(a + b + 2))
        return s


def jacobi_scaled(n, alpha, y, w):
    """w^n P_n^(alpha,0)(2y/w - 1) as a polynomial in y, w, by the finite sum
    P_n^(a,b)(t) = sum_s C(n+a, n-s) C(n+b, s) ((t-1)/2)^s ((t+1)/2)^(n-s)."""
    out = Poly()
    for s in range(n + 1):
        out = out + comb(n + alpha, n - s) * comb(n, s) * (y - w) ** s * y ** (n - s)
    return out


def dubiner_raw(i, j, k):
    """Unnormalised collapsed Dubiner function phi_ijk as an exact polynomial."""
    x, y, z = Poly.var(0), Poly.var(1), Poly.var(2)
    one = Poly.const(1)
    return (jacobi_scaled(i, 0, z, one - x - y)
            * jacobi_scaled(j, 2 * i + 1, y, one - x)
            * jacobi_scaled(k, 2 * i + 2 * j + 2, x, one))


def modes(p):
    return [(i, j, n - i - j) for n in range(p + 1) for i in range(n + 1) for j in range(n - i + 1)]


def inv3(M):
    """Exact inverse of a 3x3 Fraction matrix (list of lists)."""
    a, b, c = M[0]
    d, e, f = M[1]
    g, h, i = M[2]
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [[e * i - f * h, c * h - b * i, b * f - c * e],
           [f * g - d * i, a * i - c * g, c * d - a * f],
           [d * h - e * g, b * g - a * h, a * e - b * d]]
    return [[adj[r][s] / det for s in range(3)] for r in range(3)], det
