"""Brute-force exact pins of the oracle's element and face matrices.

Two tetrahedra with rational vertices share one face.  Every basis function
of Sec. II (Eq. (dubiner_functions), standard collapsed exponents, Eq.
(mapped_eh) covariant map) is expanded into monomials in *physical*
coordinates with exact rational arithmetic, its curl is taken by exact
differentiation, and mass, volume-curl and face-coupling integrals are
computed exactly.  The oracle's quadrature values must agree to 1e-12.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from exact_poly import Poly, dubiner_raw, inv3, modes
from oracle.assemble import Assembly
from oracle.mesh import Mesh

F = Fraction
VERTS = [
    (F(0), F(0), F(0)),
    (F(7, 5), F(1, 7), F(-1, 9)),
    (F(1, 3), F(6, 5), F(1, 8)),
    (F(-1, 6), F(1, 4), F(9, 7)),
    (F(11, 8), F(13, 10), F(10, 9)),
]
TETS = [[0, 1, 2, 3], [1, 2, 3, 4]]          # share the face {1, 2, 3}


def _element_polys(vids, p):
    """Exact physical-coordinate data of one element (vertex ids ascending)."""
    V = [VERTS[i] for i in vids]
    A = [[V[c + 1][r] - V[0][r] for c in range(3)] for r in range(3)]
    Ainv, det = inv3(A)
    x = [Poly.var(i) for i in range(3)]
    lin = [sum((Ainv[i][j] * (x[j] - V[0][j]) for j in range(3)), Poly()) for i in range(3)]
    fwd = [sum((A[i][j] * x[j] for j in range(3)), Poly()) + V[0][i] for i in range(3)]
    raws = [dubiner_raw(*m) for m in modes(p)]
    norms = [(r * r).int_tet() for r in raws]
    phys = [r.compose(lin) for r in raws]                  # phihat_l(A^-1 (r - b))
    vj = [[Ainv[j][c] for c in range(3)] for j in range(3)]  # A^-T e_j
    return dict(V=V, A=A, det=det, fwd=fwd, phys=phys, norms=norms, vj=vj)


def _vector_basis(el):
    """List over (j, l) of (scalar poly, constant direction) pairs."""
    return [(el["phys"][l], el["vj"][j]) for j in range(3) for l in range(len(el["phys"]))]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _curl(f, v):
    """curl (f v) = grad f x v for constant v: three polys."""
    g = [f.diff(i) for i in range(3)]
    return [g[1] * v[2] - g[2] * v[1], g[2] * v[0] - g[0] * v[2], g[0] * v[1] - g[1] * v[0]]


def _vol_int(el, poly):
    return abs(el["det"]) * poly.compose(el["fwd"]).int_tet()


def _face_map(Q):
    s, t = Poly.var(0), Poly.var(1)
    return [Q[0][i] + s * (Q[1][i] - Q[0][i]) + t * (Q[2][i] - Q[0][i]) for i in range(3)]


@pytest.mark.parametrize("p", [1, 2])
def test_element_and_face_matrices_exact(p):
    xyz = np.array([[float(c) for c in v] for v in VERTS])
    mesh = Mesh(xyz, np.array(TETS))
    asm = Assembly(mesh, p, 1.0, 1.0, "central")
    N = asm.N
    el = _element_polys(sorted(TETS[0]), p)
    nb = _element_polys(sorted(TETS[1]), p)
    basis = _vector_basis(el)
    scale = np.array([1.0 / math.sqrt(el["norms"][l]) for j in range(3) for l in range(N)])

    # mass and volume curl (C_eh[i, j] = int curl phi_i . phi_j)
    M = np.zeros((3 * N, 3 * N))
    C = np.zeros((3 * N, 3 * N))
    curls = [_curl(f, v) for f, v in basis]
    for i, (fi, vi) in enumerate(basis):
        for j, (fj, vj) in enumerate(basis):
            dot_v = sum(vi[c] * vj[c] for c in range(3))
            M[i, j] = float(dot_v * _vol_int(el, fi * fj))
            C[i, j] = float(_vol_int(el, sum((curls[i][c] * (vj[c] * fj) for c in range(3)),
                                                 Poly())))
    S = np.outer(scale, scale)
    assert np.allclose(asm.M1[0], M * S, rtol=0, atol=1e-12 * np.abs(M * S).max())
    assert np.allclose(asm.C_eh[0], C * S, rtol=0, atol=1e-12 * np.abs(C * S).max())

    # the shared face: vertices of TETS[0] minus its opposite vertex 0
    sv = sorted(TETS[0])
    f = sv.index(0)
    ent = [e for e in asm.face if e["T"] == 0 and e["f"] == f][0]
    assert ent["nb"] == 1
    Q = [VERTS[v] for v in sv if v != 0]
    nt = _cross([Q[1][i] - Q[0][i] for i in range(3)], [Q[2][i] - Q[0][i] for i in range(3)])
    if sum(nt[i] * (Q[0][i] - VERTS[0][i]) for i in range(3)) < 0:
        nt = [-c for c in nt]
    fm = _face_map(Q)
    own_r = [(fi.compose(fm), vi) for fi, vi in basis]
    nbr_r = [(fi.compose(fm), vi) for fi, vi in _vector_basis(nb)]
    scale_nb = np.array([1.0 / math.sqrt(nb["norms"][l]) for j in range(3) for l in range(N)])

    def face_block(trial, twice):
        out = np.zeros((3 * N, 3 * N))
        for j, (fj, vj) in enumerate(trial):
            w = _cross(nt, vj)
            if twice:
                # n x (n x v) with n = nt/|nt|: (nt (nt.v) - v |nt|^2)/|nt|^2; the
                # 1/|nt| of the second factor is applied below
                w = _cross(nt, w)
            for i, (fi, vi) in enumerate(own_r):
                dot = sum(vi[c] * w[c] for c in range(3))
                out[i, j] = float(dot * (fi * fj).int_tri())
        return out

    nn = math.sqrt(float(sum(c * c for c in nt)))
    # int_F phi_i . (n x phi_j) dS = int_ref phi_i . (nt x phi_j) ds dt
    x_own = face_block(own_r, False) * np.outer(scale, scale)
    x_nbr = face_block(nbr_r, False) * np.outer(scale, scale_nb)
    xx_own = face_block(own_r, True) * np.outer(scale, scale) / nn
    xx_nbr = face_block(nbr_r, True) * np.outer(scale, scale_nb) / nn
    for got, want in ((ent["x_own"], x_own), (ent["x_nbr"], x_nbr),
                      (ent["xx_own"], xx_own), (ent["xx_nbr"], xx_nbr)):
        assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_exact_basis_is_orthogonal():
    """The corrected exponents give exactly orthogonal functions (Eq. (ortho_cond))."""
    raws = [dubiner_raw(*m) for m in modes(3)]
    for a in range(len(raws)):
        for b in range(a + 1, len(raws)):
            assert (raws[a] * raws[b]).int_tet() == 0


def test_printed_exponents_are_not_orthogonal():
    """The formula as printed (no (1-x)^j, last index 2i+1) is not orthogonal."""
    from exact_poly import jacobi_scaled
    x, y, z = Poly.var(0), Poly.var(1), Poly.var(2)
    one = Poly.const(1)

    def printed(i, j, k):
        # P_j^(2i+1,0)(2y/(1-x)-1) without the (1-x)^j factor is not a polynomial
        # for j > 0; test on modes with j = 0, where the only change is the index
        return (jacobi_scaled(i, 0, z, one - x - y) * jacobi_scaled(k, 2 * i + 1, x, one))

    ms = [(i, 0, k) for i in range(3) for k in range(3) if i + k <= 2]
    raws = [printed(*m) for m in ms]
    off = [(raws[a] * raws[b]).int_tet() for a in range(len(ms)) for b in range(a + 1, len(ms))]
    assert any(v != 0 for v in off)
