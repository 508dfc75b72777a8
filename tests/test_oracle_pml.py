"""Pins of the oracle's PML coupling (Sec. IV) against facts that do not come
from the oracle itself.

1. Algebra, one element.  The oracle's semi-discrete operator L = M^-1 K
   with the auxiliary unknowns p (E equation) and q (H equation) is
   eliminated in the Laplace domain (d/dt -> lambda, complex).  What remains
   of the E rows, multiplied by the E mass matrix, must be the mass matrix of
   the complex-stretched permittivity of Sec. IV (Eq. (cartesian_stretching)):
       lambda eps~_aa = eps (lambda + s_b)(lambda + s_c) / (lambda + s_a),
   the product form, not the partial fractions the oracle assembles.  The
   tensor mass matrix is integrated exactly in rational arithmetic over a
   tetrahedron with rational vertices (brute force, tests/exact_poly.py).
   A sign, scale or transpose slip in any of the four couplings
   E<-E (eta), E<-P, P<-P (Sigma), P<-E (xi), or in their H/Q twins, or a
   permutation of the three damping values, changes this matrix.
2. Energy: a pulse launched inside the PML box never puts more energy into
   the layer than it started with, and the total field energy never grows.
3. Absorption, on the oracle alone: with the layer the interior field is
   nearly gone once the pulse has crossed it; with sigma = 0 (the same PEC
   box, no absorption) most of the energy is still there.
"""
from fractions import Fraction
import functools
import math

import numpy as np
import pytest

import workloads as W
from exact_poly import Poly, dubiner_raw, inv3, modes
from oracle.assemble import Assembly, pml_sigma
from oracle.mesh import Mesh
from oracle.solver import Solver

F = Fraction
TET = [(F(0), F(0), F(0)), (F(7, 5), F(1, 7), F(-1, 9)), (F(1, 3), F(6, 5), F(1, 8)),
       (F(-1, 6), F(1, 4), F(9, 7))]
SIGMA = (3.0, 7.0, 11.5)          # three different damping values (a corner region)


def _exact_scalar_gram(p):
    """G[l][m] = int_T phi_l phi_m over the physical element, with phi_l the
    orthonormal reference function composed with the inverse element map,
    integrated exactly; plus the rows of A^-1 (the covariant directions)."""
    V = TET
    A = [[V[c + 1][r] - V[0][r] for c in range(3)] for r in range(3)]
    Ainv, det = inv3(A)
    x = [Poly.var(i) for i in range(3)]
    lin = [sum((Ainv[i][j] * (x[j] - V[0][j]) for j in range(3)), Poly()) for i in range(3)]
    fwd = [sum((A[i][j] * x[j] for j in range(3)), Poly()) + V[0][i] for i in range(3)]
    raws = [dubiner_raw(*m) for m in modes(p)]
    norms = [(r * r).int_tet() for r in raws]
    phys = [r.compose(lin) for r in raws]
    N = len(raws)
    G = np.zeros((N, N))
    for l in range(N):
        for m in range(l, N):
            val = abs(det) * (phys[l] * phys[m]).compose(fwd).int_tet()
            G[l, m] = G[m, l] = float(val) / math.sqrt(float(norms[l] * norms[m]))
    vj = np.array([[float(Ainv[j][c]) for c in range(3)] for j in range(3)])  # A^-T e_j
    return G, vj


def _tensor_mass(G, vj, d):
    """int phi_{j,l} . diag(d) phi_{k,m}: (v_j . diag(d) v_k) G_lm, index (j, l)."""
    D = (vj * d[None, :]) @ vj.T
    return np.kron(D, G)


@pytest.mark.parametrize("p", [1, 2])
def test_pml_coupling_eliminates_to_stretched_tensor(p):
    xyz = np.array([[float(c) for c in v] for v in TET])
    mesh = Mesh(xyz, np.array([[0, 1, 2, 3]]))
    eps, mu = 2.3, 0.7
    sig = np.array(SIGMA)
    asm = Assembly(mesh, p, eps, mu, "central", sigma=sig[None, :])
    n3 = asm.n3
    assert asm.nblk == 4
    # the oracle's operator L = M^-1 K, column by column
    L = asm.apply_minv(asm.Kmat.toarray())
    blk = lambda i, j: L[i * n3:(i + 1) * n3, j * n3:(j + 1) * n3]
    E, H, P, Q = 0, 1, 2, 3
    for a, b in ((E, Q), (H, P), (P, H), (Q, E), (P, Q), (Q, P)):
        assert np.abs(blk(a, b)).max() == 0.0
    G, vj = _exact_scalar_gram(p)
    M1 = _tensor_mass(G, vj, np.ones(3))
    assert np.allclose(asm.M1[0], M1, rtol=0, atol=1e-12 * np.abs(M1).max())
    rng = np.random.default_rng(5)
    for lam in [0.8 - 1.9j, 0.1 + 4.0j, 3.0 + 0.0j, -0.3 - 7.5j] + list(
            rng.uniform(-2, 2, 3) + 1j * rng.uniform(-9, 9, 3)):
        I = np.eye(n3)
        for fld, aux, mat in ((E, P, eps), (H, Q, mu)):
            schur = lam * I - blk(fld, fld) - blk(fld, aux) @ np.linalg.solve(
                lam * I - blk(aux, aux), blk(aux, fld))
            got = mat * M1 @ schur
            sa = sig
            sb = np.roll(sig, -1)
            sc = np.roll(sig, -2)
            d = mat * (lam + sb) * (lam + sc) / (lam + sa)
            want = _tensor_mass(G, vj, d)
            assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), (lam, fld)


@functools.lru_cache(maxsize=None)
def _pulse_run(sigma_max, T=2.0, n=4, p=2):
    """Divergence-free pulse E = (-y, x, 0) exp(-|r|^2 / 0.04) at the centre of
    [-1,1]^3 (PEC walls), PML 0.5 thick (a gradient field would not propagate
    and would stay in the interior whatever the layer does)."""
    xyz, tets = W.kuhn_mesh(n, (-1, -1, -1), (1, 1, 1))
    mesh = Mesh(xyz, tets)
    th = 0.5
    sig = pml_sigma(mesh.centroids(), (-1 + th,) * 3, (1 - th,) * 3, th, sigma_max, 2)
    asm = Assembly(mesh, p, 1.0, 1.0, "upwind", sigma=sig)
    s = Solver(asm)
    g = lambda r: np.exp(-(r ** 2).sum(1) / 0.04)
    ey = s.project(lambda r: np.stack([-r[:, 1] * g(r), r[:, 0] * g(r), 0 * g(r)], axis=1), "E")
    u = np.zeros((asm.K, 1, 6, asm.N))
    u[:, 0, 0:3, :] = ey
    x = s.pack(u, np.zeros_like(u))
    inpml = np.any(sig > 0, axis=1)
    dt = W.stable_dt(2.0 / n, p)
    steps = int(round(T / dt))

    def energies(x):
        e = x[:asm.K * asm.n3].reshape(asm.K, asm.n3)
        h = x[asm.K * asm.n3:2 * asm.K * asm.n3].reshape(asm.K, asm.n3)
        per = 0.5 * (np.einsum("ki,kij,kj->k", e, asm.M1, e) +
                     np.einsum("ki,kij,kj->k", h, asm.M1, h))
        return per.sum(), per[inpml].sum(), per[~inpml].sum()

    hist = [energies(x[:, 0])]
    s.lsrk4(x, 0.0, dt, steps, callback=lambda n_, t, xx: hist.append(energies(xx[:, 0])))
    return np.array(hist), int(inpml.sum()), asm.K


def test_pml_energy_never_exceeds_initial():
    hist, npml, K = _pulse_run(40.0)
    assert 0 < npml < K
    w0 = hist[0, 0]
    assert hist[0, 1] < 1e-4 * w0            # the pulse starts inside the box
    assert hist[:, 1].max() > 1e-1 * w0      # and does reach the layer
    assert np.all(hist[:, 1] <= w0)
    assert np.all(hist[:, 0] <= w0 * (1 + 1e-12))


def test_pml_absorbs_what_pec_walls_keep():
    with_pml, _, _ = _pulse_run(40.0)
    walls, _, _ = _pulse_run(0.0)
    w0 = with_pml[0, 0]
    assert walls[0, 0] == w0
    # interior energy once the pulse has crossed the layer and come back
    assert with_pml[-1, 2] < 2e-3 * w0
    assert walls[-1, 2] > 0.2 * w0
    assert with_pml[-1, 2] < 1e-2 * walls[-1, 2]
