"""Pins of the mixed-order oracle (E of degree pE, H of degree pH; Sec. III,
Eqs. (triale)/(trialh)) against facts that do not come from it.

* pE = pH: the operator and mass inverses equal the single-degree oracle's
  (itself pinned by exact brute force, P2-P7).
* Exact brute force with rectangular blocks: mass, volume curl and the face
  couplings between the two spaces on two tetrahedra with rational vertices,
  with the basis expanded into monomials in physical coordinates.
* Central flux + PEC: the operator is skew (K_HE = -K_EH^T, no E-E or H-H
  blocks), so the discrete energy is conserved; upwind: negative
  semidefinite symmetric part.
* The TM110 cavity mode: E converges under upwind LSRK4 at order pH + 1, the
  lower of the two degrees (measured 1.91 from 2^3 to 4^3 and 2.14 from 4^3
  to 8^3 for pE = 2, pH = 1; equal degrees 2 give 2.98 and 2.88).
"""
import math

import numpy as np
import pytest

import workloads as W
from exact_poly import Poly
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.mixed import MixedAssembly, MixedSolver
from test_oracle_exact import (TETS, VERTS, _cross, _curl, _element_polys, _face_map,
                               _vector_basis, _vol_int)


@pytest.mark.parametrize("p,flux", [(1, "upwind"), (2, "central")])
def test_equal_degrees_are_the_single_degree_oracle(p, flux):
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=11)
    m = Mesh(xyz, tets)
    eps = W.lognormal_material(m.K, 2.0, 0.3, 12)
    a = Assembly(m, p, eps, 1.3, flux)
    b = MixedAssembly(m, p, p, eps, 1.3, flux)
    d = (a.Kmat - b.Kmat).toarray()
    assert np.abs(d).max() <= 1e-13 * abs(a.Kmat).max()
    assert np.allclose(b.MinvE, a.Minv[0], rtol=1e-12, atol=0)
    assert np.allclose(b.MinvH, a.Minv[1], rtol=1e-12, atol=0)


def test_rectangular_blocks_exact():
    pE, pH = 2, 1
    xyz = np.array([[float(c) for c in v] for v in VERTS])
    mesh = Mesh(xyz, np.array(TETS))
    asm = MixedAssembly(mesh, pE, pH, 1.0, 1.0, "central")
    sv = sorted(TETS[0])
    elE, elH = _element_polys(sv, pE), _element_polys(sv, pH)
    nbE, nbH = _element_polys(sorted(TETS[1]), pE), _element_polys(sorted(TETS[1]), pH)
    basE, basH = _vector_basis(elE), _vector_basis(elH)
    NE, NH = asm.NE, asm.NH
    sc = lambda el, N: np.array([1.0 / math.sqrt(el["norms"][l]) for j in range(3) for l in range(N)])
    sE, sH = sc(elE, NE), sc(elH, NH)
    # volume: M_E, M_H, C_eh[i, j] = int curl phi^E_i . phi^H_j
    ME = np.array([[float(sum(vi[c] * vj[c] for c in range(3)) * _vol_int(elE, fi * fj))
                    for fj, vj in basE] for fi, vi in basE]) * np.outer(sE, sE)
    MH = np.array([[float(sum(vi[c] * vj[c] for c in range(3)) * _vol_int(elH, fi * fj))
                    for fj, vj in basH] for fi, vi in basH]) * np.outer(sH, sH)
    curls = [_curl(f, v) for f, v in basE]
    C = np.array([[float(_vol_int(elE, sum((curls[i][c] * (vj[c] * fj) for c in range(3)), Poly())))
                   for fj, vj in basH] for i in range(len(basE))]) * np.outer(sE, sH)
    for got, want in ((asm.ME[0], ME), (asm.MH[0], MH), (asm.C_eh[0], C)):
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # the shared face: int_F phi^a_i . (n x phi^b_j) for (a, b) = (E, H), (H, E), own and nbr
    f = sv.index(0)
    ent = [e for e in asm.face if e["T"] == 0 and e["f"] == f][0]
    assert ent["nb"] == 1
    Q = [VERTS[v] for v in sv if v != 0]
    nt = _cross([Q[1][i] - Q[0][i] for i in range(3)], [Q[2][i] - Q[0][i] for i in range(3)])
    if sum(nt[i] * (Q[0][i] - VERTS[0][i]) for i in range(3)) < 0:
        nt = [-c for c in nt]
    fm = _face_map(Q)
    onF = lambda bas: [(fi.compose(fm), vi) for fi, vi in bas]

    def block(test, trial, s_test, s_trial):
        out = np.zeros((len(test), len(trial)))
        for j, (fj, vj) in enumerate(trial):
            w = _cross(nt, vj)
            for i, (fi, vi) in enumerate(test):
                out[i, j] = float(sum(vi[c] * w[c] for c in range(3)) * (fi * fj).int_tri())
        return out * np.outer(s_test, s_trial)

    cases = [(("x", "E", "H", "own"), block(onF(basE), onF(basH), sE, sH)),
             (("x", "H", "E", "own"), block(onF(basH), onF(basE), sH, sE)),
             (("x", "E", "H", "nbr"), block(onF(basE), onF(_vector_basis(nbH)), sE, sc(nbH, NH))),
             (("x", "H", "E", "nbr"), block(onF(basH), onF(_vector_basis(nbE)), sH, sc(nbE, NE)))]
    for key, want in cases:
        assert np.abs(ent[key] - want).max() <= 1e-12 * np.abs(want).max(), key


def test_central_flux_is_skew_and_upwind_dissipates():
    xyz, tets = W.kuhn_mesh(2, jitter=0.12, seed=13)
    m = Mesh(xyz, tets)
    eps = W.lognormal_material(m.K, 2.0, 0.3, 14)
    mu = W.lognormal_material(m.K, 1.0, 0.2, 15)
    c = MixedAssembly(m, 2, 1, eps, mu, "central")
    K = c.Kmat.toarray()
    nE = m.K * c.nE
    assert np.abs(K[:nE, :nE]).max() == 0 and np.abs(K[nE:, nE:]).max() == 0
    assert np.abs(K[nE:, :nE] + K[:nE, nE:].T).max() <= 1e-13 * np.abs(K).max()
    u = MixedAssembly(m, 2, 1, eps, mu, "upwind").Kmat.toarray()
    ev = np.linalg.eigvalsh(0.5 * (u + u.T))
    assert ev.max() <= 1e-12 * np.abs(u).max() and ev.min() < -1e-3


def test_tm110_converges_at_the_lower_order():
    om = math.pi * math.sqrt(2.0)
    T = 0.5
    ez = lambda t: (lambda r: np.stack([0 * r[:, 0], 0 * r[:, 0],
                                        np.sin(math.pi * r[:, 0]) * np.sin(math.pi * r[:, 1])
                                        * math.cos(om * t)], axis=1))
    errs = []
    for n in (2, 4):
        xyz, tets = W.kuhn_mesh(n)
        a = MixedAssembly(Mesh(xyz, tets), 2, 1, 1.0, 1.0, "upwind")
        s = MixedSolver(a)
        u = np.zeros((a.K, 1, 6, a.NE))
        u[:, 0, 0:3] = s.project(ez(0.0), "E")
        dt = W.stable_dt(1.0 / n, 2) / 2
        steps = int(round(T / dt))
        x = s.lsrk4(s.pack(u), 0.0, T / steps, steps)
        coef = s.unpack(x)[:, 0, 0:3]
        ref = s.project(ez(T), "E")
        errs.append(np.linalg.norm(coef - ref) / np.linalg.norm(ref))
    rate = math.log2(errs[0] / errs[1])
    assert rate > 1.7, (errs, rate)     # order pH + 1 = 2
