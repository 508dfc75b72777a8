"""Pins of the oracle's symmetric interior penalty with a facet field
(Sec. III, Eqs. (jmp_var_def), (1st_weak_equation), (weak_penalty)).

* Eliminating h_s leaves the classic tangential-jump penalty: the facet
  coupling satisfies C_F M_F^-1 C_F^T = alpha sum_F (1/mu_F) (n x [[e]], n x [[phi]])_F,
  with the right side integrated here directly from both sides' basis
  functions (no facet basis involved); a wrong normal, tangent, side sign,
  facet mass or mu_F fails it.
* A globally continuous polynomial field of degree p has no tangential jump,
  so it drives no facet field.
* The extended system is skew: its energy, with the facet term, is conserved
  by LSRK4 to the method's dissipation (1e-7 over 50 steps here) while the
  facet field carries energy.
* What the penalty is for (the central flux's spurious modes): on a 3^3 PEC
  unit-cube cavity at p = 1 the central-flux spectrum has more than a hundred
  eigenvalues with 0.5 < omega < 5 where the cavity has only the three
  TM/TE-110 modes at pi sqrt(2); with alpha = 100 exactly three remain there,
  within 5 % of pi sqrt(2).
"""
import math

import numpy as np

import workloads as W
from oracle.assemble import Assembly
from oracle.basis import tri_quadrature
from oracle.mesh import Mesh
from oracle.sip import SipAssembly, SipSolver
from oracle.solver import Solver


def _case(p=2, seed=3):
    xyz, tets = W.kuhn_mesh(2, jitter=0.12, seed=seed)
    m = Mesh(xyz, tets)
    eps = W.lognormal_material(m.K, 2.0, 0.3, seed + 1)
    mu = W.lognormal_material(m.K, 1.0, 0.2, seed + 2)
    return m, Assembly(m, p, eps, mu, "central")


def test_eliminating_the_facet_field_gives_the_tangential_jump_penalty():
    m, a = _case()
    alpha = 3.7
    sa = SipAssembly(a, alpha)
    nE = a.K * a.n3
    J = np.zeros((nE, nE))
    st, wst = tri_quadrature(a.p + 2)
    for T in range(m.K):
        for f in range(4):
            Tp = m.nbr[T, f]
            if Tp <= T:
                continue
            P, opp = m.face_vertices(T, f)
            c = np.cross(P[1] - P[0], P[2] - P[0])
            n = c / np.linalg.norm(c)
            n = n if np.dot(n, P[0] - opp) > 0 else -n
            r = P[0] + st[:, :1] * (P[1] - P[0]) + st[:, 1:2] * (P[2] - P[0])
            w = wst * np.linalg.norm(c)
            jump = np.concatenate([np.cross(n[None, :, None], a._basis_vectors(T, r), axis=1),
                                   -np.cross(n[None, :, None], a._basis_vectors(Tp, r), axis=1)],
                                  axis=2)
            idx = np.concatenate([T * a.n3 + np.arange(a.n3), Tp * a.n3 + np.arange(a.n3)])
            J[np.ix_(idx, idx)] += np.einsum("q,qci,qcj->ij", w, jump, jump) / (0.5 * (a.mu[T] + a.mu[Tp]))
    CF = sa.C_F.toarray()
    lhs = CF @ (sa.minv_s[:, None] * CF.T)
    assert np.abs(lhs - alpha * J).max() <= 1e-12 * np.abs(alpha * J).max()


def test_continuous_fields_drive_no_facet_field():
    m, a = _case()
    sa = SipAssembly(a, 2.0)
    fe = lambda r: np.stack([r[:, 0] * r[:, 1], r[:, 2] ** 2 - r[:, 0], r[:, 1] * r[:, 2] + 1.0], axis=1)
    e = Solver(a).project(fe, "E").reshape(-1)            # degree 2 = p: reproduced exactly
    CF = sa.C_F.toarray()
    assert np.abs(CF.T @ e).max() <= 1e-12 * np.abs(CF).max() * np.abs(e).max()


def test_extended_energy_is_conserved():
    m, a = _case()
    ss = SipSolver(Solver(a), 3.7)
    x = ss.pack(W.random_state(a.K, 1, a.p, seed=9))
    E0 = ss.sip.energy(x)
    x1 = ss.lsrk4(x, 0.0, W.stable_dt(0.5, a.p) / 4, 50)
    nEH = 2 * a.K * a.n3
    facet = 0.5 * np.sum(x1[nEH:] ** 2 / ss.sip.minv_s[:, None])
    assert facet > 1e-3 * E0[0]                          # the facet field is active
    assert abs(ss.sip.energy(x1)[0] - E0[0]) <= 1e-6 * E0[0]


def test_penalty_removes_the_spurious_cavity_modes():
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=7)
    a = Assembly(Mesh(xyz, tets), 1, 1.0, 1.0, "central")

    def omegas(Kmat, minv):
        lam = np.linalg.eigvals(minv(Kmat.toarray()))
        w = np.sort(np.abs(lam.imag))
        return w[(w > 0.5) & (w < 5.0)]

    plain = omegas(a.Kmat, a.apply_minv)
    sa = SipAssembly(a, 100.0)
    pen = omegas(sa.Kmat, sa.apply_minv)
    assert len(plain) // 2 > 100
    assert len(pen) == 6                                  # three modes, each as a +-omega pair
    assert np.all(np.abs(pen - math.pi * math.sqrt(2.0)) < 0.05 * math.pi * math.sqrt(2.0))
