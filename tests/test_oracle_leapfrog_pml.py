"""Pins of the oracle's leapfrog with trapezoid-treated PML terms (Sec. V)
against facts that do not come from the scheme itself.

* With sigma = 0 it is the plain staggered leapfrog.
* It converges at second order in time to the exact solution of the
  semi-discrete PML system, exp(T L) x0 with L = M^-1 K the oracle's
  assembled operator (the LSRK4 path's operator, Sec. IV), computed by a
  dense matrix exponential on a small mesh: a sign or coupling slip in any
  of the four PML updates converges to something else or not at all.
* The layer absorbs: with central flux (no numerical dissipation) the
  interior keeps most of a pulse's energy between PEC walls and loses it
  with the PML.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle.assemble import Assembly, pml_sigma
from oracle.mesh import Mesh
from oracle.solver import Solver


def _setup(n, p, sigma_max, th=0.5, seed=3, jitter=0.1):
    xyz, tets = W.kuhn_mesh(n, (-1, -1, -1), (1, 1, 1), jitter=jitter, seed=seed)
    m = Mesh(xyz, tets)
    sig = pml_sigma(m.centroids(), (-1 + th,) * 3, (1 - th,) * 3, th, sigma_max, 2)
    eps = W.lognormal_material(m.K, 1.5, 0.2, seed + 1)
    return m, sig, eps


def test_zero_sigma_is_plain_leapfrog():
    m, sig, eps = _setup(2, 2, 0.0)
    a0 = Assembly(m, 2, eps, 1.3, "central")
    a1 = Assembly(m, 2, eps, 1.3, "central", sigma=np.zeros((m.K, 3)))
    s0, s1 = Solver(a0, S=2), Solver(a1, S=2)
    u = W.random_state(m.K, 2, 2, seed=4)
    dt = W.stable_dt(1.0, 2)
    x0 = s0.leapfrog(s0.pack(u), 0.0, dt, 30)
    x1 = s1.leapfrog_pml(s1.pack(u, np.zeros_like(u)), 0.0, dt, 30)
    nF = 2 * m.K * a0.n3
    assert np.abs(x1[:nF] - x0).max() < 1e-12 * np.abs(x0).max()
    assert np.all(x1[nF:] == 0.0)


def test_second_order_in_time_to_the_semidiscrete_solution():
    m, sig, eps = _setup(2, 1, 10.0)
    assert np.any(sig > 0) and np.any(np.all(sig == 0, axis=1))
    a = Assembly(m, 1, eps, 1.0, "central", sigma=sig)
    s = Solver(a, S=1)
    u = W.random_state(m.K, 1, 1, seed=5)
    aux = W.random_state(m.K, 1, 1, seed=6) * 0.3
    x0 = s.pack(u, aux)
    L = a.apply_minv(a.Kmat.toarray())
    T = 0.24
    nE = m.K * a.n3
    errs = []
    for steps in (24, 48, 96):
        dt = T / steps
        x = s.leapfrog_pml(x0, 0.0, dt, steps)
        # e and q are at T; h and p half a step later
        ex_T = expm(T * L) @ x0
        ex_h = expm((T + 0.5 * dt) * L) @ x0
        err = max(np.abs(x[:nE] - ex_T[:nE]).max(),
                  np.abs(x[3 * nE:] - ex_T[3 * nE:]).max(),
                  np.abs(x[nE:3 * nE] - ex_h[nE:3 * nE]).max())
        errs.append(err / np.abs(ex_T).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[-1] < 1e-3


def _interior_energy(sigma_max, n=4, p=2, T=2.0):
    m, sig, _ = _setup(n, p, sigma_max, jitter=0.0)
    a = Assembly(m, p, 1.0, 1.0, "central", sigma=sig)
    s = Solver(a)
    g = lambda r: np.exp(-(r ** 2).sum(1) / 0.04)
    ee = s.project(lambda r: np.stack([-r[:, 1] * g(r), r[:, 0] * g(r), 0 * g(r)], axis=1), "E")
    u = np.zeros((m.K, 1, 6, a.N))
    u[:, 0, 0:3] = ee
    inside = ~np.any(sig > 0, axis=1)
    dt = W.stable_dt(2.0 / n, p)
    x = s.leapfrog_pml(s.pack(u, np.zeros_like(u)), 0.0, dt, int(round(T / dt)))
    e = x[:m.K * a.n3].reshape(m.K, a.n3)
    w = lambda v, mask: 0.5 * np.einsum("ki,kij,kj->", v[mask], a.M1[mask], v[mask])
    e0 = u[:, 0, 0:3].reshape(m.K, a.n3)
    return w(e, inside) / w(e0, np.ones(m.K, bool))


def test_layer_absorbs_under_leapfrog():
    kept_walls = _interior_energy(0.0)
    kept_pml = _interior_energy(40.0)
    assert kept_walls > 0.05
    assert kept_pml < 0.1 * kept_walls, (kept_pml, kept_walls)
