"""Pins of the oracle's discrete adjoint (used to check the GPU adjoint).

* dot-product test: <F_u v, w> = <v, F_u^T w> for the assembled operator with
  upwind flux, heterogeneous materials and PML;
* the adjoint gradient of a receiver-misfit loss with respect to per-element
  eps and mu agrees with central finite differences of the loss computed by
  the oracle's forward stepping;
* the complex-step material derivative agrees with a finite difference of the
  right-hand side.
"""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import MaterialDerivative, apply_transpose, gradient, loss_records
from oracle.assemble import Assembly, pml_sigma
from oracle.mesh import Mesh
from oracle.solver import Solver


def _problem():
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=61)
    m = Mesh(xyz, tets)
    K = m.K
    eps = W.lognormal_material(K, 2.0, 0.3, 62)
    mu = W.lognormal_material(K, 1.0, 0.2, 63)
    sigma = pml_sigma(m.centroids(), (-0.5,) * 3, (0.5,) * 3, 0.5, 10.0, 2)
    srcs = [W.dipole((0.1, 0.05, -0.1), 2.0, 1.5), W.dipole((-0.2, 0.15, 0.12), 3.0, 1.5)]
    rec = np.array([[0.3, -0.2, 0.1], [-0.25, 0.3, -0.15], [0.05, 0.05, 0.35]])
    return m, eps, mu, sigma, srcs, rec


def test_dot_product_of_the_transpose():
    m, eps, mu, sigma, srcs, rec = _problem()
    a = Assembly(m, 1, eps, mu, "upwind", sigma=sigma)
    s = Solver(a, S=2)
    rng = np.random.default_rng(0)
    v = rng.standard_normal((a.ndof, 2))
    w = rng.standard_normal((a.ndof, 2))
    lhs = np.sum(s.rhs(v) * w)
    rhs = np.sum(v * apply_transpose(s, w))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_complex_step_material_derivative():
    m, eps, mu, sigma, srcs, rec = _problem()
    T = 40
    d = MaterialDerivative(m, 1, eps, mu, "upwind", sigma, 2, srcs, "eps", T)
    rng = np.random.default_rng(1)
    a = Assembly(m, 1, eps, mu, "upwind", sigma=sigma)
    x = rng.standard_normal((a.ndof, 2))
    lr = rng.standard_normal((a.ndof, 2))
    got = d.dot(lr, x, 0.37)
    delta = 1e-6 * eps[T]
    vals = []
    for sgn in (1, -1):
        e2 = eps.copy()
        e2[T] += sgn * delta
        s2 = Solver(Assembly(m, 1, e2, mu, "upwind", sigma=sigma, rows=d.rows), S=2, sources=srcs)
        vals.append(np.sum(lr[d.idx] * s2.rhs(x, 0.37)))
    fd = (vals[0] - vals[1]) / (2 * delta)
    assert abs(got - fd) < 1e-6 * abs(fd)


@pytest.mark.parametrize("which", ["eps", "mu"])
def test_adjoint_gradient_matches_finite_differences(which):
    m, eps, mu, sigma, srcs, rec = _problem()
    K, p, S, steps = m.K, 1, 2, 6
    dt = W.stable_dt(2 / 3, p)
    x0 = np.zeros((Assembly(m, p, eps, mu, "upwind", sigma=sigma, rows=[0]).ndof, S))
    target = 0.1 * np.random.default_rng(2).standard_normal((steps, S, len(rec), 3))

    def loss(e, u):
        r = loss_records(m, p, e, u, "upwind", sigma, S, srcs, x0, 0.0, dt, steps, rec)
        return 0.5 * np.sum((r - target) ** 2)

    elements = [12, 77, 150]
    g, _ = gradient(m, p, eps, mu, "upwind", sigma, S, srcs, x0, 0.0, dt, steps, rec,
                    lambda r: r - target, elements=elements, which=(which,))
    fds = []
    for i, T in enumerate(elements):
        base = (eps if which == "eps" else mu).copy()
        d = 1e-4 * base[T]
        vals = []
        for sgn in (1, -1):
            b = base.copy()
            b[T] += sgn * d
            vals.append(loss(b, mu) if which == "eps" else loss(eps, b))
        fds.append((vals[0] - vals[1]) / (2 * d))
    fds = np.array(fds)
    # relative to the largest sampled entry: far from the sources the entries are
    # small and their finite differences are dominated by rounding of the loss
    assert np.abs(g[which] - fds).max() <= 1e-6 * np.abs(fds).max(), (g[which], fds)
