"""The GPU adjoint gradient against central finite differences of the GPU
forward loss (FP64) on 20 seeded elements of a small inverse problem of the
same kind as the benchmarked one (PML, lognormal eps, dipoles, receivers)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def test_adjoint_matches_central_differences_on_20_elements(D):
    import torch
    w = W.inverse_problem(n=6, p=2, n_sources=3, n_receivers=6, steps=30)
    xyz, tets = w.mesh()
    rec = w.extra["receivers"]
    g = D.Solver(xyz, tets, w.extra["eps"], 1.0, w.p, "fp64", w.flux, w.integrator, w.dt, S=w.S,
                 pml=w.pml, max_receivers=len(rec))
    g.set_sources(w.extra["sources"])
    g.set_receivers(rec)
    steps = 30
    mu = torch.ones(g.K, dtype=torch.float64)
    with torch.no_grad():
        target = D.receiver_records(g, torch.tensor(w.extra["eps_target"]), mu, steps)

    def loss(e):
        with torch.no_grad():
            r = D.receiver_records(g, torch.tensor(e), mu, steps)
        return float(0.5 * ((r - target) ** 2).sum())

    eps = torch.tensor(w.extra["eps"], requires_grad=True)
    r = D.receiver_records(g, eps, mu.clone().requires_grad_(True), steps)
    (0.5 * ((r - target) ** 2).sum()).backward()
    grad = eps.grad.numpy()
    rng = np.random.default_rng(7)
    elements = rng.choice(g.K, 20, replace=False)
    fd = []
    for T in elements:
        d = 1e-5 * w.extra["eps"][T]
        ep, em = w.extra["eps"].copy(), w.extra["eps"].copy()
        ep[T] += d
        em[T] -= d
        fd.append((loss(ep) - loss(em)) / (2 * d))
    fd = np.array(fd)
    assert np.abs(grad[elements] - fd).max() <= 1e-4 * np.abs(fd).max()
