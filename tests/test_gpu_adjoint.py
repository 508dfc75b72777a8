"""The hand-written adjoint (dgm_forward_record / dgm_adjoint and the autograd
Function on top) against the oracle's discrete adjoint, for upwind flux,
heterogeneous eps/mu, PML, several sources and receivers, and a step count
whose sqrt(N) checkpoint segments are ragged."""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import gradient, loss_records
from oracle.assemble import Assembly, pml_sigma
from oracle.mesh import Mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _problem(p):
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=61)
    m = Mesh(xyz, tets)
    K = m.K
    eps = W.lognormal_material(K, 2.0, 0.3, 62)
    mu = W.lognormal_material(K, 1.0, 0.2, 63)
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=10.0, order=2)
    sigma = pml_sigma(m.centroids(), pml["lo"], pml["hi"], pml["thickness"], pml["sigma_max"], 2)
    srcs = [W.dipole((0.1, 0.05, -0.1), 2.0, 1.5), W.dipole((-0.2, 0.15, 0.12), 3.0, 1.5)]
    rec = np.array([[0.3, -0.2, 0.1], [-0.25, 0.3, -0.15], [0.05, 0.05, 0.35]])
    dt = W.stable_dt(2 / 3, p)
    return xyz, tets, m, eps, mu, pml, sigma, srcs, rec, dt


@pytest.mark.parametrize("p", [1, 2])
def test_adjoint_gradient_matches_oracle(D, p):
    import torch
    xyz, tets, m, eps, mu, pml, sigma, srcs, rec, dt = _problem(p)
    steps, S = 10, 2
    target = 0.1 * np.random.default_rng(2).standard_normal((steps, S, len(rec), 3))
    g = D.Solver(xyz, tets, eps, mu, p, "fp64", "upwind", "lsrk4", dt, S=S, pml=pml,
                 max_receivers=len(rec))
    g.set_sources(srcs)
    g.set_receivers(rec)
    e_t = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    m_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    records = D.receiver_records(g, e_t, m_t, steps)
    loss = 0.5 * ((records - torch.tensor(target, device=records.device)) ** 2).sum()
    loss.backward()
    x0 = np.zeros((Assembly(m, p, eps, mu, "upwind", sigma=sigma, rows=[0]).ndof, S))
    ref_rec = loss_records(m, p, eps, mu, "upwind", sigma, S, srcs, x0, 0.0, dt, steps, rec)
    assert np.abs(records.detach().cpu().numpy() - ref_rec).max() < 1e-12 * np.abs(ref_rec).max()
    elements = [0, 12, 40, 77, 100, 150, 161]
    ref, _ = gradient(m, p, eps, mu, "upwind", sigma, S, srcs, x0, 0.0, dt, steps, rec,
                      lambda r: r - target, elements=elements)
    ge = e_t.grad.numpy()[elements]
    gm = m_t.grad.numpy()[elements]
    assert np.abs(ge - ref["eps"]).max() < 1e-10 * np.abs(ref["eps"]).max()
    assert np.abs(gm - ref["mu"]).max() < 1e-10 * np.abs(ref["mu"]).max()


def test_fp32_adjoint_close_to_fp64(D):
    import torch
    xyz, tets, m, eps, mu, pml, sigma, srcs, rec, dt = _problem(2)
    steps, S = 10, 2
    target = 0.1 * np.random.default_rng(3).standard_normal((steps, S, len(rec), 3))
    grads = []
    for prec in ("fp64", "fp32"):
        g = D.Solver(xyz, tets, eps, mu, 2, prec, "upwind", "lsrk4", dt, S=S, pml=pml,
                     max_receivers=len(rec))
        g.set_sources(srcs)
        g.set_receivers(rec)
        e_t = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
        m_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
        r = D.receiver_records(g, e_t, m_t, steps)
        (0.5 * ((r - torch.tensor(target, device=r.device)) ** 2).sum()).backward()
        grads.append(np.concatenate([e_t.grad.numpy(), m_t.grad.numpy()]))
    assert np.abs(grads[1] - grads[0]).max() < 1e-4 * np.abs(grads[0]).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_index_width_paths_agree(D, prec):
    """The forward and adjoint kernels use 32-bit index arithmetic when every
    index fits; forcing their 64-bit versions gives the same records and the
    same eps/mu gradients bit for bit."""
    import torch
    xyz, tets, m, eps, mu, pml, sigma, srcs, rec, dt = _problem(2)
    steps, S = 7, 2
    target = 0.1 * np.random.default_rng(3).standard_normal((steps, S, len(rec), 3))
    out = []
    for force in (False, True):
        g = D.Solver(xyz, tets, eps, mu, 2, prec, "upwind", "lsrk4", dt, S=S, pml=pml,
                     max_receivers=len(rec))
        if force:
            g.set_index64(True)
        g.set_sources(srcs)
        g.set_receivers(rec)
        e_t = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
        m_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
        records = D.receiver_records(g, e_t, m_t, steps)
        loss = 0.5 * ((records - torch.tensor(target, device=records.device)) ** 2).sum()
        loss.backward()
        out.append((records.detach().cpu().numpy(), e_t.grad.numpy().copy(), m_t.grad.numpy().copy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert np.abs(out[0][1]).max() > 0
