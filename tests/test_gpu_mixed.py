"""Mixed orders on the GPU (E of degree p + 1, H of degree p; Sec. III,
Eqs. (triale)/(trialh); dgm_plan_create_mixed) against the mixed-order
oracle: right-hand side with a dipole source, central and upwind flux, p = 1..3,
element-wise materials, jittered geometry, two columns; an LSRK4 trajectory;
energy; projection of a polynomial field."""
import numpy as np
import pytest

import workloads as W
from oracle.mesh import Mesh
from oracle.mixed import MixedAssembly, MixedSolver
from oracle_ref import rel_err, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _case(p, flux, S=2, seed=0):
    xyz, tets = W.kuhn_mesh(3, jitter=0.12, seed=101 + seed)
    K = len(tets)
    eps = W.lognormal_material(K, 2.0, 0.3, 102 + seed)
    mu = W.lognormal_material(K, 1.0, 0.2, 103 + seed)
    srcs = [W.dipole((0.41, 0.37, 0.55), 2.0, 1.0), None][:S]
    NE, NH = W.n_modes(p + 1), W.n_modes(p)
    u = W.random_state(K, S, p + 1, seed=104 + seed)
    u[:, :, 3:6, NH:] = 0.0                      # H has only its first NH modes
    o = MixedSolver(MixedAssembly(Mesh(xyz, tets), p + 1, p, eps, mu, flux), S=S, sources=srcs)
    return xyz, tets, eps, mu, srcs, u, o


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["central", "upwind"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_rhs_matches_oracle(D, p, flux, prec):
    xyz, tets, eps, mu, srcs, u, o = _case(p, flux)
    g = D.Solver(xyz, tets, eps, mu, p, prec, flux, "lsrk4", 1e-3, S=2, mixed=True)
    assert (g.N, g.NH) == (W.n_modes(p + 1), W.n_modes(p))
    g.set_sources(srcs)
    t = 0.37
    got = g.from_device(g.rhs(u, t=t))
    ref = o.unpack(o.rhs(o.pack(u), t))
    assert rel_err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_lsrk4_trajectory_and_energy(D, prec):
    p = 2
    xyz, tets, eps, mu, srcs, u, o = _case(p, "upwind", seed=5)
    dt = W.stable_dt(1 / 3, p + 1)
    g = D.Solver(xyz, tets, eps, mu, p, prec, "upwind", "lsrk4", dt, S=2, mixed=True)
    g.set_sources(srcs)
    g.set_state(u)
    e0 = g.energy()
    assert np.allclose(e0, o.energy(o.pack(u)), rtol=TOL[prec], atol=0)
    g.advance(12, 0.0)
    got = g.state()
    x = o.lsrk4(o.pack(u), 0.0, dt, 12)
    ref = o.unpack(x)
    assert rel_l2(got, ref) < TOL[prec] and rel_err(got, ref) < 10 * TOL[prec]
    assert np.allclose(g.energy(), o.energy(x), rtol=10 * TOL[prec], atol=0)
    assert np.all(g.energy() < e0)               # upwind flux dissipates


def test_mixed_projection_of_a_polynomial_field(D):
    p = 2
    xyz, tets, eps, mu, srcs, u, o = _case(p, "central")
    fe = lambda r: np.stack([r[:, 0] * r[:, 1] * r[:, 2], r[:, 1] ** 3 - r[:, 0], r[:, 2] ** 2], axis=1)
    fh = lambda r: np.stack([r[:, 0] ** 2, r[:, 1] * r[:, 2] + 1.0, r[:, 0] - r[:, 2]], axis=1)
    g = D.Solver(xyz, tets, eps, mu, p, "fp64", "central", "lsrk4", 1e-3, S=1, mixed=True)
    g.project(lambda r: np.concatenate([fe(r), fh(r)], axis=1))
    got = g.state()[:, 0]
    want_e = o.project(fe, "E")                  # degree p + 1 = 3 reproduces fe exactly
    want_h = o.project(fh, "H")                  # degree p = 2 reproduces fh exactly
    assert np.abs(got[:, 0:3, :] - want_e).max() < 1e-11
    assert np.abs(got[:, 3:6, :o.asm.NH] - want_h).max() < 1e-11
    assert np.all(got[:, 3:6, o.asm.NH:] == 0.0)
