"""PEC cavity workload (4^3 Kuhn grid, 384 elements, p = 2, vacuum, central
flux, leapfrog, dt = 0.3 h / (p+1)^2, 200 steps) on the GPU: parity with the
oracle's trajectory (FP64, 1e-12) and closeness to the closed-form TM110
mode, whose initial field is projected by the library itself."""
import math

import numpy as np
import pytest

import workloads as W
from oracle_ref import build, rel_l2
from test_oracle_cavity import e_exact, h_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_cavity_tm110(D, prec, tol):
    w = W.cavity_tm110()
    xyz, tets = w.mesh()
    g = D.Solver(xyz, tets, 1.0, 1.0, w.p, prec, w.flux, w.integrator, w.dt)
    g.project(lambda r: np.concatenate([e_exact(r, 0.0), np.zeros_like(r)], axis=1))
    u0 = g.state()
    g.leapfrog_start(0.0)
    g.advance(w.steps, 0.0)
    got = g.state()
    o = build(xyz, tets, w.p, 1.0, 1.0, "central")
    x = o.leapfrog(o.pack(u0), 0.0, w.dt, w.steps)
    ref = o.unpack(x)[0]
    assert rel_l2(got, ref) < tol
    T = w.steps * w.dt
    K, N = len(tets), w.N
    err_e = o.l2_error(got[:, 0, 0:3, :], lambda r: e_exact(r, T))
    err_h = o.l2_error(got[:, 0, 3:6, :], lambda r: h_exact(r, T + 0.5 * w.dt))
    norm_e = o.l2_error(np.zeros((K, 3, N)), lambda r: e_exact(r, 0.0))
    assert err_e < 0.02 * norm_e and err_h < 0.02 * norm_e
