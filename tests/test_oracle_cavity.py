"""P7: the oracle against the closed-form TM110 mode of the PEC unit cube.

E_z = sin(pi x) sin(pi y) cos(w t), H = -(pi/w) (sin(pi x) cos(pi y),
-cos(pi x) sin(pi y), 0) sin(w t), w = pi sqrt(2), is an exact solution of
Eqs. (ampere_cont)/(faraday_cont) with eps = mu = 1 and e x n = 0 on the
walls.  Upwind flux with LSRK4 converges at O(h^{p+1}); central flux with
leapfrog at about O(h^p) on these meshes.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.solver import Solver

OM = math.pi * math.sqrt(2.0)


def e_exact(r, t):
    out = np.zeros_like(r)
    out[:, 2] = np.sin(math.pi * r[:, 0]) * np.sin(math.pi * r[:, 1]) * math.cos(OM * t)
    return out


def h_exact(r, t):
    out = np.zeros_like(r)
    s = math.sin(OM * t) / OM
    out[:, 0] = -math.pi * np.sin(math.pi * r[:, 0]) * np.cos(math.pi * r[:, 1]) * s
    out[:, 1] = math.pi * np.cos(math.pi * r[:, 0]) * np.sin(math.pi * r[:, 1]) * s
    return out


def run_cavity(n, p, integrator, flux, T=0.5):
    xyz, tets = W.kuhn_mesh(n)
    a = Assembly(Mesh(xyz, tets), p, 1.0, 1.0, flux)
    s = Solver(a)
    dt = W.stable_dt(1.0 / n, p)
    steps = int(math.ceil(T / dt))
    dt = T / steps
    nE = a.K * a.n3
    x = np.zeros((a.ndof, 1))
    x[:nE, 0] = s.project(lambda r: e_exact(r, 0.0), "E").reshape(-1)
    if integrator == "leapfrog":
        x = s.leapfrog(x, 0.0, dt, steps)
        th = T + 0.5 * dt
    else:
        x = s.lsrk4(x, 0.0, dt, steps)
        th = T
    ee = s.l2_error(x[:nE, 0].reshape(a.K, 3, a.N), lambda r: e_exact(r, T))
    eh = s.l2_error(x[nE:, 0].reshape(a.K, 3, a.N), lambda r: h_exact(r, th))
    return ee, eh


@pytest.mark.parametrize("p", [1, 2])
def test_p7_upwind_lsrk4_converges_at_p_plus_one(p):
    e2 = run_cavity(2, p, "lsrk4", "upwind")
    e4 = run_cavity(4, p, "lsrk4", "upwind")
    for a, b in zip(e2, e4):
        assert math.log2(a / b) > p + 1 - 0.15


def test_p7_central_leapfrog_converges():
    e2 = run_cavity(2, 2, "leapfrog", "central")
    e4 = run_cavity(4, 2, "leapfrog", "central")
    for a, b in zip(e2, e4):
        assert math.log2(a / b) > 2.4
    assert max(e4) < 6e-3
