"""Parity at the full size of the jittered-sphere workload (32^3 Kuhn grid,
196,608 elements, p = 3, upwind flux), in the launch configuration the bench
times, on sampled elements the oracle computes one by one.

* dgm_rhs: the oracle assembles only the sampled elements' rows.
* one LSRK4 time step (five stage launches of the bench's kernel): the value
  of a sampled element after five stages depends on its 5-ring of neighbours,
  so the oracle assembles the 4-ring neighbourhood and advances those rows;
  errors from the untouched elements outside the neighbourhood move inward by
  one ring per stage and never reach the sampled elements.
"""
import numpy as np
import pytest

import workloads as W
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.solver import LSRK4_A, LSRK4_B, Solver as OSolver
from oracle_ref import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


@pytest.fixture(scope="module")
def workload():
    w = W.jittered_sphere()
    xyz, tets = w.mesh()
    c, r, ein, eout = w.extra["sphere"]
    eps = W.sphere_material(xyz, tets, c, r, ein, eout)
    mesh = Mesh(xyz, tets)
    rng = np.random.default_rng(77)
    K = len(tets)
    bnd = np.nonzero((mesh.nbr < 0).any(axis=1))[0]
    inside = np.nonzero(eps > 1)[0]
    sample = np.unique(np.concatenate([rng.choice(K, 10, replace=False), rng.choice(bnd, 3),
                                       rng.choice(inside, 3), [0, K - 1]]))
    u = W.random_state(K, 1, w.p, seed=78)
    return w, xyz, tets, eps, mesh, sample, u


def _ring(mesh, seeds, depth):
    cur = set(int(s) for s in seeds)
    for _ in range(depth):
        nxt = set(cur)
        for e in cur:
            nxt.update(int(n) for n in mesh.nbr[e] if n >= 0)
        cur = nxt
    return np.array(sorted(cur))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fullsize_rhs_sampled(D, workload, prec):
    w, xyz, tets, eps, mesh, sample, u = workload
    g = D.Solver(xyz, tets, eps, 1.0, w.p, prec, "upwind", "lsrk4", w.dt)
    got = g.from_device(g.rhs(u))[sample]
    o = OSolver(Assembly(mesh, w.p, eps, 1.0, "upwind", rows=sample))
    ref = o.unpack(o.rhs(o.pack(u)))[0]
    assert rel_err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fullsize_lsrk4_step_sampled(D, workload, prec):
    w, xyz, tets, eps, mesh, sample, u = workload
    g = D.Solver(xyz, tets, eps, 1.0, w.p, prec, "upwind", "lsrk4", w.dt)
    g.set_state(u)
    g.advance(1, 0.0)
    got = g.state()[sample]
    rows = _ring(mesh, sample[:6], 4)
    o = OSolver(Assembly(mesh, w.p, eps, 1.0, "upwind", rows=rows))
    x = o.pack(u)
    K, n3 = len(tets), 3 * W.n_modes(w.p)
    idx = np.concatenate([(b * K + rows)[:, None] * n3 + np.arange(n3)[None, :]
                          for b in range(2)]).ravel()
    res = np.zeros((len(idx), 1))
    for k in range(5):
        res = LSRK4_A[k] * res + w.dt * o.rhs(x)
        x[idx] += LSRK4_B[k] * res
    ref = np.transpose(x[idx].reshape(2, len(rows), 3, -1), (1, 0, 2, 3)).reshape(len(rows), 1, 6, -1)
    pos = np.searchsorted(rows, sample[:6])
    assert rel_err(got[:6], ref[pos]) < TOL[prec]
