"""Receivers (point evaluation of E, Eq. (mapped_eh)) against the oracle's own
evaluation of the same coefficients, for several columns."""
import numpy as np
import pytest

import workloads as W
from oracle_ref import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_receivers_match_oracle_point_values(D, prec, tol):
    xyz, tets = W.kuhn_mesh(3, jitter=0.12, seed=51)
    K, p, S = len(tets), 3, 3
    pos = W.random_points_in_box(7, (0.02, 0.02, 0.02), (0.98, 0.98, 0.98), seed=52)
    pos = np.concatenate([pos, xyz[[5, 17]]])            # two points on mesh vertices
    u = W.random_state(K, S, p, seed=53)
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3, S=S,
                 max_receivers=len(pos))
    g.set_state(u)
    g.set_receivers(pos)
    got = g.sample_receivers().cpu().numpy()             # [S, R, 3]
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", S=S)
    m = o.asm.mesh
    ref = np.zeros_like(got)
    for r, x in enumerate(pos):
        T = m.locate(x)
        # the oracle's collapsed-coordinate formula divides 0/0 on a vertex:
        # evaluate it 1e-10 towards the element's centroid there
        xe = x if r < 7 else x + 1e-10 * (m.verts[T].mean(axis=0) - x)
        for s in range(S):
            ref[s, r] = o.evaluate(u[T, s, 0:3].reshape(-1), T, xe[None, :])[0]
    scale = np.abs(ref).max()
    assert np.abs(got[:, :7] - ref[:, :7]).max() <= tol * scale
    assert np.abs(got[:, 7:] - ref[:, 7:]).max() <= max(tol, 1e-7) * scale


def test_receiver_capacity_is_enforced(D):
    xyz, tets = W.kuhn_mesh(2)
    g = D.Solver(xyz, tets, 1.0, 1.0, 2, "fp32", "upwind", "lsrk4", 1e-3, max_receivers=2)
    with pytest.raises(D.DgmError):
        g.set_receivers(np.full((3, 3), 0.5))
    with pytest.raises(D.DgmError):
        g.set_receivers(np.array([[2.0, 0.5, 0.5]]))
