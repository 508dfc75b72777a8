"""Phase 1 of the stage kernel by tiled bulk copies (TMA) against per-thread loads.

Where a plan has one column per element (S = 1) and K a multiple of 4 (FP32)
or 2 (FP64), dgm_bind builds tensor maps and one thread of each CTA moves the
tile's coefficients, element constants and face constants with four bulk
copies; dgm_set_tile_loads(1) forces the per-thread loads that every other
plan uses.  Both fill the same shared-memory rows with the same values, so
trajectories must agree bit for bit:

* LSRK4 steps with PML auxiliaries, a point source and element-wise
  materials, FP32 and FP64, p = 2, 3, on a 6^3 Kuhn grid (1296 elements: the
  last 32-column tile holds 16 columns, so the copies run past the end of the
  tensors and read zeros there), for each single-column tile shape of the
  FP32 autotuner (32 x 384, 32 x 192, 16 x 192);
* the interior penalty (its own face-constant and A^T boxes) and incident
  faces;
* right-hand side only, leapfrog half steps, and the plan-level choice
  (bulk where allowed, per-thread where K or S rule it out).

One bulk-copy trajectory is also compared with the oracle directly.
"""
import numpy as np
import pytest

import workloads as W
from oracle_ref import build, rel_err, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


PML = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)


def _mesh(n, seed):
    return W.kuhn_mesh(n, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=seed)


def _pair(D, make, steps, t0=0.0):
    """Run the same problem with bulk copies and with per-thread loads."""
    out = []
    for per_thread in (False, True):
        g = make()
        if per_thread:
            g.set_tile_loads(True)
        assert g.bulk_tile_loads() == (not per_thread)
        steps(g)
        out.append(g)
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("p", [2, 3])
def test_lsrk4_bulk_equals_per_thread(D, prec, p):
    xyz, tets = _mesh(6, 31 + p)
    K = len(tets)
    assert K % 32 == 16
    eps = W.lognormal_material(K, 2.0, 0.3, 32)
    mu = W.lognormal_material(K, 1.2, 0.2, 33)
    dt = W.stable_dt(2 / 6, p) / 2
    u = W.random_state(K, 1, p, seed=34) * 1e-2

    def make():
        g = D.Solver(xyz, tets, eps, mu, p, prec, "upwind", "lsrk4", dt, S=1, pml=PML)
        g.set_sources([W.dipole((0.11, -0.07, 0.05), 2.0, 1.0)])
        g.set_state(u)
        return g

    a, b = _pair(D, make, lambda g: g.advance(4, 0.0))
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.from_device(a.aux[a.current()]), b.from_device(b.aux[b.current()]))
    a.status()                          # no timeout or bad index latched


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fp32_tile_shapes_bulk_equals_per_thread(D, variant):
    p = 3
    xyz, tets = _mesh(6, 41)
    K = len(tets)
    dt = W.stable_dt(2 / 6, p) / 2
    u = W.random_state(K, 1, p, seed=42)

    def make():
        g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", dt, S=1)
        g.set_variant(variant)
        g.set_state(u)
        return g

    a, b = _pair(D, make, lambda g: g.advance(3, 0.0))
    assert np.array_equal(a.state(), b.state())


def test_tile_orders_bulk_equals_per_thread(D):
    """The copies start at the tile the CTA visits (tile_index)."""
    p = 3
    xyz, tets = _mesh(4, 43)          # 384 elements: 12 tiles of 32
    dt = W.stable_dt(2 / 4, p) / 2
    u = W.random_state(len(tets), 1, p, seed=44)
    ref = None
    for groups in (1, 3, 4, 6, 12):
        def make():
            g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "central", "lsrk4", dt, S=1)
            g.set_tile_groups(groups)
            g.set_state(u)
            return g
        a, b = _pair(D, make, lambda g: g.advance(2, 0.0))
        assert np.array_equal(a.state(), b.state())
        if ref is None:
            ref = a.state()
        assert np.array_equal(a.state(), ref)


def test_interior_penalty_bulk_equals_per_thread(D):
    """The penalty's kernel copies 16 face-constant rows per face and A^T."""
    p = 3
    xyz, tets = _mesh(6, 45)
    K = len(tets)
    eps = W.lognormal_material(K, 2.0, 0.3, 46)
    dt = W.stable_dt(2 / 6, p) / 2
    u = W.random_state(K, 1, p, seed=47)

    def make():
        g = D.Solver(xyz, tets, eps, 1.0, p, "fp32", "central", "lsrk4", dt, S=1, sip=4.0)
        g.set_state(u)
        return g

    a, b = _pair(D, make, lambda g: g.advance(3, 0.0))
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.facet_state(), b.facet_state())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_incident_faces_bulk_equals_per_thread(D, prec):
    p, n = 2, 6
    xyz, tets = W.kuhn_mesh(n, jitter=0.1, seed=48)
    faces = np.concatenate([W.box_faces(n, tets, 2, 0), W.box_faces(n, tets, 0, 1)])
    dt = W.stable_dt(1 / n, p) / 2
    wave = dict(E0=(0.8, -0.3, 0.45), direction=(0.0, 0.0, 1.0), speed=1.0, f0=0.3, bw=0.25, t0=0.4)

    def make():
        g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=1)
        g.set_incident(faces, **wave)
        return g

    a, b = _pair(D, make, lambda g: g.advance(5, 0.0))
    assert np.abs(a.state()).max() > 0          # the wave has entered
    assert np.array_equal(a.state(), b.state())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rhs_and_leapfrog_bulk_equal_per_thread(D, prec):
    """Right-hand side of the plan's own field buffer (the bulk path; a
    caller's buffer takes per-thread loads) and leapfrog half steps."""
    p = 3
    xyz, tets = _mesh(6, 49)
    dt = W.stable_dt(2 / 6, p) / 2
    u = W.random_state(len(tets), 1, p, seed=50)
    out = []
    for per_thread in (False, True):
        g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=1)
        g.set_tile_loads(per_thread)
        g.set_state(u)
        out.append(g.from_device(g.rhs(g.fields[g.current()], t=0.2)))
        out.append(g.from_device(g.rhs(u, t=0.2)))
    assert np.array_equal(out[0], out[2])
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[2], out[3])
    lf = []
    for per_thread in (False, True):
        g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "central", "leapfrog", dt, S=1)
        g.set_tile_loads(per_thread)
        g.set_state(u)
        g.leapfrog_start(0.0)
        g.advance(6, 0.0)
        lf.append(g.state())
    assert np.array_equal(lf[0], lf[1])


def test_bulk_copies_only_where_the_layout_allows(D):
    """S = 1 and rows on 16-byte boundaries: K % 4 == 0 in FP32, K even in FP64."""
    x3, t3 = W.kuhn_mesh(3)                      # 162 elements
    x4, t4 = W.kuhn_mesh(4)                      # 384 elements
    cases = [((x3, t3), "fp32", 1, False), ((x3, t3), "fp64", 1, True),
             ((x4, t4), "fp32", 1, True), ((x4, t4), "fp32", 2, False)]
    for (xyz, tets), prec, S, expect in cases:
        g = D.Solver(xyz, tets, 1.0, 1.0, 2, prec, "upwind", "lsrk4", 1e-3, S=S)
        assert g.bulk_tile_loads() == expect, (len(tets), prec, S)
        g.set_tile_loads(True)
        assert not g.bulk_tile_loads()
        g.set_tile_loads(False)
        assert g.bulk_tile_loads() == expect


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_bulk_trajectory_matches_oracle(D, prec, tol):
    p = 2
    xyz, tets = _mesh(4, 51)
    K = len(tets)
    srcs = [W.dipole((0.11, -0.07, 0.05), 2.0, 1.0)]
    dt = W.stable_dt(2 / 4, p)
    u = W.random_state(K, 1, p, seed=52) * 1e-2
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=1, pml=PML)
    assert g.bulk_tile_loads()
    g.set_sources(srcs)
    g.set_state(u)
    g.advance(6, 0.0)
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=PML, S=1, sources=srcs)
    ref, ref_aux = o.unpack(o.lsrk4(o.pack(u, np.zeros_like(u)), 0.0, dt, 6))
    assert rel_l2(g.state(), ref) < tol
    assert rel_err(g.state(), ref) < 10 * tol
    assert rel_l2(g.from_device(g.aux[g.current()]), ref_aux[g.pml_elements()]) < tol
