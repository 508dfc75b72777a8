"""Batched advance (one CUDA graph launch per two steps over several problems)
against the same problems advanced one by one, and one member against the
oracle.  Members differ in order, precision, size, columns, PML and sources."""
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


def _members(D):
    out = []
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1))
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.1, 0.05, -0.02), 2.0, 1.0), W.dipole((-0.2, 0.1, 0.15), 3.0, 1.0), None]
    out.append(dict(args=(xyz, tets, 1.0, 1.0, 2, "fp32", "upwind", "lsrk4", W.stable_dt(2 / 3, 2)),
                    kw=dict(S=3, pml=pml), srcs=srcs, seed=1))
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=2)
    out.append(dict(args=(xyz, tets, 2.0, 1.0, 3, "fp64", "upwind", "lsrk4", W.stable_dt(0.5, 3)),
                    kw=dict(S=1), srcs=None, seed=2))
    xyz, tets = W.kuhn_mesh(4)
    out.append(dict(args=(xyz, tets, 1.0, 1.0, 1, "fp32", "upwind", "lsrk4", W.stable_dt(0.25, 1)),
                    kw=dict(S=2), srcs=None, seed=3))
    return out


def _make(D, spec):
    g = D.Solver(*spec["args"], **spec["kw"])
    if spec["srcs"]:
        g.set_sources(spec["srcs"])
    K, p, S = g.K, g.p, g.S
    g.set_state(W.random_state(K, S, p, seed=spec["seed"]) * 1e-2)
    return g


@pytest.mark.parametrize("steps", [4, 5])
def test_batch_matches_individual_advance(D, steps):
    import torch
    specs = _members(D)
    batch_members = [_make(D, s) for s in specs]
    single = [_make(D, s) for s in specs]
    b = D.Batch(batch_members)
    b.advance(steps)
    torch.cuda.synchronize()
    for gb, gs, spec in zip(batch_members, single, specs):
        gs.advance(steps, 0.0)
        tol = 1e-12 if spec["args"][5] == "fp64" else 1e-6
        assert rel_l2(gb.state(), gs.state()) < tol
        if gb.npml:
            a1 = gb.from_device(gb.aux[gb.current()])
            a2 = gs.from_device(gs.aux[gs.current()])
            assert rel_l2(a1, a2) < tol


def test_batch_member_matches_oracle(D):
    import torch
    spec = _members(D)[0]
    g = _make(D, spec)
    u0 = g.state()
    aux0 = np.zeros_like(u0)
    b = D.Batch([g, _make(D, _members(D)[2])])
    b.advance(6)
    torch.cuda.synchronize()
    xyz, tets, eps, mu, p, prec, flux, integ, dt = spec["args"]
    o = build(xyz, tets, p, eps, mu, flux, pml=spec["kw"]["pml"], S=3, sources=spec["srcs"])
    ref, ref_aux = o.unpack(o.lsrk4(o.pack(u0, aux0), 0.0, dt, 6))
    got = g.state()
    assert rel_l2(got, ref) < 1e-5
    assert rel_err(got, ref) < 1e-4                     # element by element
    ga = g.from_device(g.aux[g.current()])
    assert rel_l2(ga, ref_aux[g.pml_elements()]) < 1e-5


def test_autotuned_variants_match_oracle(D):
    """Every tile-shape variant the autotuner may pick gives the same stage:
    three single-column shapes and, up to p = 3, the paired kernels (two columns
    per thread, packed FP32x2 and scalar arithmetic) and, at p = 2, 3, the
    tensor-core variant (curl and lift as TF32 split products on tcgen05).
    486 columns leave a ragged last tile for every shape."""
    import torch
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=71)
    K, p, S = len(tets), 3, 3
    u = W.random_state(K, S, p, seed=72)
    dt = W.stable_dt(1 / 3, p)
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", S=S)
    ref = o.unpack(o.lsrk4(o.pack(u), 0.0, dt, 3))[0]
    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", dt, S=S)
    chosen, ms = g.autotune()
    assert len(ms) == 6 and 0 <= chosen < 6 and np.all(ms > 0)
    for v in range(6):
        g2 = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", dt, S=S)
        g2.set_state(u)
        g2.set_variant(v)
        g2.advance(3)
        assert rel_l2(g2.state(), ref) < 1e-5, v


def test_autotune_reads_state_only(D):
    """The autotuner times LSRK4 stage sequences in its workspace and the
    plan's second field and auxiliary buffers: the state (fields and PML
    auxiliaries, mid-run) is left bit for bit, and the steps after it equal
    those of an untuned twin plan set to the same shape and tile order."""
    xyz, tets = W.kuhn_mesh(2, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=73)
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.1, 0.05, -0.02), 2.0, 1.0)]
    p = 3
    dt = W.stable_dt(1.0, p)
    u = W.random_state(len(tets), 1, p, seed=75) * 1e-2
    twins = []
    for _ in range(2):
        g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", dt, S=1, pml=pml)
        g.set_sources(srcs)
        g.set_state(u)
        g.advance(2, 0.0)
        twins.append(g)
    a, b = twins
    aux = lambda g: g.from_device(g.aux[g.current()])
    st0, aux0 = a.state().copy(), aux(a).copy()
    assert np.abs(aux0).max() > 0
    chosen, ms = a.autotune()
    assert np.array_equal(a.state(), st0) and np.array_equal(aux(a), aux0)
    b.set_variant(chosen)
    b.set_tile_groups(a.tile_groups())
    for g in (a, b):
        g.advance(2, 2 * dt)
    assert np.array_equal(a.state(), b.state()) and np.array_equal(aux(a), aux(b))


_HIGH_P_REF = {}


def _high_p_case(p):
    """48-element PML mesh with a source (one partial tile) and the oracle's two
    LSRK4 steps from a seeded state, computed once per degree."""
    if p not in _HIGH_P_REF:
        xyz, tets = W.kuhn_mesh(2, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=73)
        pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
        srcs = [W.dipole((0.1, 0.05, -0.02), 2.0, 1.0)]
        dt = W.stable_dt(1.0, p)
        u = W.random_state(len(tets), 1, p, seed=74) * 1e-2
        o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=pml, S=1, sources=srcs)
        ref, ref_aux = o.unpack(o.lsrk4(o.pack(u, np.zeros_like(u)), 0.0, dt, 2))
        _HIGH_P_REF[p] = (xyz, tets, pml, srcs, dt, u, ref, ref_aux)
    return _HIGH_P_REF[p]


@pytest.mark.parametrize("p,prec,nv", [(4, "fp32", 4), (4, "fp64", 1), (5, "fp32", 4)])
def test_autotuner_variants_high_degree(D, p, prec, nv):
    """Above p = 3 the FP32 autotuner has four single-column shapes (the paired
    tile does not fit in shared memory; 32 x 512 is added) and FP64 has one;
    each gives the oracle's stage on a PML problem with a source."""
    import torch
    xyz, tets, pml, srcs, dt, u, ref, ref_aux = _high_p_case(p)
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=1, pml=pml)
    chosen, ms = g.autotune()
    assert len(ms) == nv and 0 <= chosen < nv and np.all(ms > 0)
    tol = 1e-5 if prec == "fp32" else 1e-12
    for v in range(nv):
        g2 = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=1, pml=pml)
        g2.set_sources(srcs)
        g2.set_state(u)
        g2.set_variant(v)
        g2.advance(2)
        assert rel_l2(g2.state(), ref) < tol, v
        assert rel_l2(g2.from_device(g2.aux[g2.current()]), ref_aux[g2.pml_elements()]) < tol, v


@pytest.mark.parametrize("p,v", [(1, 3), (2, 3), (3, 3), (1, 4), (2, 4), (3, 4), (2, 5), (3, 5)])
def test_paired_variants_pml_sources_match_oracle(D, p, v):
    """Paired kernels (v = 3, 4) on a problem where the two columns of a thread
    differ, and the tensor-core variant (v = 5, p = 2, 3) on the same problem:
    PML and non-PML elements, elements with and without a source, jittered
    geometry with element-wise materials, S = 3 columns per element (the last
    without a source)."""
    import torch
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=80 + p)
    K = len(tets)
    rng = np.random.default_rng(90 + p)
    eps = rng.uniform(1.0, 3.0, K)
    mu = rng.uniform(1.0, 2.0, K)
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.1, 0.05, -0.02), 2.0, 1.0), W.dipole((-0.2, 0.1, 0.15), 3.0, 1.0), None]
    S = 3
    dt = W.stable_dt(2 / 3, p)
    g = D.Solver(xyz, tets, eps, mu, p, "fp32", "upwind", "lsrk4", dt, S=S, pml=pml)
    g.set_sources(srcs)
    g.set_variant(v)
    u0 = W.random_state(K, S, p, seed=100 + p) * 1e-2
    g.set_state(u0)
    g.advance(4)
    torch.cuda.synchronize()
    o = build(xyz, tets, p, eps, mu, "upwind", pml=pml, S=S, sources=srcs)
    aux0 = np.zeros((K, S, 6, u0.shape[-1]))
    ref_u, ref_aux = o.unpack(o.lsrk4(o.pack(u0, aux0), 0.0, dt, 4))
    got = g.state()
    e_l2, e_max = rel_l2(got, ref_u), rel_err(got, ref_u)
    assert e_l2 < 1e-5 and e_max < 1e-4, (e_l2, e_max)
    a = g.from_device(g.aux[g.current()])
    assert rel_l2(a, ref_aux[g.pml_elements()]) < 1e-5
