"""The partitioned device path on one GPU: a mesh cut into slabs, each part a
plan over its owned elements plus halo (dgm_set_active), stepped stage by
stage (dgm_stage) with the halo refreshed after every stage by the device
pack/unpack kernels (dgm_halo_pack / dgm_halo_unpack) and plain copies
between the parts' buffers.  The parts run one after another on one device,
so no kernel waits on another.  Each owned element must equal the
single-domain run bit for bit (the same arithmetic per column), with PML,
sources and several columns."""
import numpy as np
import pytest

import workloads as W
from oracle_ref import build, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


@pytest.mark.parametrize("prec,nparts,variant", [("fp64", 2, 0), ("fp32", 2, 0), ("fp32", 3, 0),
                                                 ("fp32", 2, 3), ("fp32", 2, 5)])
def test_partitioned_steps_equal_single_domain(D, prec, nparts, variant):
    xyz, tets = W.kuhn_mesh(4, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=31)
    K, p, S = len(tets), 3, 2
    eps = W.lognormal_material(K, 2.0, 0.3, 32)
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=10.0, order=2)
    srcs = [W.dipole((0.11, -0.07, 0.3), 2.0, 1.0), None]
    dt = W.stable_dt(0.5, p)
    u = W.random_state(K, S, p, seed=33) * 1e-2
    steps = 4
    glob = D.Solver(xyz, tets, eps, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
    glob.set_sources(srcs)
    part = D.partition_slabs(xyz, tets, nparts, axis=2)
    parts = [D.PartitionedSolver(xyz, tets, eps, 1.0, p, prec, "upwind", dt, part, nparts, r,
                                 pml=pml, S=S, exchange=None) for r in range(nparts)]
    if prec == "fp32":
        glob.set_variant(variant)
    for pt in parts:
        pt.set_sources(srcs)
        pt.set_state(u)
        if prec == "fp32":
            pt.solver.set_variant(variant)
        assert pt.halo.n_ghost > 0
    glob.set_state(u)
    glob.advance(steps, 0.0)
    D.advance_local(parts, steps, 0.0)
    want = glob.state()
    seen = np.zeros(K, dtype=bool)
    for pt in parts:
        ids, got = pt.owned_state()
        assert np.array_equal(got, want[ids])
        seen[ids] = True
        pt.solver.status()
    assert seen.all()
    if prec == "fp64":   # and the single-domain run is the oracle's
        o = build(xyz, tets, p, eps, 1.0, "upwind", pml=pml, S=S, sources=srcs)
        ref = o.unpack(o.lsrk4(o.pack(u, np.zeros_like(u)), 0.0, dt, steps))[0]
        assert rel_l2(want, ref) < 1e-12


def test_halo_pack_unpack_round_trip(D):
    import torch
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=34)
    K, p, S = len(tets), 2, 3
    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", 1e-3, S=S)
    u = W.random_state(K, S, p, seed=35)
    g.set_state(u)
    idx = torch.tensor([5, 0, 47, 12], dtype=torch.int64, device=g.device)
    buf = g.halo_pack(idx)
    ref = np.transpose(u[[5, 0, 47, 12]], (2, 3, 0, 1)).reshape(6 * g.N, 4, S)
    assert np.array_equal(buf.cpu().numpy(), ref.astype(np.float32))
    g.halo_unpack(torch.tensor([1, 2, 3, 4], dtype=torch.int64, device=g.device), buf)
    v = g.state()
    assert np.array_equal(v[[1, 2, 3, 4]], u[[5, 0, 47, 12]].astype(np.float32))
    bad = torch.tensor([3, K + 5], dtype=torch.int64, device=g.device)
    g.halo_pack(bad)                       # the bad id is skipped and latched
    with pytest.raises(D.DgmError) as ei:
        g.status()
    assert ei.value.code == 1 and "halo" in str(ei.value)
