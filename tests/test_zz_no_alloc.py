"""The allocation-free energy entry point (dgm_energy_noalloc) against dgm_energy.

dgm_energy_noalloc serves callers that must not allocate device memory (a
latency-critical loop where an allocation would synchronise the device, or
an application whose device memory belongs to another framework's
allocator).  It keeps its reduction scratch in a fixed array inside the
library.  This file is collected last so that a failure here does not hide
the other tests; it passes both alone in a fresh process and after them.
"""
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


@pytest.mark.parametrize("prec,S", [("fp64", 3), ("fp32", 5)])
def test_noalloc_energy_matches_energy_on_consecutive_calls(D, prec, S):
    import torch
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=41)
    K, p = len(tets), 3
    eps = W.lognormal_material(K, 2.0, 0.3, 42)
    g = D.Solver(xyz, tets, eps, 1.5, p, prec, "upwind", "lsrk4", 1e-3, S=S)
    for call, seed in enumerate((43, 44)):        # two calls in a row, different states
        g.set_state(W.random_state(K, S, p, seed=seed))
        want = g.energy()
        out = torch.full((S,), float("nan"), dtype=torch.float64, device=g.device)
        g.energy_noalloc(out)
        torch.cuda.synchronize(g.device)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), call


def test_noalloc_energy_rejects_too_many_columns(D):
    import torch
    xyz, tets = W.kuhn_mesh(1)
    g = D.Solver(xyz, tets, 1.0, 1.0, 1, "fp32", "upwind", "lsrk4", 1e-3, S=65)
    out = torch.zeros(65, dtype=torch.float64, device=g.device)
    with pytest.raises(D.DgmError) as ei:
        g.energy_noalloc(out)
    assert ei.value.code == 1 and "at most 64 columns" in str(ei.value)


def test_noalloc_energy_at_the_column_limit(D):
    """A plan with exactly DGM_NOALLOC_MAX_COLUMNS (64) columns uses every entry
    of the fixed scratch array; it matches dgm_energy on two calls in a row."""
    import torch
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=45)
    K, p, S = len(tets), 2, 64
    g = D.Solver(xyz, tets, 1.3, 0.8, p, "fp64", "upwind", "lsrk4", 1e-3, S=S)
    for call, seed in enumerate((46, 47)):
        g.set_state(W.random_state(K, S, p, seed=seed))
        want = g.energy()
        out = torch.full((S,), float("nan"), dtype=torch.float64, device=g.device)
        g.energy_noalloc(out)
        torch.cuda.synchronize(g.device)
        got = out.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), call


def test_noalloc_energy_allocates_no_device_memory(D):
    """After a first call (which looks up the scratch array's address), many
    calls leave the device's free memory unchanged: no allocation happens."""
    import torch
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=48)
    K, p, S = len(tets), 3, 8
    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", 1e-3, S=S)
    g.set_state(W.random_state(K, S, p, seed=49))
    out = torch.zeros(S, dtype=torch.float64, device=g.device)
    g.energy_noalloc(out)
    torch.cuda.synchronize(g.device)
    free0 = torch.cuda.mem_get_info(g.device)[0]
    for _ in range(200):
        g.energy_noalloc(out)
    torch.cuda.synchronize(g.device)
    assert torch.cuda.mem_get_info(g.device)[0] == free0
