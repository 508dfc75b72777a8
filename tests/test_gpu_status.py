"""Device status word: a non-finite state is latched as DGM_ENAN.

The NaN is written into the state from the host (nothing faults on the
device); the energy reduction sees it, dgm_energy returns DGM_ENAN, and
dgm_status_check reports the latched error once and then clears it.
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_in_state_is_latched(D, prec):
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=3)
    K, p, S = len(tets), 2, 3
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3, S=S)
    u = W.random_state(K, S, p, seed=4)
    g.set_state(u)
    assert np.all(np.isfinite(g.energy()))
    g.status()                                   # nothing latched
    u[7, 1, 4, 2] = np.nan                       # column 1 only
    g.set_state(u)
    with pytest.raises(D.DgmError) as ei:
        g.energy()
    assert ei.value.code == 6 and "column 1" in str(ei.value)
    with pytest.raises(D.DgmError) as ei:
        g.status()
    assert ei.value.code == 6
    g.status()                                   # read once, then cleared
    u[7, 1, 4, 2] = 0.0
    g.set_state(u)
    assert np.all(np.isfinite(g.energy()))
