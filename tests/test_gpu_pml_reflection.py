"""PML absorption on the GPU path: a dipole in [-1,1]^3 with the PML against the
same problem on [-2,2]^3 (bench.run_reflection).  With the PML the E field in the
inner box stays close to the larger domain's; without it (sigma_max = 0) the
walls reflect, which shows the measurement can see a reflection; the error falls
with resolution."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.fixture(scope="module")
def bench():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    import bench as b
    return b


def test_pml_absorbs_and_converges(bench):
    coarse = bench.run_reflection(n=8, p=2, chunks=4)
    walls = bench.run_reflection(n=8, p=2, chunks=4, sigma_max=0.0)
    fine = bench.run_reflection(n=16, p=4, chunks=4)
    assert walls["reflection"] > 5 * coarse["reflection"]
    assert fine["reflection"] < coarse["reflection"] / 10
    assert fine["reflection"] < 2e-3
