"""GPU parity of the right-hand side (dgm_rhs through the C ABI) with the oracle.

Element-by-element comparison on seeded inputs at sizes the oracle finishes
in seconds, spanning several CTA tiles with a ragged tail (162 elements =
5 x 32 + 2 = 10 x 16 + 2 columns), every supported order, both fluxes,
heterogeneous materials, several batch columns, PML auxiliaries and point
sources.  Tolerances: FP64 1e-12 and FP32 1e-5 relative to the max-norm of
the oracle's result.
"""
import numpy as np
import pytest

import workloads as W
from oracle_ref import build, rel_err, rhs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _mesh(n=3, jitter=0.15, seed=11, lo=(0, 0, 0), hi=(1, 1, 1)):
    xyz, tets = W.kuhn_mesh(n, lo, hi, jitter, seed)
    K = len(tets)
    eps = W.lognormal_material(K, 2.0, 0.3, seed + 1)
    mu = W.lognormal_material(K, 1.2, 0.2, seed + 2)
    return xyz, tets, eps, mu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("flux", ["upwind", "central"])
def test_rhs_matches_oracle(D, prec, p, flux):
    xyz, tets, eps, mu = _mesh()
    S = 3 if p <= 2 else 1
    u = W.random_state(len(tets), S, p, seed=100 + p)
    g = D.Solver(xyz, tets, eps, mu, p, prec, flux, "lsrk4", 1e-3, S=S)
    got = g.from_device(g.rhs(u))
    ref, _ = rhs(build(xyz, tets, p, eps, mu, flux, S=S), u)
    assert rel_err(got, ref) < TOL[prec]


def test_rhs_p5_fp32(D):
    xyz, tets, eps, mu = _mesh(n=2)
    u = W.random_state(len(tets), 1, 5, seed=5)
    g = D.Solver(xyz, tets, eps, mu, 5, "fp32", "upwind", "lsrk4", 1e-3)
    got = g.from_device(g.rhs(u))
    ref, _ = rhs(build(xyz, tets, 5, eps, mu, "upwind"), u)
    assert rel_err(got, ref) < TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_element_all_walls(D, prec):
    xyz = np.array([[0.1, 0.0, 0.0], [1.0, 0.2, 0.1], [0.0, 0.9, 0.2], [0.3, 0.1, 1.1]])
    tets = np.array([[2, 0, 3, 1]])
    u = W.random_state(1, 2, 3, seed=1)
    g = D.Solver(xyz, tets, 3.0, 2.0, 3, prec, "upwind", "lsrk4", 1e-3, S=2)
    got = g.from_device(g.rhs(u))
    ref, _ = rhs(build(xyz, tets, 3, 3.0, 2.0, "upwind", S=2), u)
    assert rel_err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rhs_with_pml(D, prec):
    xyz, tets, eps, mu = _mesh(n=4, jitter=0.0, lo=(-1, -1, -1), hi=(1, 1, 1))
    pml = dict(lo=(-0.45,) * 3, hi=(0.45,) * 3, thickness=0.55, sigma_max=12.0, order=2)
    K, p, S = len(tets), 2, 2
    u = W.random_state(K, S, p, seed=7)
    aux = W.random_state(K, S, p, seed=8)
    g = D.Solver(xyz, tets, eps, mu, p, prec, "upwind", "lsrk4", 1e-3, S=S, pml=pml)
    idx = g.pml_elements()
    assert 0 < len(idx) < K
    aux[np.setdiff1d(np.arange(K), idx)] = 0.0
    du, daux = g.rhs(u, g.aux_to_device(aux))
    ref_u, ref_a = rhs(build(xyz, tets, p, eps, mu, "upwind", pml=pml, S=S), u, aux)
    assert rel_err(g.from_device(du), ref_u) < TOL[prec]
    assert rel_err(g.from_device(daux), ref_a[idx]) < TOL[prec]
    assert np.abs(np.delete(ref_a, idx, axis=0)).max() == 0.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rhs_with_dipoles(D, prec):
    xyz, tets, eps, mu = _mesh(n=3)
    K, p, S = len(tets), 3, 3
    srcs = [W.dipole((0.41, 0.52, 0.33), 2.0, 1.0), None,
            W.dipole((0.7, 0.2, 0.6), 1.5, 0.8, direction=(0.3, -0.2, 0.9))]
    u = W.random_state(K, S, p, seed=9)
    g = D.Solver(xyz, tets, eps, mu, p, prec, "upwind", "lsrk4", 1e-3, S=S)
    g.set_sources(srcs)
    for t in (0.31, 0.45):
        got = g.from_device(g.rhs(u, t=t))
        ref, _ = rhs(build(xyz, tets, p, eps, mu, "upwind", S=S, sources=srcs), u, t=t)
        assert rel_err(got, ref) < TOL[prec]
        u0 = np.zeros_like(u)   # source-only response is non-trivial
        assert np.abs(g.from_device(g.rhs(u0, t=t))).max() > 1e-3


def test_status_word_is_clean(D):
    xyz, tets, eps, mu = _mesh(n=2)
    g = D.Solver(xyz, tets, eps, mu, 2, "fp64", "upwind", "lsrk4", 1e-3)
    g.rhs(W.random_state(len(tets), 1, 2, seed=1))
    g.status()
