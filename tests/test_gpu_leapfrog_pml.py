"""Leapfrog with the PML's dissipative terms by the trapezoid rule (Sec. V) on
the GPU against the oracle's leapfrog_pml: E and the H-equation auxiliary q
at integer steps, H and the E-equation auxiliary p half a step later, central
flux, a dipole source, element-wise materials, S = 2 columns."""
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


_REF = {}


def _case(p):
    if p not in _REF:
        xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=91)
        K, S = len(tets), 2
        eps = W.lognormal_material(K, 1.5, 0.2, 92)
        mu = W.lognormal_material(K, 1.0, 0.1, 93)
        pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
        srcs = [W.dipole((0.1, -0.05, 0.08), 2.0, 1.0), None]
        dt = W.stable_dt(2 / 3, p)
        u = W.random_state(K, S, p, seed=94) * 1e-2
        aux = W.random_state(K, S, p, seed=95) * 1e-3
        o = build(xyz, tets, p, eps, mu, "central", pml=pml, S=S, sources=srcs)
        pml_el = np.any(o.asm.sigma != 0, axis=1)
        aux[~pml_el] = 0.0                     # auxiliaries live in the layer only
        steps = 40
        ref, ref_aux = o.unpack(o.leapfrog_pml(o.pack(u, aux), 0.0, dt, steps))
        _REF[p] = (xyz, tets, eps, mu, pml, srcs, dt, u, aux, steps, ref, ref_aux)
    return _REF[p]


@pytest.mark.parametrize("p,prec,tol", [(2, "fp64", 1e-12), (2, "fp32", 1e-5), (3, "fp64", 1e-12),
                                        (3, "fp32", 1e-5)])
def test_leapfrog_pml_matches_oracle(D, p, prec, tol):
    xyz, tets, eps, mu, pml, srcs, dt, u, aux, steps, ref, ref_aux = _case(p)
    g = D.Solver(xyz, tets, eps, mu, p, prec, "central", "leapfrog", dt, S=2, pml=pml)
    assert 0 < g.npml < g.K
    g.set_sources(srcs)
    g.set_state(u, aux[g.pml_elements()])
    g.leapfrog_start(0.0)
    g.advance(steps, 0.0)
    got = g.state()
    got_aux = g.from_device(g.aux[g.current()])
    assert rel_l2(got, ref) < tol and rel_err(got, ref) < 10 * tol
    ra = ref_aux[g.pml_elements()]
    assert rel_l2(got_aux, ra) < tol and rel_err(got_aux, ra) < 10 * tol
