"""Interior penalty with a facet field on the GPU (dgm_set_sip; Sec. III,
Eqs. (jmp_var_def), (1st_weak_equation), (weak_penalty)) against the oracle's
extended system (tests/test_oracle_sip.py pins it).

The GPU stores h_s as physical components per face mode of its own face
basis, the oracle in tangent-times-polynomial coefficients of its own facet
basis; both describe the same field, so the facet field is compared through
basis-free quantities per facet: its L2 norm squared and its integral (a
vector), each over the facet.  The fields e, h are compared element by
element.

* The facet field's time derivative from rest (random e, h): p = 1..3, FP64
  and FP32, jittered geometry, element-wise eps and mu (mu_F the mean of the
  two sides), two columns.
* LSRK4 trajectories of the extended system from random e, h with a dipole
  source, where h_s grows from zero and feeds back into E: fields element by
  element, facet norms and integrals, and the extended energy.
* Zero penalty (alpha = 0) is the plain central flux, bit for bit.

Tolerances: FP64 1e-12 and FP32 1e-5, relative to the oracle's largest entry.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.sip import SipSolver
from oracle.solver import Solver
from oracle_ref import rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
ALPHA = 4.0


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _case(p, S=2, seed=0, sources=True):
    xyz, tets = W.kuhn_mesh(3, jitter=0.12, seed=61 + seed)
    K = len(tets)
    eps = W.lognormal_material(K, 2.0, 0.3, 62 + seed)
    mu = W.lognormal_material(K, 1.2, 0.2, 63 + seed)
    srcs = [W.dipole((0.41, 0.37, 0.55), 2.0, 1.0), None][:S] if sources else None
    o = SipSolver(Solver(Assembly(Mesh(xyz, tets), p, eps, mu, "central"), S=S, sources=srcs), ALPHA)
    return xyz, tets, eps, mu, srcs, o


def _gpu_facet_moments(o, hs):
    """GPU facet field (nF, S, 3, NF), reference-orthonormal face modes ->
    (int_F |h_s|^2, int_F h_s): 2|F| sum |X_m|^2 and sqrt(2) |F| X_0."""
    area = np.array([fr[2] for fr in o.sip.frames])
    norm2 = 2.0 * area[:, None] * np.sum(hs * hs, axis=(2, 3))
    mean = math.sqrt(2.0) * area[:, None, None] * hs[:, :, :, 0]
    return norm2, mean


def _oracle_facet_moments(o, x):
    norm2, mean = o.sip.facet_moments(x)
    return norm2, mean


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_facet_field_rate_from_rest(D, p, prec):
    xyz, tets, eps, mu, srcs, o = _case(p)
    g = D.Solver(xyz, tets, eps, mu, p, prec, "central", "lsrk4", 1e-3, S=2, sip=ALPHA)
    assert g.info.n_facets == o.sip.nF
    g.set_sources(srcs)
    u = W.random_state(len(tets), 2, p, seed=70 + p)
    t = 0.3
    du = g.from_device(g.rhs(u, t=t))
    dhs = g.facet_rhs()
    y = o.rhs(o.pack(u), t)
    ref_u, ref_s = o.unpack(y)
    assert rel_err(du, ref_u) < TOL[prec]               # h_s = 0: the plain central flux
    n2g, mg = _gpu_facet_moments(o, dhs)
    yx = o.pack(np.zeros_like(u), ref_s)
    n2o, mo = _oracle_facet_moments(o, yx)
    assert np.abs(n2o).max() > 1e-3
    assert rel_err(n2g, n2o) < 10 * TOL[prec]
    assert rel_err(mg, mo) < TOL[prec]


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_extended_lsrk4_trajectory(D, p, prec):
    xyz, tets, eps, mu, srcs, o = _case(p, seed=2)
    dt = W.stable_dt(1 / 3, p) / 2
    g = D.Solver(xyz, tets, eps, mu, p, prec, "central", "lsrk4", dt, S=2, sip=ALPHA)
    g.set_sources(srcs)
    u = W.random_state(len(tets), 2, p, seed=80 + p)
    g.set_state(u)
    steps = 20
    g.advance(steps, 0.0)
    got_u, got_s = g.state(), g.facet_state()
    x = o.lsrk4(o.pack(u), 0.0, dt, steps)
    ref_u, _ = o.unpack(x)
    assert rel_err(got_u, ref_u) < 10 * TOL[prec]
    n2g, mg = _gpu_facet_moments(o, got_s)
    n2o, mo = _oracle_facet_moments(o, x)
    assert np.abs(mo).max() > 1e-3                      # the facet field is active
    assert rel_err(n2g, n2o) < 10 * TOL[prec]
    assert rel_err(mg, mo) < 10 * TOL[prec]
    # extended energy: fields (the library's reduction) + facets
    mu_F = o.sip.mu_F
    facet_e = 0.5 * np.sum((mu_F / ALPHA)[:, None] * n2g, axis=0)
    assert np.allclose(g.energy() + facet_e, o.sip.energy(x), rtol=10 * TOL[prec], atol=0)


def test_zero_penalty_is_the_central_flux(D):
    p = 2
    xyz, tets, eps, mu, srcs, o = _case(p)
    dt = W.stable_dt(1 / 3, p) / 2
    u = W.random_state(len(tets), 2, p, seed=5)
    out = []
    for kw in (dict(sip=None), dict(sip=0.0)):
        g = D.Solver(xyz, tets, eps, mu, p, "fp64", "central", "lsrk4", dt, S=2, **kw)
        g.set_state(u)
        g.advance(5, 0.0)
        out.append(g.state())
    assert np.array_equal(out[0], out[1])


def test_paired_variants_skipped_with_the_penalty(D):
    xyz, tets = W.kuhn_mesh(4)
    g = D.Solver(xyz, tets, 1.0, 1.0, 3, "fp32", "central", "lsrk4", 1e-3, sip=ALPHA)
    v, ms = g.autotune(reps=2)
    assert v not in (3, 4) and ms[3] == 0 and ms[4] == 0
