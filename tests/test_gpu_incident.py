"""Incident faces on the GPU (dgm_set_incident: Sec. V's plane-wave source,
entering through tagged boundary faces with the exterior state
e+ = e- + 2 E_inc, h+ = -h-) against the oracle's assembly of the same ghost
state (tests/test_oracle_incident.py pins it to an analytic TEM pulse).

* Right-hand side, element by element: the forcing alone (zero state) and on
  a random state with point sources, p = 1..3, both fluxes, FP64 and FP32,
  jittered geometry, element-wise materials, incident faces on two sides of
  the box, an oblique wave with a polarisation that is not transverse (every
  covariant component is exercised).  The pulse is smooth on the faces, so
  both sides' face rules are converged: the GPU's (p + 6)^2-point rule and
  the oracle's 16^2-point rule agree to rounding.
* An LSRK4 trajectory from rest (stage times c_k dt), upwind.
* Physics on the GPU alone: a TEM pulse injected into a parallel-plate slab
  arrives with the analytic shape (0.3 % on an 8^3 grid, p = 2, FP32).
* The paired FP32 variants are skipped by the autotuner and refused.

Tolerances: FP64 1e-12 and FP32 1e-5 of the oracle's max-norm.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.assemble import Assembly
from oracle.mesh import Mesh
from oracle.solver import Solver
from oracle_ref import rel_err, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
D3 = np.array([0.3, 0.2, 0.93]) / np.linalg.norm([0.3, 0.2, 0.93])
WAVE = dict(E0=(0.8, -0.3, 0.45), direction=tuple(D3), speed=0.9, f0=0.3, bw=0.25, t0=0.4)


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _case(p, flux, S=2, seed=0, sources=True):
    n = 3
    xyz, tets = W.kuhn_mesh(n, jitter=0.12, seed=31 + seed)
    K = len(tets)
    eps = W.lognormal_material(K, 2.0, 0.3, 32 + seed)
    mu = W.lognormal_material(K, 1.0, 0.2, 33 + seed)
    faces = np.concatenate([W.box_faces(n, tets, 2, 0), W.box_faces(n, tets, 0, 1)])
    srcs = ([W.dipole((0.41, 0.37, 0.55), 2.0, 1.0), None][:S]) if sources else None
    a = Assembly(Mesh(xyz, tets), p, eps, mu, flux, incident=faces)
    o = Solver(a, S=S, sources=srcs)
    w = WAVE
    o.set_incident(w["E0"], w["direction"], w["speed"], w["f0"], w["bw"], w["t0"], quad=16)
    return xyz, tets, eps, mu, faces, srcs, o


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["upwind", "central"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_incident_rhs_matches_oracle(D, p, flux, prec):
    xyz, tets, eps, mu, faces, srcs, o = _case(p, flux)
    g = D.Solver(xyz, tets, eps, mu, p, prec, flux, "lsrk4", 1e-3, S=2)
    g.set_sources(srcs)
    g.set_incident(faces, **WAVE)
    K, N = len(tets), W.n_modes(p)
    t = 0.55
    zero = np.zeros((K, 2, 6, N))
    got0 = g.from_device(g.rhs(zero, t=t))
    ref0 = o.unpack(o.rhs(o.pack(zero), t))[0]
    assert np.abs(ref0).max() > 0.1                  # the wave is on the faces at t
    assert rel_err(got0, ref0) < TOL[prec]
    u = W.random_state(K, 2, p, seed=40 + p)
    got = g.from_device(g.rhs(u, t=t))
    ref = o.unpack(o.rhs(o.pack(u), t))[0]
    assert rel_err(got, ref) < TOL[prec]
    # n = 0 restores PEC: from rest only the point source is left
    g.set_incident([], **WAVE)
    o.inc = None
    ref_src = o.unpack(o.rhs(o.pack(zero), t))[0]
    assert np.abs(ref_src).max() > 0
    assert rel_err(g.from_device(g.rhs(zero, t=t)), ref_src) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_incident_lsrk4_trajectory(D, prec):
    p = 2
    xyz, tets, eps, mu, faces, srcs, o = _case(p, "upwind", S=1, seed=3, sources=False)
    dt = W.stable_dt(1 / 3, p) / 2
    g = D.Solver(xyz, tets, eps, mu, p, prec, "upwind", "lsrk4", dt, S=1)
    g.set_incident(faces, **WAVE)
    K, N = len(tets), W.n_modes(p)
    g.set_state(np.zeros((K, 1, 6, N)))
    steps, t0 = 40, 0.1
    g.advance(steps, t0)
    got = g.state()
    ref = o.unpack(o.lsrk4(np.zeros((o.asm.ndof, 1)), t0, dt, steps))[0]
    assert np.abs(ref).max() > 0.05
    assert rel_l2(got, ref) < TOL[prec] and rel_err(got, ref) < 10 * TOL[prec]


def test_tem_pulse_arrives_with_the_analytic_shape(D):
    """E = x g(t - z), H = y g(t - z) between the plates x = 0, 0.5, injected
    through z = 0 of a slab long in y; compared in the middle of the slab
    before the pulse reaches the far wall or the side walls' disturbance
    reaches the middle."""
    n, p = 8, 2
    lo, hi = (0, -1, 0), (0.5, 1.5, 1)
    xyz, tets = W.kuhn_mesh(n, lo, hi)
    faces = W.box_faces(n, tets, 2, 0)
    sig, t0, T = 0.15, 0.6, 1.0
    dt0 = 0.3 * min((np.array(hi) - np.array(lo)) / n) / (p + 1) ** 2
    steps = int(round(T / dt0))
    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", T / steps)
    g.set_incident(faces, E0=(1, 0, 0), direction=(0, 0, 1), speed=1.0, f0=0.0,
                   bw=1.0 / (2 * math.pi * sig), t0=t0)
    g.set_state(np.zeros((len(tets), 1, 6, W.n_modes(p))))
    g.advance(steps, 0.0)
    got = g.state()[:, 0]
    g.status()
    pulse = lambda r: np.exp(-(T - t0 - r[:, 2]) ** 2 / (2 * sig * sig))
    z = lambda r: 0.0 * r[:, 0]
    g.project(lambda r: np.stack([pulse(r), z(r), z(r), z(r), pulse(r), z(r)], axis=1))
    want = g.state()[:, 0]
    c = W.centroids(xyz, tets)
    mid = (c[:, 1] > 0.0) & (c[:, 1] < 0.5)
    e_err = np.linalg.norm(got[mid, 0:3] - want[mid, 0:3]) / np.linalg.norm(want[mid, 0:3])
    h_err = np.linalg.norm(got[mid, 3:6] - want[mid, 3:6]) / np.linalg.norm(want[mid, 3:6])
    assert e_err < 0.006 and h_err < 0.006, (e_err, h_err)


def test_paired_variants_are_skipped(D):
    xyz, tets = W.kuhn_mesh(4)
    g = D.Solver(xyz, tets, 1.0, 1.0, 3, "fp32", "upwind", "lsrk4", 1e-3)
    g.set_incident(W.box_faces(4, tets, 2, 0), **WAVE)
    v, ms = g.autotune(reps=2)
    assert v not in (3, 4) and ms[3] == 0 and ms[4] == 0
    with pytest.raises(D.DgmError):
        g.set_variant(3)
