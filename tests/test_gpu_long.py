"""GPU parity over the full step counts of the benchmarked workloads.

Each workload's physics runs on a replica mesh small enough for the oracle
to step it in seconds: the same degree, flux, integrator, materials,
sources, PML and -- so that the arithmetic per step is the same -- the same
time step and step count as the full-size workload.  Only the mesh size
differs.

* jittered sphere: 3^3 jittered Kuhn grid (162 tets), p = 3, eps = 4 sphere,
  upwind, LSRK4, Gaussian pulse, dt = 5.859e-4, 1000 steps;
* dipole in a PML: [-1,1]^3 on a 2^3 grid (48 tets), p = 4, z dipole f0 = 2,
  from rest, dt = 6e-4, 2000 steps; the quadratic layer (sigma_max 40) starts
  at |x| = 0.6 and is 0.4 thick, so that the replica's centroids (at 0.25,
  0.5, 0.75 of a unit cube) fall in it -- with the full workload's 0.25-thick
  layer at 0.75 no replica element would be damped;
* inverse problem (forward records): [-1,1]^3 on a 2^3 grid, p = 3, the
  same PML, lognormal eps, 8 dipole columns, 32 receivers recording E after
  every step, dt = 1.5625e-3, 1500 steps.

Errors are measured at checkpoints relative to the largest oracle norm seen
up to then (the dipole runs start from rest, so the first checkpoints'
own norms say little): relative L2 over the whole state and the
element-wise maximum relative to the largest entry.  Bars: FP64 1e-12,
FP32 1e-5.
"""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import Receivers
from oracle_ref import build

pytestmark = pytest.mark.gpu

CHECKS = 4          # checkpoints per run


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


def _compare(traj_got, traj_ref, tol):
    """Worst relative L2 and relative element-wise error over the checkpoints,
    both against the largest reference norm (or entry) seen so far."""
    worst_l2 = worst_max = 0.0
    peak_l2 = peak_max = 0.0
    for got, ref in zip(traj_got, traj_ref):
        peak_l2 = max(peak_l2, float(np.linalg.norm(ref)))
        peak_max = max(peak_max, float(np.abs(ref).max()))
        worst_l2 = max(worst_l2, float(np.linalg.norm(got - ref)) / peak_l2)
        worst_max = max(worst_max, float(np.abs(got - ref).max()) / peak_max)
    return worst_l2, worst_max


# -- jittered sphere -------------------------------------------------------------
@pytest.fixture(scope="module")
def sphere_case():
    full = W.jittered_sphere()
    w = W.jittered_sphere(n=3)
    xyz, tets = w.mesh()
    c, r, ein, eout = w.extra["sphere"]
    eps = W.sphere_material(xyz, tets, c, r, ein, eout)
    assert 0 < int((eps == ein).sum()) < len(tets)
    o = build(xyz, tets, w.p, eps, 1.0, w.flux)
    r0 = np.asarray(full.extra["r0"])
    ey = o.project(lambda q: np.stack([0 * q[:, 0], np.exp(-((q - r0) ** 2).sum(1) / 0.01),
                                       0 * q[:, 0]], axis=1), "E")
    u0 = np.zeros((len(tets), 1, 6, w.N))
    u0[:, 0, 0:3] = ey
    steps, dt = full.steps, full.dt
    per = steps // CHECKS
    x, traj = o.pack(u0), []
    for k in range(CHECKS):
        x = o.lsrk4(x, k * per * dt, dt, per)
        traj.append(o.unpack(x)[0])
    return dict(xyz=xyz, tets=tets, eps=eps, p=w.p, u0=u0, dt=dt, per=per, traj=traj)


@pytest.mark.parametrize("prec,tol,variant", [("fp64", 1e-12, None), ("fp32", 1e-5, None),
                                              ("fp32", 1e-5, 5)])
def test_jittered_sphere_1000_steps(D, sphere_case, prec, tol, variant):
    """variant None: the autotuner's choice; 5: the tensor-core variant (curl and
    lift as three TF32 products per pair on tcgen05)."""
    c = sphere_case
    g = D.Solver(c["xyz"], c["tets"], c["eps"], 1.0, c["p"], prec, "upwind", "lsrk4", c["dt"])
    if variant is not None:
        g.set_variant(variant)
    elif prec == "fp32":
        g.autotune()
    g.set_state(c["u0"])
    got = []
    for k in range(CHECKS):
        g.advance(c["per"], k * c["per"] * c["dt"])
        got.append(g.state())
    l2, mx = _compare(got, c["traj"], tol)
    assert l2 < tol, (l2, mx)
    assert mx < 10 * tol, (l2, mx)


# -- dipole in a PML -----------------------------------------------------------------
PML = dict(lo=(-0.6,) * 3, hi=(0.6,) * 3, thickness=0.4, sigma_max=40.0, order=2)


@pytest.fixture(scope="module")
def dipole_case():
    full = W.dipole_pml()
    xyz, tets = W.kuhn_mesh(2, (-1, -1, -1), (1, 1, 1))
    p = full.p
    src = [W.dipole((0.13, -0.21, 0.08), 2.0, 1.0)]
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=PML, sources=src)
    steps, dt = full.steps, full.dt
    per = steps // CHECKS
    x, traj, traj_aux = np.zeros((o.asm.ndof, 1)), [], []
    for k in range(CHECKS):
        x = o.lsrk4(x, k * per * dt, dt, per)
        u, aux = o.unpack(x)
        traj.append(u)
        traj_aux.append(aux)
    return dict(xyz=xyz, tets=tets, p=p, src=src, dt=dt, per=per, traj=traj, traj_aux=traj_aux)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_dipole_pml_2000_steps(D, dipole_case, prec, tol):
    c = dipole_case
    g = D.Solver(c["xyz"], c["tets"], 1.0, 1.0, c["p"], prec, "upwind", "lsrk4", c["dt"],
                 pml=PML)
    assert 0 < g.npml < g.K
    g.set_sources(c["src"])
    if prec == "fp32":
        g.autotune()
    got, got_aux = [], []
    for k in range(CHECKS):
        g.advance(c["per"], k * c["per"] * c["dt"])
        got.append(g.state())
        got_aux.append(g.from_device(g.aux[g.current()]))
    idx = g.pml_elements()
    l2, mx = _compare(got, c["traj"], tol)
    assert l2 < tol, (l2, mx)
    assert mx < 10 * tol, (l2, mx)
    l2a, mxa = _compare(got_aux, [a[idx] for a in c["traj_aux"]], tol)
    assert l2a < tol, (l2a, mxa)


# -- inverse problem: forward records --------------------------------------------------
@pytest.fixture(scope="module")
def records_case():
    full = W.inverse_problem()
    xyz, tets = W.kuhn_mesh(2, (-1, -1, -1), (1, 1, 1))
    K, p, S = len(tets), full.p, full.S
    rng = np.random.default_rng(77)
    src = [W.dipole(rng.uniform(-0.6, 0.6, 3), rng.uniform(1.0, 4.0), 1.0) for _ in range(S)]
    rec = rng.uniform(-0.7, 0.7, size=(32, 3))
    eps = W.lognormal_material(K, 2.0, 0.3, 78)
    o = build(xyz, tets, p, eps, 1.0, "upwind", pml=PML, S=S, sources=src)
    R = Receivers(o.asm, rec)
    steps, dt = full.steps, full.dt
    records = []
    x = o.lsrk4(np.zeros((o.asm.ndof, S)), 0.0, dt, steps,
                callback=lambda n, t, xx: records.append(R.sample(xx)))
    return dict(xyz=xyz, tets=tets, p=p, S=S, src=src, rec=rec, eps=eps, dt=dt, steps=steps,
                records=np.array(records), final=o.unpack(x)[0])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_inverse_problem_records_1500_steps(D, records_case, prec, tol):
    c = records_case
    g = D.Solver(c["xyz"], c["tets"], c["eps"], 1.0, c["p"], prec, "upwind", "lsrk4", c["dt"],
                 S=c["S"], pml=PML, max_receivers=len(c["rec"]))
    g.set_sources(c["src"])
    g.set_receivers(c["rec"])
    ws = g.adjoint_workspace(c["steps"])
    got = g.forward_record(c["steps"], 0.0, ws).cpu().numpy()
    ref = c["records"]
    assert got.shape == ref.shape
    peak = np.abs(ref).max()
    # records after every step, each against the largest record so far
    run_peak = np.maximum.accumulate(np.abs(ref).reshape(len(ref), -1).max(axis=1))
    err = np.abs(got - ref).reshape(len(ref), -1).max(axis=1) / np.maximum(run_peak, 1e-300)
    assert err[run_peak > 1e-3 * peak].max() < 10 * tol
    fin = g.state()
    l2, mx = _compare([fin], [c["final"]], tol)
    assert l2 < tol, (l2, mx)
