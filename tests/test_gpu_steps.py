"""GPU parity of time stepping, energy, projection and the host end-to-end call.

LSRK4 (five 2N-storage stages per step, upwind flux, PML, sources) and
staggered leapfrog (central flux) trajectories are compared with the oracle
after several steps; the FP64 energy reduction and the L2 projection of an
initial field are compared with the oracle's assembled-matrix values.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle_ref import build, rel_err, rel_l2
from oracle.solver import Solver as OSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2002_08733_gb300 import build as B, dgmax
    B.build()
    dgmax.load_library()
    return dgmax


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_lsrk4_trajectory(D, prec, tol):
    xyz, tets = W.kuhn_mesh(3, jitter=0.15, seed=21)
    K, p, S = len(tets), 3, 2
    eps = W.sphere_material(xyz, tets, (0.5, 0.5, 0.5), 0.3, 4.0, 1.0)
    dt = W.stable_dt(1 / 3, p)
    u = W.random_state(K, S, p, seed=22)
    g = D.Solver(xyz, tets, eps, 1.0, p, prec, "upwind", "lsrk4", dt, S=S)
    g.set_state(u)
    g.advance(12, 0.0)
    got = g.state()
    o = build(xyz, tets, p, eps, 1.0, "upwind", S=S)
    ref = o.unpack(o.lsrk4(o.pack(u), 0.0, dt, 12))[0]
    assert rel_l2(got, ref) < tol
    assert rel_err(got, ref) < 10 * tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("S", [1, 2, 3])
def test_lsrk4_tile_load_paths(D, prec, tol, S):
    """With C = 162 S columns a row starts on a 16-byte boundary for some S
    (FP32: S = 2; FP64: every S) and not for others (FP32: S = 1, 3), and the
    last tile is ragged.  Phase 1 moves the tile with tiled bulk copies only
    for FP64 at S = 1 (one column per element, aligned rows); every other case
    here takes per-thread loads (tests/test_gpu_bulk.py compares the two
    paths).  Six LSRK4 steps with PML auxiliaries and a source in column 0
    match the oracle for each S."""
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=23)
    K, p = len(tets), 2
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.11, -0.07, 0.05), 2.0, 1.0)] + [None] * (S - 1)
    dt = W.stable_dt(2 / 3, p)
    u = W.random_state(K, S, p, seed=24) * 1e-2
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
    g.set_sources(srcs)
    g.set_state(u)
    g.advance(6, 0.0)
    got = g.state()
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=pml, S=S, sources=srcs)
    ref, ref_aux = o.unpack(o.lsrk4(o.pack(u, np.zeros_like(u)), 0.0, dt, 6))
    assert rel_l2(got, ref) < tol
    ga = g.from_device(g.aux[g.current()])
    assert rel_l2(ga, ref_aux[g.pml_elements()]) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("S", [1, 2])
def test_index_width_paths(D, prec, tol, S):
    """The stage kernels use 32-bit index arithmetic when every index fits and
    64-bit otherwise; forcing the 64-bit kernels on a small problem must give
    the same results bit for bit (five LSRK4 steps and one right-hand side,
    with PML, a source and S columns), and both match the oracle."""
    xyz, tets = W.kuhn_mesh(3, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=25)
    K, p = len(tets), 2
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.11, -0.07, 0.05), 2.0, 1.0)] + [None] * (S - 1)
    dt = W.stable_dt(2 / 3, p)
    u = W.random_state(K, S, p, seed=26) * 1e-2
    got = []
    for force in (False, True):
        g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
        if force:
            g.set_index64(True)
        g.set_sources(srcs)
        du, dad = g.rhs(u)
        g.set_state(u)
        g.advance(5, 0.0)
        got.append([g.state(), g.from_device(g.aux[g.current()]), g.from_device(du),
                    g.from_device(dad)])
    for a, b in zip(got[0], got[1]):
        assert np.array_equal(a, b)
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=pml, S=S, sources=srcs)
    ref, ref_aux = o.unpack(o.lsrk4(o.pack(u, np.zeros_like(u)), 0.0, dt, 5))
    assert rel_l2(got[0][0], ref) < tol
    assert rel_l2(got[0][1], ref_aux[g.pml_elements()]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tile_order_does_not_change_results(D, prec):
    """The tile visiting order (dgm_set_tile_groups) is a scheduling choice:
    plain order, interleaved groups that divide the tile count and a count
    that does not (plain order then) give bit-identical LSRK4 steps with PML
    and a source; the autotuner's choice is one of its candidates."""
    xyz, tets = W.kuhn_mesh(4, (-1, -1, -1), (1, 1, 1), jitter=0.1, seed=27)
    K, p, S = len(tets), 2, 2
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.11, -0.07, 0.05), 2.0, 1.0), None]
    dt = W.stable_dt(0.5, p)
    u = W.random_state(K, S, p, seed=28) * 1e-2
    got = []
    for groups in (1, 2, 6, 8, 5):
        g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
        g.set_tile_groups(groups)
        assert g.tile_groups() == groups
        g.set_sources(srcs)
        g.set_state(u)
        g.advance(4, 0.0)
        got.append((g.state(), g.from_device(g.aux[g.current()])))
    for st, ax in got[1:]:
        assert np.array_equal(st, got[0][0]) and np.array_equal(ax, got[0][1])
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
    g.autotune()
    assert g.tile_groups() in (1, 2, 3, 4, 6, 8, 12)
    with pytest.raises(D.DgmError):
        g.set_tile_groups(0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_lsrk4_pml_dipole_trajectory(D, prec, tol):
    xyz, tets = W.kuhn_mesh(4, (-1, -1, -1), (1, 1, 1))
    K, p, S = len(tets), 2, 1
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=20.0, order=2)
    srcs = [W.dipole((0.11, -0.07, 0.05), 2.0, 1.0)]
    dt = W.stable_dt(0.5, p)
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", dt, S=S, pml=pml)
    g.set_sources(srcs)
    g.advance(40, 0.0)
    got = g.state()
    o = build(xyz, tets, p, 1.0, 1.0, "upwind", pml=pml, S=S, sources=srcs)
    x = o.lsrk4(np.zeros((o.asm.ndof, S)), 0.0, dt, 40)
    ref, ref_aux = o.unpack(x)
    assert np.abs(ref).max() > 1e-4
    assert rel_l2(got, ref) < tol
    ga = g.from_device(g.aux[g.current()])
    assert rel_l2(ga, ref_aux[g.pml_elements()]) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_leapfrog_cavity_trajectory(D, prec, tol):
    xyz, tets = W.kuhn_mesh(3)
    K, p = len(tets), 2
    dt = W.stable_dt(1 / 3, p)
    u = W.random_state(K, 1, p, seed=31)
    g = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "central", "leapfrog", dt)
    g.set_state(u)
    g.leapfrog_start(0.0)
    g.advance(25, 0.0)
    got = g.state()
    o = build(xyz, tets, p, 1.0, 1.0, "central")
    ref = o.unpack(o.leapfrog(o.pack(u), 0.0, dt, 25))[0]
    assert rel_l2(got, ref) < tol


def test_energy_matches_oracle(D):
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=3)
    K, p, S = len(tets), 3, 4
    eps = W.lognormal_material(K, 2.0, 0.3, 4)
    mu = W.lognormal_material(K, 1.0, 0.2, 5)
    u = W.random_state(K, S, p, seed=6)
    g = D.Solver(xyz, tets, eps, mu, p, "fp64", "upwind", "lsrk4", 1e-3, S=S)
    g.set_state(u)
    o = build(xyz, tets, p, eps, mu, "upwind", S=S)
    ref = o.asm.energy(o.pack(u))
    got = g.energy()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_central_flux_energy_is_conserved_on_gpu(D):
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=8)
    p = 3
    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp64", "central", "lsrk4", 2e-3)
    g.set_state(W.random_state(len(tets), 1, p, seed=9))
    w0 = g.energy()[0]
    g.advance(50)
    w1 = g.energy()[0]
    assert abs(w1 - w0) < 1e-6 * w0     # LSRK4 damping of a skew operator is O(dt^5)


def test_upwind_energy_decays_on_gpu(D):
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=8)
    g = D.Solver(xyz, tets, 1.0, 1.0, 2, "fp32", "upwind", "lsrk4", 2e-3)
    g.set_state(W.random_state(len(tets), 1, 2, seed=9))
    w = [g.energy()[0]]
    for _ in range(5):
        g.advance(10)
        w.append(g.energy()[0])
    assert all(b < a for a, b in zip(w, w[1:]))


def test_projection_matches_oracle(D):
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=12)
    p = 3

    def field(r):
        out = np.zeros((len(r), 6))
        out[:, 2] = np.sin(math.pi * r[:, 0]) * np.sin(math.pi * r[:, 1])
        out[:, 3] = np.cos(2 * r[:, 2]) * r[:, 0]
        out[:, 4] = np.exp(-((r - 0.4) ** 2).sum(axis=1) / 0.1)
        return out

    g = D.Solver(xyz, tets, 1.0, 1.0, p, "fp64", "upwind", "lsrk4", 1e-3)
    g.project(field)
    got = g.state()[:, 0]
    o = build(xyz, tets, p, 1.0, 1.0, "upwind")
    # the oracle projects with its own quadrature (one degree higher), so for a
    # non-polynomial field the two agree only to the quadrature error (~1e-5 here)
    ref_e = o.project(lambda r: field(r)[:, 0:3], "E")
    ref_h = o.project(lambda r: field(r)[:, 3:6], "H")
    ref = np.concatenate([ref_e, ref_h], axis=1)
    assert rel_err(got, ref) < 1e-4
    # on a polynomial field of degree p both are exact
    poly = lambda r: np.stack([r[:, 0] * r[:, 1], r[:, 2] ** 2, r[:, 0] ** 3, 1 + r[:, 1],
                               r[:, 2] * r[:, 0], r[:, 1] ** 2 * r[:, 2]], axis=1)
    g.project(poly)
    got = g.state()[:, 0]
    ref = np.concatenate([o.project(lambda r: poly(r)[:, 0:3], "E"),
                          o.project(lambda r: poly(r)[:, 3:6], "H")], axis=1)
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_end_to_end_matches_device_path(D, prec):
    import torch
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=14)
    p = 2
    u = W.random_state(len(tets), 1, p, seed=15)
    a = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3)
    a.set_state(u)
    a.advance(7)
    want = a.fields[a.current()].cpu()
    b = D.Solver(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3)
    hin = b.to_device(u).cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    b.advance_host(hin, hout, 7)
    assert torch.equal(hout, want)
