"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module only *generates inputs*: vertex coordinates and tetrahedra of
structured Kuhn meshes (optionally jittered), per-element material values,
random modal coefficient states, and source/receiver positions.  It contains
none of the discontinuous Galerkin arithmetic (no basis, no quadrature, no
geometric factors, no fluxes); each consumer does its own.

Mesh convention
---------------
The unit cube grid has (n+1)^3 vertices with global id i + (n+1) j + (n+1)^2 k.
Each cube is split into 6 tetrahedra along the paths
v000 -> v000 + e_a -> v000 + e_a + e_b -> v111 for the 6 orderings (a, b, c)
of the axes.  Along such a path the vertex id grows at every step, so each
tetrahedron is emitted with its vertices already in ascending global id.
Tetrahedra are numbered "type-major": id = t * n^3 + cube, cube = ci + n cj +
n^2 ck, t the index of the axis ordering.  With this numbering the neighbour
across a given local face of consecutive elements is itself (mostly)
consecutive in memory, which the GPU path exploits for coalesced loads.

State convention
----------------
A state is an array of shape (K, S, 6, N): element, batch column (source),
field component (Ex, Ey, Ez, Hx, Hy, Hz as covariant coefficients of the
element's mapped modal basis) and mode.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

AXIS_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def n_modes(p: int) -> int:
    """Number of modes of a complete polynomial space of degree p in 3-D."""
    return (p + 1) * (p + 2) * (p + 3) // 6


def n_face_modes(p: int) -> int:
    """Number of modes of a complete polynomial space of degree p in 2-D."""
    return (p + 1) * (p + 2) // 2


def kuhn_mesh(n: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), jitter: float = 0.0,
              seed: int = 0):
    """Structured Kuhn tetrahedral mesh of the box [lo, hi] with n cubes per axis.

    jitter: interior vertices are displaced by U(-jitter*h, +jitter*h) per
    coordinate (h the cube edge along that axis), drawn from
    numpy.random.default_rng(seed).

    Returns (xyz float64 [nv, 3], tets int64 [6 n^3, 4]).
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    h = (hi - lo) / n
    m = n + 1
    idx = np.arange(m)
    I, J, Kk = np.meshgrid(idx, idx, idx, indexing="ij")
    # flatten so that id = i + m j + m^2 k
    I = I.transpose(2, 1, 0).reshape(-1)
    J = J.transpose(2, 1, 0).reshape(-1)
    Kk = Kk.transpose(2, 1, 0).reshape(-1)
    xyz = np.stack([lo[0] + h[0] * I, lo[1] + h[1] * J, lo[2] + h[2] * Kk], axis=1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter, jitter, size=xyz.shape) * h[None, :]
        interior = (I > 0) & (I < n) & (J > 0) & (J < n) & (Kk > 0) & (Kk < n)
        xyz[interior] += d[interior]
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci = ci.transpose(2, 1, 0).reshape(-1)
    cj = cj.transpose(2, 1, 0).reshape(-1)
    ck = ck.transpose(2, 1, 0).reshape(-1)
    base = np.stack([ci, cj, ck], axis=1)
    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((6, n ** 3, 4), dtype=np.int64)
    for t, order in enumerate(AXIS_ORDERS):
        p = base.copy()
        verts = [p.copy()]
        for ax in order:
            p = p + unit[ax]
            verts.append(p.copy())
        for v in range(4):
            q = verts[v]
            tets[t, :, v] = q[:, 0] + m * q[:, 1] + m * m * q[:, 2]
    return xyz, tets.reshape(-1, 4)


def box_faces(n, tets, axis, side):
    """Faces of a kuhn_mesh(n, ...) grid on one side of the box (side 0: the
    `lo` plane, 1: the `hi` plane of `axis`), as vertex-id triples: the faces
    whose three vertices have grid index 0 (or n) along `axis`.  Topology
    only; jitter does not move boundary vertices.  2 n^2 faces."""
    m = n + 1
    tets = np.asarray(tets, dtype=np.int64)
    grid = [tets % m, (tets // m) % m, tets // (m * m)][axis]
    on = grid == (0 if side == 0 else n)
    out = []
    for f in range(4):
        keep = [v for v in range(4) if v != f]
        sel = np.all(on[:, keep], axis=1)
        out.extend(tets[sel][:, keep].tolist())
    return np.asarray(out, dtype=np.int64).reshape(-1, 3)


def centroids(xyz, tets):
    """Arithmetic mean of each tetrahedron's four vertices."""
    return xyz[tets].mean(axis=1)


def sphere_material(xyz, tets, center, radius, inside, outside):
    """Per-element value: `inside` where the centroid lies strictly inside the sphere."""
    c = centroids(xyz, tets)
    d = np.linalg.norm(c - np.asarray(center, dtype=np.float64)[None, :], axis=1)
    return np.where(d < radius, float(inside), float(outside))


def lognormal_material(K, median, sigma, seed):
    """Per-element lognormal values with the given median and log-standard deviation."""
    rng = np.random.default_rng(seed)
    return median * np.exp(sigma * rng.standard_normal(K))


def random_state(K, S, p, seed, decay=1.0, dtype=np.float64):
    """Seeded random modal state of shape (K, S, 6, N).

    Mode l of total degree d is scaled by (1 + d)^-decay so that the state
    resembles a smooth field's coefficients.
    """
    N = n_modes(p)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((K, S, 6, N))
    deg = np.concatenate([np.full((d + 1) * (d + 2) // 2, d) for d in range(p + 1)])
    u *= (1.0 + deg)[None, None, None, :] ** (-decay)
    return u.astype(dtype)


def random_points_in_box(count, lo, hi, seed):
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.uniform(size=(count, 3))


@dataclass
class Workload:
    """One synthetic problem: mesh, materials, order, time stepping and sources."""
    name: str
    n: int
    lo: tuple
    hi: tuple
    p: int
    flux: str            # "central" | "upwind"
    integrator: str      # "leapfrog" | "lsrk4"
    steps: int
    dt: float
    jitter: float = 0.0
    seed: int = 0
    S: int = 1
    pml: dict | None = None
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return 6 * self.n ** 3

    @property
    def N(self):
        return n_modes(self.p)

    def mesh(self):
        return kuhn_mesh(self.n, self.lo, self.hi, self.jitter, self.seed)


def stable_dt(edge, p, cfl=0.3):
    """Time step cfl * h / (p+1)^2 with h the cube edge of the Kuhn grid."""
    return cfl * edge / (p + 1) ** 2


def cavity_tm110(n=4, p=2, steps=200):
    """PEC unit-cube cavity, vacuum, central flux, leapfrog (TM110 initial field)."""
    return Workload("cavity_tm110_n%d_p%d" % (n, p), n, (0, 0, 0), (1, 1, 1), p,
                    "central", "leapfrog", steps, stable_dt(1.0 / n, p))


def jittered_sphere(n=32, p=3, steps=1000, seed=2002):
    """Jittered Kuhn cube [0,1]^3, eps=4 inside a centred sphere of radius 0.25,
    upwind flux, LSRK4, Gaussian pulse E_y = exp(-|r-r0|^2/0.01)."""
    w = Workload("jittered_sphere_n%d_p%d" % (n, p), n, (0, 0, 0), (1, 1, 1), p,
                 "upwind", "lsrk4", steps, stable_dt(1.0 / n, p), jitter=0.15, seed=seed)
    rng = np.random.default_rng(seed + 1)
    w.extra["r0"] = tuple(rng.uniform(0.3, 0.7, size=3))
    w.extra["sphere"] = ((0.5, 0.5, 0.5), 0.25, 4.0, 1.0)
    return w


def dipole_pml(n=40, p=4, steps=2000, seed=2003, thickness=0.25, sigma_max=40.0):
    """Cube [-1,1]^3 with a quadratic-profile PML of the given thickness on all
    faces, z-directed point dipole (Gaussian-modulated sine, f0=2, bw=1)."""
    w = Workload("dipole_pml_n%d_p%d" % (n, p), n, (-1, -1, -1), (1, 1, 1), p,
                 "upwind", "lsrk4", steps, stable_dt(2.0 / n, p), seed=seed,
                 pml=dict(lo=(-1 + thickness,) * 3, hi=(1 - thickness,) * 3,
                          thickness=thickness, sigma_max=sigma_max, order=2))
    inner = 1 - thickness
    rng = np.random.default_rng(seed)
    h = 2.0 / n
    w.extra["sources"] = [dipole(rng.uniform(-inner + 2 * h, inner - 2 * h, size=3), 2.0, 1.0)]
    return w


def dipole(pos, f0, bw, direction=(0.0, 0.0, 1.0)):
    """Point dipole source record: position, direction, centre frequency f0,
    bandwidth bw and envelope delay t0 = 4 s with s = 1/(2 pi bw)."""
    return dict(pos=tuple(float(v) for v in pos), dir=tuple(float(v) for v in direction),
                f0=float(f0), bw=float(bw), t0=4.0 / (2.0 * math.pi * bw))


def batched_sources_and_cavities(seed=2004, n_sources=64, n_cavities=16, n=24, p=3):
    """Batch of many dipole excitations sharing one PML mesh plus uneven cavities.

    Sources: [-1,1]^3 on an n^3 Kuhn grid, degree p, PML 0.25 thick (quadratic
    profile, sigma_max 40), n_sources z-dipoles at seeded interior positions
    with f0 seeded in [1, 4] (bandwidth 1), one per batch column.
    Cavities: unit-cube PEC cavities with n_i seeded in 6..28 and p_i in 2..5,
    vacuum, each with its own dt = 0.3 h_i / (p_i+1)^2, TM110 initial field.
    Upwind flux and LSRK4 everywhere.
    """
    rng = np.random.default_rng(seed)
    w = dipole_pml(n=n, p=p, seed=seed)
    inner = 1 - w.pml["thickness"]
    h = 2.0 / n
    w.S = n_sources
    w.extra["sources"] = [dipole(rng.uniform(-inner + 2 * h, inner - 2 * h, size=3),
                                 rng.uniform(1.0, 4.0), 1.0) for _ in range(n_sources)]
    cav = []
    for _ in range(n_cavities):
        ni = int(rng.integers(6, 29))
        pi = int(rng.integers(2, 6))
        c = Workload("cavity_n%d_p%d" % (ni, pi), ni, (0, 0, 0), (1, 1, 1), pi, "upwind",
                     "lsrk4", 0, stable_dt(1.0 / ni, pi))
        cav.append(c)
    return w, cav


def inverse_problem(seed=2005, n=24, p=3, n_sources=8, n_receivers=32, steps=1500):
    """Differentiable inverse problem: [-1,1]^3 on an n^3 Kuhn grid with a PML
    (0.25 thick, quadratic, sigma_max 40), degree p, per-element eps lognormal
    (median 2, sigma 0.3), mu = 1, n_sources z-dipoles (one per column) and
    n_receivers receiver points in the interior, a seeded target eps field."""
    rng = np.random.default_rng(seed)
    w = dipole_pml(n=n, p=p, seed=seed, steps=steps)
    inner = 1 - w.pml["thickness"]
    h = 2.0 / n
    w.S = n_sources
    w.extra["sources"] = [dipole(rng.uniform(-inner + 2 * h, inner - 2 * h, size=3),
                                 rng.uniform(1.0, 4.0), 1.0) for _ in range(n_sources)]
    w.extra["receivers"] = rng.uniform(-inner + h, inner - h, size=(n_receivers, 3))
    w.extra["eps"] = lognormal_material(w.K, 2.0, 0.3, seed + 1)
    w.extra["eps_target"] = lognormal_material(w.K, 2.0, 0.3, seed + 2)
    return w

