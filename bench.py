"""Throughput bench of the DG time-domain Maxwell hot path on one GB300.

Workload (one "step" = one LSRK4 time step = five fused right-hand-side /
stage launches over the whole mesh): the jittered-sphere problem -- 32^3
Kuhn grid of [0,1]^3 with interior vertices jittered by +-0.15 h (196,608
tetrahedra), p = 3 (20 modes per component), eps = 4 inside the centred
sphere of radius 0.25, upwind flux, low-storage RK4, Gaussian pulse
E_y = exp(-|r - r0|^2 / 0.01).  Synthetic, seeded.

metric: DoF-updates/s = 6 N K S steps / time.  The FP32 path is the headline
value; the plain FP64 path is measured on the same mesh and reported beside
it.  Inputs (three field-size buffers) exceed the 129 MB L2.

--impl reference runs the FP64 CPU oracle as it stands (assembled matrices,
scipy sparse products) on a bounded sample of the same workload.
"""
from __future__ import annotations

import os

# the oracle runs on one host core (reported as cores)
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse
import json
import math
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "DoF-updates/s"
# FP32 LSRK stage-kernel variants in autotuner order (degree 3 instantiations)
VARIANT_NAMES = ["32 cols x 384 thr", "32 cols x 192 thr", "16 cols x 192 thr",
                 "64 cols paired x 384 thr, packed FP32x2", "64 cols paired x 384 thr, scalar",
                 "64 cols x 512 thr, curl and lift on tensor cores (tcgen05, 3xTF32)"]
KERNEL_NAMES = ["stage_kernel<3,float,32,384,LSRK>", "stage_kernel<3,float,32,192,LSRK>",
                "stage_kernel<3,float,16,192,LSRK>", "stage2_kernel<3,F2x,384>",
                "stage2_kernel<3,P2,384>", "stage_kernel<3,float,64,512,LSRK,TC>"]
UNIT = "DoF-updates/s"


def kernel_name(variant, K, N, S):
    """The stage kernel a variant launches; single-column shapes use 32-bit index
    arithmetic when every index fits (the library's own test: field and
    face-jump rows x columns, geometry, per-face table below 2^32)."""
    name = KERNEL_NAMES[variant]
    if variant < 3 or variant == 5:
        NF = {4: 3, 10: 6, 20: 10, 35: 15, 56: 21}[N]
        C = K * S
        fits = max(6 * N * C, 24 * NF * C, 16 * K, 52 * K) < 2 ** 32
        name = name[:-1] + (",unsigned int>" if fits else ",long>")
    return name


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def build_problem(w):
    xyz, tets = w.mesh()
    c, r, ein, eout = w.extra["sphere"]
    eps = W.sphere_material(xyz, tets, c, r, ein, eout)
    return xyz, tets, eps


def pulse(r0):
    r0 = np.asarray(r0)

    def f(r):
        out = np.zeros((len(r), 6))
        out[:, 1] = np.exp(-((r - r0[None, :]) ** 2).sum(axis=1) / 0.01)
        return out
    return f


def stage_bytes(K, N, S, real_size):
    """Algorithmic DRAM bytes of one LSRK4 step (five stage launches).

    Per stage: read u, write u_out, write res (and read res except in the first
    stage, whose coefficient a_1 = 0), plus per element the geometry record
    (16 reals in the kernel's precision) and the neighbour table (4 int32).
    The per-face neighbour table the kernel also reads (40 reals per element,
    a precomputed copy of neighbour data) is not counted: it is a design
    choice, not data the method needs, and shows up in the measured traffic."""
    field = 6 * N * K * S * real_size
    geo = K * (16 * real_size + 4 * 4)
    return (3 * field + geo) + 4 * (4 * field + geo)


def world_rate(units, seconds, world, device=None):
    """Whole-job rate over `world` ranks: the units all ranks processed divided
    by the slowest rank's time (all ranks must call it; world 1: plain ratio)."""
    if world <= 1:
        return units / seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item())


def run_gpu(args, precision, steps, warmup, world, rank):
    import torch
    from paper_2002_08733_gb300 import dgmax as D

    w = W.jittered_sphere(n=args.n)
    xyz, tets, eps = build_problem(w)
    dev = torch.device("cuda", rank % max(torch.cuda.device_count(), 1))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    g = D.Solver(xyz, tets, eps, 1.0, w.p, precision, w.flux, w.integrator, w.dt, device=dev,
                 stream=stream)
    g.project(pulse(w.extra["r0"]))
    K, N, S = g.K, g.N, g.S
    dofs = 6 * N * K * S
    tuned = None
    if precision == "fp32" and args.variant is not None:
        g.set_variant(args.variant)
        if args.tile_groups is not None:
            g.set_tile_groups(args.tile_groups)
        if args.tile_loads is not None:
            g.set_tile_loads(args.tile_loads == "per_thread")
        tuned = {"variant": int(args.variant), "forced": True, "tile_groups": g.tile_groups(),
                 "bulk_tile_loads": g.bulk_tile_loads()}
    elif precision == "fp32":
        v, ms = g.autotune()
        tuned = {"variant": int(v), "ms_per_launch": [float(x) for x in ms],
                 "variants": VARIANT_NAMES[:len(ms)], "tile_groups": g.tile_groups(),
                 "bulk_tile_loads": g.bulk_tile_loads()}
    t = 0.0
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.advance(1, t)
            t += w.dt
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(dev.index or 0)
        with sampler:
            ev0.record(stream)
            for _ in range(steps):
                g.advance(1, t)
                t += w.dt
            ev1.record(stream)
            ev1.synchronize()
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1)
        value = world_rate(dofs * steps, ms * 1e-3, world, dev)
        ms = dofs * steps * world / value * 1e3       # the slowest rank's time
        g.status()
        energy = float(g.energy()[0])
    out = dict(precision=precision, ms=ms, steps=steps, dofs=dofs, K=K, N=N, S=S, tuned=tuned,
               value=value, clocks=sampler.summary(),
               energy=energy, launches=5 * steps, real_size=g.info.real_size,
               bytes_fields=g.info.bytes_fields, solver=g, t=t)
    return out


def run_pml(precision, steps, warmup, n=40, integrator="lsrk4", variant=None, groups=None,
            loads=None):
    """Dipole-in-PML workload: [-1,1]^3 on an n^3 Kuhn grid (384,000 tets at n=40),
    p=4, PML 0.25 thick with quadratic profile and sigma_max=40, z-directed
    dipole, starting from rest; upwind flux with LSRK4 or, with
    integrator="leapfrog", the central flux with staggered leapfrog and the
    PML terms by the trapezoid rule (two launches per step).  Returns timing
    and the algorithmic bytes of one step (fields plus PML auxiliaries)."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w = W.dipole_pml(n=n)
    xyz, tets = w.mesh()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    flux = w.flux if integrator == "lsrk4" else "central"
    g = D.Solver(xyz, tets, 1.0, 1.0, w.p, precision, flux, integrator, w.dt, device=dev,
                 stream=stream, pml=w.pml)
    g.set_sources(w.extra["sources"])
    tuned = None
    if precision == "fp32" and integrator == "lsrk4" and variant is not None:
        g.set_variant(variant)     # profiling runs: the shape the autotuner picks, pinned
        if groups is not None:
            g.set_tile_groups(groups)
        if loads is not None:
            g.set_tile_loads(loads == "per_thread")
        tuned = {"variant": int(variant), "forced": True, "tile_groups": g.tile_groups(),
                 "bulk_tile_loads": g.bulk_tile_loads()}
    elif precision == "fp32" and integrator == "lsrk4":   # tile shape (state untouched)
        v, ms_v = g.autotune()
        tuned = {"variant": int(v), "ms_per_launch": [float(x) for x in ms_v],
                 "tile_groups": g.tile_groups(),
                 "bulk_tile_loads": g.bulk_tile_loads()}
    t = 0.0
    if integrator == "leapfrog":
        g.leapfrog_start(0.0)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.advance(1, t)
            t += w.dt
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            g.advance(1, t)
            t += w.dt
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        g.status()
    final = g.fields[g.current()].double().cpu()
    dofs = 6 * g.N * g.K
    rs = g.info.real_size
    field = 6 * g.N * g.K * rs
    aux = 6 * g.N * g.npml * rs
    geo = g.K * (16 * rs + 4 * 4 + 4)
    if integrator == "lsrk4":
        step_bytes = (3 * field + 3 * aux + geo) + 4 * (4 * field + 4 * aux + geo)
    else:   # two launches: read both fields, write one; read both auxiliaries, write one
        step_bytes = 2 * (field + field // 2 + aux + aux // 2 + geo)
    return dict(value=dofs * steps / (ms * 1e-3), ms_per_step=ms / steps, steps=steps, K=g.K,
                N=g.N, n_pml=g.npml, bytes_per_step=step_bytes,
                hbm_frac=step_bytes / (ms / steps * 1e-3) / 1e9 / _peaks().get("hbm_gbs", 6800.0),
                autotune=tuned, _final=final)


def run_batched(steps, warmup):
    """Many sources on one PML mesh plus 16 uneven cavities (p 2..5), FP32,
    advanced together by one CUDA graph launch per two steps; each member's
    stage-kernel tile shape chosen by the autotuner."""
    import math as _m
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w, cavs = W.batched_sources_and_cavities()
    xyz, tets = w.mesh()
    dev = torch.device("cuda", 0)
    members, dofs, chosen = [], 0, []
    g = D.Solver(xyz, tets, 1.0, 1.0, w.p, "fp32", w.flux, w.integrator, w.dt, device=dev,
                 S=w.S, pml=w.pml)
    g.set_sources(w.extra["sources"])
    members.append(g)
    om = _m.pi * _m.sqrt(2.0)
    for c in cavs:
        cx, ct = c.mesh()
        gc = D.Solver(cx, ct, 1.0, 1.0, c.p, "fp32", c.flux, c.integrator, c.dt, device=dev)
        gc.project(lambda r: np.concatenate(
            [np.zeros((len(r), 2)), (np.sin(_m.pi * r[:, 0]) * np.sin(_m.pi * r[:, 1]))[:, None],
             np.zeros((len(r), 3))], axis=1))
        members.append(gc)
    step_bytes = 0
    for m in members:
        v, ms = m.autotune()
        chosen.append(int(v))
        dofs += 6 * m.N * m.K * m.S
        # algorithmic bytes of one LSRK4 step of the member (fields, PML auxiliaries, geometry)
        field = 6 * m.N * m.K * m.S * 4
        aux = 6 * m.N * m.npml * m.S * 4
        geo = m.K * (16 * 4 + 4 * 4 + 4)
        step_bytes += (3 * field + 3 * aux + geo) + 4 * (4 * field + 4 * aux + geo)
    b = D.Batch(members)
    b.advance(warmup)
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    b.advance(steps)
    ev1.record(st)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    for m in members:
        m.status()
    hbm = _peaks().get("hbm_gbs", 6800.0)
    return dict(value=dofs * steps / (ms * 1e-3), ms_per_step=ms / steps, steps=steps,
                bytes_per_step=step_bytes,
                hbm_frac=step_bytes / (ms / steps * 1e-3) / 1e9 / hbm,
                members=len(members), dofs_per_step=dofs, sources=w.S,
                cavities=[(c.n, c.p) for c in cavs], variants=chosen,
                graph_launches=steps // 2)


def run_reflection(n=16, p=4, chunks=8, T=2.4, sigma_max=40.0):
    """PML reflection (the dipole workload's PML: 0.25 thick, quadratic,
    sigma_max 40) on a coarser grid: [-1,1]^3 with the PML against the same
    problem on [-2,2]^3 at the same h, whose own boundary is too far away to be
    seen in the inner box before T.  Both grids are Kuhn grids numbered type by
    type, so an element of the small grid is the element of the large one with
    the same type and a shifted cube.  Reflection = max over sampled times of
    the E-coefficient difference in the small grid's inner box [-0.75, 0.75]^3,
    relative to the max over the same times of the large grid's E there.  FP32.
    sigma_max sets the small grid's PML only (0: its walls reflect fully)."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    ws = W.dipole_pml(n=n, p=p, sigma_max=sigma_max)
    src = ws.extra["sources"]
    xs, ts = ws.mesh()
    xl, tl = W.kuhn_mesh(2 * n, (-2, -2, -2), (2, 2, 2))
    th = ws.pml["thickness"]
    pml_l = dict(lo=(-2 + th,) * 3, hi=(2 - th,) * 3, thickness=th,
                 sigma_max=40.0, order=ws.pml["order"])
    gs = D.Solver(xs, ts, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", ws.dt, pml=ws.pml)
    gl = D.Solver(xl, tl, 1.0, 1.0, p, "fp32", "upwind", "lsrk4", ws.dt, pml=pml_l)
    for g in (gs, gl):
        g.set_sources(src)
        g.autotune()
    # element e = t n^3 + i + n j + n^2 k of the small grid <-> same type, cube + n/2
    n3, L = n ** 3, 2 * n
    e = np.arange(6 * n3)
    t, c = e // n3, e % n3
    i, j, k = c % n, (c // n) % n, c // (n * n)
    el = t * L ** 3 + (i + n // 2) + L * (j + n // 2) + L * L * (k + n // 2)
    cen = W.centroids(xs, ts)
    inner = np.all(np.abs(cen) < 1 - th, axis=1)
    steps = int(round(T / ws.dt))
    per = max(1, steps // chunks)
    diff = ref = 0.0
    tt = 0.0
    torch.cuda.synchronize()
    start = time.perf_counter()
    for _ in range(chunks):
        gs.advance(per, tt)
        gl.advance(per, tt)
        tt += per * ws.dt
        us = gs.state()[inner][:, 0, 0:3, :]
        ul = gl.state()[el[inner]][:, 0, 0:3, :]
        diff = max(diff, float(np.linalg.norm(us - ul)))
        ref = max(ref, float(np.linalg.norm(ul)))
    el_s = time.perf_counter() - start
    return dict(n=n, p=p, K_small=gs.K, K_large=gl.K, steps=per * chunks, T=tt,
                reflection=diff / ref, seconds=el_s)


def run_mixed(precision, steps, warmup, n=32, p=2):
    """Mixed orders (E of degree p + 1, H of degree p; Sec. III) on the
    jittered-sphere mesh (upwind, LSRK4, the same pulse), the plain
    one-thread-per-column kernel.  DoFs per column: 3 (N_E + N_H) per element."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w = W.jittered_sphere(n=n, p=p + 1)
    xyz, tets, eps = build_problem(w)
    dev = torch.device("cuda", 0)
    g = D.Solver(xyz, tets, eps, 1.0, p, precision, "upwind", "lsrk4", w.dt, device=dev,
                 mixed=True)
    g.project(pulse(w.extra["r0"]))
    t = 0.0
    for _ in range(warmup):
        g.advance(1, t)
        t += w.dt
    torch.cuda.synchronize(dev)
    st = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    g.advance(steps, t)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    g.status()
    dofs = 3 * (g.N + g.NH) * g.K
    return dict(precision=precision, K=g.K, p_E=p + 1, p_H=p, N_E=g.N, N_H=g.NH, steps=steps,
                ms_per_step=ms / steps, value=dofs * steps / (ms * 1e-3))


def run_boundary_and_penalty(steps, warmup, n=32, alpha=10.0):
    """The incident-field boundary and the interior penalty on the jittered-sphere
    mesh (p = 3, FP32, autotuned): time per LSRK4 step with incident faces on the
    z = 0 side (upwind) against the same plan without them, and with the facet
    field of the penalty (central flux) against the plain central flux.  The
    penalty's algorithmic bytes add, per stage and facet, the facet field read by
    both sides, the owner's residual read and write and its output write."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w = W.jittered_sphere(n=n)
    xyz, tets, eps = build_problem(w)
    dev = torch.device("cuda", 0)
    faces = W.box_faces(n, tets, 2, 0)

    def timed(flux, incident=False, sip=None):
        g = D.Solver(xyz, tets, eps, 1.0, w.p, "fp32", flux, "lsrk4", w.dt, device=dev, sip=sip)
        g.project(pulse(w.extra["r0"]))
        if incident:
            g.set_incident(faces, E0=(1.0, 0.0, 0.0), direction=(0.0, 0.0, 1.0), speed=0.5,
                           f0=2.0, bw=1.0, t0=0.5)
        v, _ = g.autotune()
        t = 0.0
        for _ in range(warmup):
            g.advance(1, t)
            t += w.dt
        torch.cuda.synchronize(dev)
        st = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.advance(steps, t)
        e1.record(st)
        e1.synchronize()
        g.status()
        return e0.elapsed_time(e1) / steps, g, v

    out = {"workload": "jittered sphere, %d^3 (%d tets), p=3, FP32, LSRK4, %d steps each" % (n, w.K, steps)}
    ms0, g0, v0 = timed("upwind")
    ms1, g1, v1 = timed("upwind", incident=True)
    out["incident"] = dict(faces=int(len(faces)), ms_per_step=ms1, plain_ms_per_step=ms0,
                           overhead=ms1 / ms0 - 1.0, variant=int(v1))
    ms2, g2, v2 = timed("central")
    ms3, g3, v3 = timed("central", sip=alpha)
    nF = int(g3.info.n_facets)
    base = stage_bytes(g3.K, g3.N, g3.S, 4)
    unit = nF * g3.S * 3 * W.n_face_modes(w.p) * 4     # one facet-field buffer, FP32
    facet = (5 * 5 - 1) * unit                          # five per stage, no residual read in the first
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    out["sip"] = dict(alpha=alpha, facets=nF, ms_per_step=ms3, plain_central_ms_per_step=ms2,
                      overhead=ms3 / ms2 - 1.0, variant=int(v3),
                      bytes_per_step=base + facet,
                      hbm_frac=(base + facet) / (ms3 * 1e-3) / (hbm * 1e9))
    return out


def fp64_reference_rate(n=8192, reps=5):
    """FP64 throughput reference of this GPU: cuBLAS DGEMM through torch.matmul
    (2 n^3 flop per product, best of `reps` after a warm-up), CUDA events."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return dict(what="cuBLAS DGEMM %d^3 (torch.matmul, float64)" % n, ms=best,
                tflops=2.0 * n ** 3 / (best * 1e-3) / 1e12)


def run_cavity():
    """PEC cavity: 4^3 Kuhn grid (384 tets), p=2, vacuum, central flux, leapfrog,
    200 steps of dt = 0.3 h/(p+1)^2 from the TM110 mode; reports the L2 error of
    E against the closed form E_z = sin(pi x) sin(pi y) cos(w t), w = pi sqrt(2),
    evaluated with the library's own projection of the exact field."""
    import math as _m
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w = W.cavity_tm110()
    xyz, tets = w.mesh()
    g = D.Solver(xyz, tets, 1.0, 1.0, w.p, "fp64", w.flux, w.integrator, w.dt)
    om = _m.pi * _m.sqrt(2.0)

    def ez(t):
        return lambda r: np.concatenate([np.zeros((len(r), 2)), (np.sin(_m.pi * r[:, 0]) * np.sin(
            _m.pi * r[:, 1]) * _m.cos(om * t))[:, None], np.zeros((len(r), 3))], axis=1)
    g.project(ez(0.0))
    g.leapfrog_start(0.0)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    g.advance(w.steps, 0.0)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    got = g.state()
    T = w.steps * w.dt
    g.project(ez(T))
    ref = g.state()
    err = float(np.linalg.norm((got - ref)[:, :, 0:3]) / np.linalg.norm(ref[:, :, 0:3]))
    dofs = 6 * g.N * g.K
    return dict(steps=w.steps, K=g.K, p=w.p, ms_per_step=ms / w.steps,
                value=dofs * w.steps / (ms * 1e-3), dtype="f64",
                e_rel_coeff_diff_vs_projected_closed_form=err)


def run_adjoint(steps, n=24):
    """Inverse-problem workload: forward with receiver records plus the
    hand-written adjoint (sqrt(N) checkpointing), FP32 state, FP64 gradient
    (n^3 Kuhn grid; 24 is the benchmarked size, smaller for profiling)."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D
    w = W.inverse_problem(steps=steps, n=n)
    xyz, tets = w.mesh()
    dev = torch.device("cuda", 0)
    rec = w.extra["receivers"]
    g = D.Solver(xyz, tets, w.extra["eps_target"], 1.0, w.p, "fp32", w.flux, w.integrator, w.dt,
                 device=dev, S=w.S, pml=w.pml, max_receivers=len(rec))
    g.set_sources(w.extra["sources"])
    g.set_receivers(rec)
    g.autotune()              # tile shape and tile order for the forward stages
    mu = torch.ones(g.K, dtype=torch.float64)
    with torch.no_grad():
        target = D.receiver_records(g, torch.tensor(w.extra["eps_target"]), mu, steps)
    eps = torch.tensor(w.extra["eps"], requires_grad=True)
    mu_p = mu.clone().requires_grad_(True)
    # warm the PyTorch kernels of the loss (their first call loads or JIT-compiles them)
    float((0.5 * ((target - target) ** 2).sum()).item())
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r = D.receiver_records(g, eps, mu_p, steps)
    loss = 0.5 * ((r - target) ** 2).sum()
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    dofs = 6 * g.N * g.K * g.S
    import ctypes
    ws = ctypes.c_size_t()
    D._lib.dgm_adjoint_workspace(g.handle, int(steps), ctypes.byref(ws))
    seg = int(math.ceil(math.sqrt(steps / 5.0)))
    return dict(steps=steps, K=g.K, S=g.S, receivers=len(rec), loss=float(loss.detach()),
                checkpoint_segment=seg, workspace_bytes=int(ws.value),
                state_bytes=int(g.info.bytes_fields + g.info.bytes_aux),
                forward_s=t1 - t0, adjoint_s=t2 - t1,
                forward_dof_updates_per_s=dofs * steps / (t1 - t0),
                adjoint_over_forward=(t2 - t1) / (t1 - t0),
                grad_eps_norm=float(eps.grad.norm()), grad_mu_norm=float(mu_p.grad.norm()))


TRAFFIC_PROFILE = "stage_kernel_full_jittered_sphere_n28_p3_fp32.md"


def profiled_traffic(path, variant, groups, columns, loads="bulk"):
    """DRAM bytes of one stage launch from the committed ncu summary: its line
    `traffic_bytes_per_element_stage variant=V tile_groups=G loads=L: B` for
    the tile shape, tile order and phase-1 load path (bulk copies or
    per-thread loads) this run uses, times the columns; None when the summary
    has no line for them (counters of another kernel configuration say nothing
    about this one)."""
    import re
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    for m in re.finditer(r"traffic_bytes_per_element_stage variant=(\d+) tile_groups=(\d+)"
                         r" loads=(\w+):\s*(\d+)", txt):
        if int(m.group(1)) == variant and int(m.group(2)) == groups and m.group(3) == loads:
            return int(m.group(4)) * columns
    return None


def run_e2e(g, steps, t0, world=1):
    """End-to-end: per step, pinned host state -> device, one step, device -> host,
    through the C-ABI call with host buffers; whole-job rate over the ranks."""
    import torch
    nbytes = g.info.bytes_fields
    hin = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hin.copy_(g.fields[g.current()].view(torch.uint8).reshape(-1).cpu())
    g.advance_host(hin, hout, 1, t0)     # warm
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t = t0
    start = time.perf_counter()
    for _ in range(steps):
        g.advance_host(hin, hout, 1, t)
        t += g.dt
    el = time.perf_counter() - start
    dofs = 6 * g.N * g.K * g.S
    return dict(value=world_rate(dofs * steps, el, world, g.device), unit=UNIT,
                h2d_bytes_per_step=int(nbytes), d2h_bytes_per_step=int(nbytes))


SPHERE_REPLICA_N = 3
# the replica's layer starts at |x| = 0.6 (0.4 thick) so that its centroids (at
# 0.25, 0.5, 0.75 of a unit cube) are damped; the full workload's 0.25-thick
# layer at 0.75 would damp none of them
DIPOLE_REPLICA = dict(n=2, src=(0.13, -0.21, 0.08),
                      pml=dict(lo=(-0.6,) * 3, hi=(0.6,) * 3, thickness=0.4,
                               sigma_max=40.0, order=2))


def cpu_reference():
    """The FP64 oracle, as it stands, on bounded samples of the two benchmarked
    workloads, at their full step counts and time steps, on replica meshes:

    * jittered sphere (p = 3, eps = 4 sphere, upwind, LSRK4, Gaussian pulse) on
      a 3^3 jittered grid (162 elements), 1000 steps -- timed: the CPU baseline;
    * dipole in a PML (p = 4, quadratic layer with sigma_max 40, z dipole from
      rest) on a 2^3 grid of [-1,1]^3 (48 elements), 2000 steps.

    Returns the baseline record and, for each replica, what the GPU runs need
    to be compared with the oracle (initial state from the oracle's own
    projection, final oracle state)."""
    import torch
    from oracle.assemble import Assembly, pml_sigma
    from oracle.mesh import Mesh
    from oracle.solver import Solver as OSolver
    full = W.jittered_sphere()
    w = W.jittered_sphere(n=SPHERE_REPLICA_N)
    xyz, tets, eps = build_problem(w)
    o = OSolver(Assembly(Mesh(xyz, tets), w.p, eps, 1.0, w.flux))
    r0 = np.asarray(full.extra["r0"])
    ey = o.project(lambda q: np.stack([0 * q[:, 0], np.exp(-((q - r0) ** 2).sum(1) / 0.01),
                                       0 * q[:, 0]], axis=1), "E")
    u0 = np.zeros((len(tets), 1, 6, w.N))
    u0[:, 0, 0:3] = ey
    start = time.perf_counter()
    x = o.lsrk4(o.pack(u0), 0.0, full.dt, full.steps)
    el = time.perf_counter() - start
    dofs = 6 * o.asm.N * o.asm.K
    base = dict(value=dofs * full.steps / el, unit=UNIT, cores=1,
                kind="oracle", seconds=el,
                sample="jittered-sphere workload (p=3, upwind, LSRK4, eps=4 sphere, Gaussian "
                       "pulse) on a %d^3 jittered Kuhn grid (%d elements), %d LSRK4 steps of "
                       "dt=%.4g as in the full workload; assembly and projection excluded; "
                       "one host core (scipy sparse products)"
                       % (SPHERE_REPLICA_N, o.asm.K, full.steps, full.dt))
    sphere = dict(xyz=xyz, tets=tets, eps=eps, p=w.p, dt=full.dt, steps=full.steps, u0=u0,
                  ref=o.unpack(x)[0],
                  workload="jittered sphere on a %d^3 replica grid (%d elements), p=3, %d "
                           "steps of dt=%.4g" % (SPHERE_REPLICA_N, o.asm.K, full.steps, full.dt))
    fd = W.dipole_pml()
    r = DIPOLE_REPLICA
    xyz, tets = W.kuhn_mesh(r["n"], (-1, -1, -1), (1, 1, 1))
    m = Mesh(xyz, tets)
    pm = r["pml"]
    sig = pml_sigma(m.centroids(), pm["lo"], pm["hi"], pm["thickness"], pm["sigma_max"],
                    pm["order"])
    src = [W.dipole(r["src"], 2.0, 1.0)]
    od = OSolver(Assembly(m, fd.p, 1.0, 1.0, "upwind", sigma=sig), S=1, sources=src)
    xd = od.lsrk4(np.zeros((od.asm.ndof, 1)), 0.0, fd.dt, fd.steps)
    ud, ad = od.unpack(xd)
    dipole = dict(xyz=xyz, tets=tets, p=fd.p, dt=fd.dt, steps=fd.steps, src=src, pml=pm,
                  ref=ud, ref_aux=ad,
                  workload="dipole in the PML on a %d^3 replica grid of [-1,1]^3 (%d elements, "
                           "%d in the layer), p=4, %d steps of dt=%.4g from rest"
                           % (r["n"], od.asm.K, int(np.any(sig > 0, axis=1).sum()), fd.steps,
                              fd.dt))
    return base, sphere, dipole


def _errors(got, ref):
    return dict(rel_l2=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                rel_max=float(np.abs(got - ref).max() / np.abs(ref).max()))


def replica_accuracy(sphere, dipole):
    """FP32 (autotuned) and FP64 GPU runs of the two replicas against the oracle
    at the full step counts: relative L2 and element-wise error of the final
    state (fields; PML auxiliaries for the dipole)."""
    from paper_2002_08733_gb300 import dgmax as D
    out = {"jittered_sphere": {"workload": sphere["workload"]},
           "dipole_pml": {"workload": dipole["workload"]}}
    for prec in ("fp32", "fp64"):
        c = sphere
        g = D.Solver(c["xyz"], c["tets"], c["eps"], 1.0, c["p"], prec, "upwind", "lsrk4",
                     c["dt"])
        if prec == "fp32":
            g.autotune()
        g.set_state(c["u0"])
        g.advance(c["steps"], 0.0)
        out["jittered_sphere"][prec] = _errors(g.state(), c["ref"])
        c = dipole
        g = D.Solver(c["xyz"], c["tets"], 1.0, 1.0, c["p"], prec, "upwind", "lsrk4", c["dt"],
                     pml=c["pml"])
        g.set_sources(c["src"])
        if prec == "fp32":
            g.autotune()
        g.advance(c["steps"], 0.0)
        e = _errors(g.state(), c["ref"])
        ea = _errors(g.from_device(g.aux[g.current()]), c["ref_aux"][g.pml_elements()])
        e.update(aux_rel_l2=ea["rel_l2"], aux_rel_max=ea["rel_max"])
        out["dipole_pml"][prec] = e
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000,
                    help="timed steps (1000 FP32 steps: about 1.2 s, long enough for clock samples)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=32,
                    help="Kuhn grid size (32 = the benchmarked workload; smaller for profiling)")
    ap.add_argument("--only", choices=["fp32", "fp64", "adjoint", "pml", "mixed", "boundary"],
                    default=None,
                    help="profile one precision (or the inverse-problem or dipole-in-PML leg) only")
    ap.add_argument("--pml-n", type=int, default=40,
                    help="Kuhn grid size of the dipole-in-PML leg (40 = the benchmarked workload)")
    ap.add_argument("--adjoint-n", type=int, default=24,
                    help="Kuhn grid size of the inverse problem (24 = the benchmarked workload)")
    ap.add_argument("--no-pml", action="store_true", help="skip the p=4 dipole-in-PML workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--batched-steps", type=int, default=1000,
                    help="steps of the batched workload (1000, its stated step count)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the inverse-problem workload")
    ap.add_argument("--variant", type=int, default=None,
                    help="force the FP32 stage-kernel tile shape instead of autotuning "
                         "(profiling runs: the autotuner's timings are distorted under ncu)")
    ap.add_argument("--tile-groups", type=int, default=None,
                    help="with --variant: force the FP32 tile visiting order (default: plain order)")
    ap.add_argument("--tile-loads", choices=["bulk", "per_thread"], default=None,
                    help="with --variant: force the stage kernel's phase-1 load path (default: "
                         "bulk copies where the plan allows them)")
    ap.add_argument("--adjoint-steps", type=int, default=1500,
                    help="steps of the inverse problem (1500, its stated step count)")
    ap.add_argument("--pml-steps", type=int, default=20)
    ap.add_argument("--mixed-steps", type=int, default=10)
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-order leg")
    ap.add_argument("--no-boundary", action="store_true",
                    help="skip the incident-boundary and interior-penalty leg")
    ap.add_argument("--boundary-steps", type=int, default=200)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    w = W.jittered_sphere(n=args.n)
    config = {"workload": "jittered_sphere: %d^3 Kuhn grid of [0,1]^3 (+-0.15h jitter), "
                          "%d tets, p=3, eps=4 sphere r=0.25, upwind, LSRK4, "
                          "Gaussian pulse" % (args.n, w.K), "K": w.K, "p": w.p, "S": 1,
              "dt": w.dt, "l2": "inputs exceed L2 (3 x field buffers > 129 MB)"}

    if args.impl == "reference":
        if rank != 0:
            return
        steps, warm = args.steps, args.warmup
        from oracle.assemble import Assembly
        from oracle.mesh import Mesh
        from oracle.solver import Solver as OSolver
        n_ref = 4
        ws = W.jittered_sphere(n=n_ref)
        xyz, tets, eps = build_problem(ws)
        o = OSolver(Assembly(Mesh(xyz, tets), ws.p, eps, 1.0, ws.flux))
        x = np.full((o.asm.ndof, 1), 1e-3)
        for _ in range(warm):
            x = o.lsrk4(x, 0.0, w.dt, 1)
        start = time.perf_counter()
        for _ in range(steps):
            x = o.lsrk4(x, 0.0, w.dt, 1)
        el = time.perf_counter() - start
        dofs = 6 * o.asm.N * o.asm.K
        v = dofs * steps / el
        sample = ("each step: one LSRK4 step (dt of the 32^3 workload) of the oracle on the "
                  "jittered-sphere workload at %d^3 (%d elements, p=3), assembly excluded; "
                  "one host core (scipy sparse products)" % (n_ref, o.asm.K))
        ref_config = dict(config)
        ref_config.update(
            workload="jittered_sphere sample: %d^3 Kuhn grid of [0,1]^3 (+-0.15h jitter), %d "
                     "tets, p=3, eps=4 sphere r=0.25, upwind, LSRK4 (the oracle's bounded "
                     "sample of the %d^3 workload)" % (n_ref, o.asm.K, args.n),
            K=o.asm.K, l2="oracle on the host CPU")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
                "steps": steps, "warmup": warm, "ms_per_step": el * 1e3 / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": ref_config,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1,
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    if args.only == "boundary":
        r = run_boundary_and_penalty(args.boundary_steps, 3, n=args.n)
        if rank == 0:
            print(json.dumps({"profile_run": "boundary", **r}))
        return
    if args.only == "mixed":
        r = [run_mixed(pr, args.mixed_steps, args.warmup, n=args.n) for pr in ("fp32", "fp64")]
        if rank == 0:
            print(json.dumps({"profile_run": "mixed", "runs": r}))
        return
    if args.only == "pml":
        r = run_pml("fp32", args.pml_steps, args.warmup, n=args.pml_n, variant=args.variant,
                    groups=args.tile_groups, loads=args.tile_loads)
        r.pop("_final")
        if rank == 0:
            print(json.dumps({"profile_run": "pml", **r}))
        return
    if args.only == "adjoint":
        r = run_adjoint(args.adjoint_steps, args.adjoint_n)
        if rank == 0:
            print(json.dumps({"profile_run": "adjoint", **r}))
        return
    if args.only == "fp64":
        r = run_gpu(args, "fp64", args.steps, args.warmup, world, rank)
        if rank == 0:
            print(json.dumps({"profile_run": "fp64", "ms_per_step": r["ms"] / r["steps"],
                              "value": r["value"]}))
        return
    r32 = run_gpu(args, "fp32", args.steps, args.warmup, world, rank)
    if args.only == "fp32":
        if rank == 0:
            print(json.dumps({"profile_run": "fp32", "ms_per_step": r32["ms"] / r32["steps"],
                              "value": r32["value"]}))
        return
    r64 = run_gpu(args, "fp64", min(args.fp64_steps, args.steps), min(args.warmup, 3), world, rank)
    e2e = None if args.no_e2e else run_e2e(r32["solver"], max(3, min(20, args.steps // 5)),
                                           r32["t"], world)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    launch_ms = r32["ms"] / r32["launches"]
    bytes_step = stage_bytes(r32["K"], r32["N"], r32["S"], r32["real_size"])
    achieved = bytes_step / 5 / (launch_ms * 1e-3) / 1e9
    # DRAM traffic of one stage launch: the committed ncu summary's full-size
    # figure for this tile shape and tile order, per element-stage times columns
    chosen = (r32["tuned"] or {}).get("variant", 0)
    groups = (r32["tuned"] or {}).get("tile_groups", 1)
    loads = "bulk" if (r32["tuned"] or {}).get("bulk_tile_loads", False) else "per_thread"
    traffic = profiled_traffic(os.path.join(ROOT, "profiles", TRAFFIC_PROFILE), chosen, groups,
                               r32["K"] * r32["S"], loads)
    line = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r32["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": peak_src,
                     "kernel": kernel_name(chosen, r32["K"], r32["N"], r32["S"]),
                     "algorithmic_bytes_per_launch": bytes_step / 5},
        "fp64": {"value": r64["value"], "ms_per_step": r64["ms"] / r64["steps"],
                 "steps": r64["steps"], "dtype": "f64"},
        "fp32_over_fp64": r32["value"] / r64["value"],
        "e2e": e2e,
        "gpu_launches": r32["launches"],
        "autotune": r32["tuned"],
        "clocks": r32["clocks"],
    }
    if world == 1:
        line["fp64"]["reference_rate"] = fp64_reference_rate()
        line["fp64"]["flop_per_dof_update"] = 1450
    if not args.no_pml and world == 1:
        p32 = run_pml("fp32", args.pml_steps, 3)
        p64 = run_pml("fp64", args.pml_steps, 3)
        f32, f64 = p32.pop("_final"), p64.pop("_final")
        err = float((f32 - f64).norm() / f64.norm())
        line["p4_pml"] = {"workload": "dipole_pml: [-1,1]^3, 40^3 Kuhn grid, 384000 tets, p=4, "
                                      "PML 0.25 sigma_max=40, z dipole, upwind, LSRK4, from rest",
                          "fp32": p32, "fp64": p64, "fp32_over_fp64": p32["value"] / p64["value"],
                          "fp32_vs_fp64_rel_l2_after_%d_steps" % (args.pml_steps + 3): err}
        lf32 = run_pml("fp32", args.pml_steps, 3, integrator="leapfrog")
        lf32.pop("_final")
        line["p4_pml_leapfrog"] = {
            "workload": "the same dipole-in-PML mesh and source, central flux, staggered "
                        "leapfrog with the PML terms by the trapezoid rule (Sec. V), same dt",
            "fp32": lf32, "lsrk4_fp32_ms_per_step": p32["ms_per_step"]}
    if not args.no_batched and world == 1:
        line["batched"] = dict(workload="64 dipoles on a 24^3 PML mesh (p=3, S=64) + 16 PEC "
                                        "cavities n 6..28, p 2..5; FP32; one graph launch per "
                                        "two steps; autotuned tile shapes",
                               **run_batched(args.batched_steps, 2))
    if not args.no_mixed and world == 1:
        line["mixed_orders"] = dict(
            workload="jittered sphere mesh (%d^3, %d tets), E of degree 3 and H of degree 2 "
                     "(Sec. III), upwind, LSRK4, the same pulse; plain one-thread-per-column "
                     "kernel with dense operators" % (args.n, w.K),
            fp32=run_mixed("fp32", args.mixed_steps, 2, n=args.n),
            fp64=run_mixed("fp64", min(args.mixed_steps, 3), 1, n=args.n))
    if not args.no_boundary and world == 1:
        line["boundary_and_penalty"] = run_boundary_and_penalty(args.boundary_steps, 3, n=args.n)
    if world == 1:
        line["cavity"] = dict(workload="PEC cavity 4^3 (384 tets), p=2, central, leapfrog, "
                                       "TM110, 200 steps (latency regime, state fits in L2)",
                              **run_cavity())
    if not args.no_pml and world == 1:
        line["pml_reflection"] = dict(
            workload="dipole in the same PML (0.25 thick, quadratic, sigma_max 40) on a 16^3 "
                     "grid of [-1,1]^3, p=4, against [-2,2]^3 at the same h; E in the inner box",
            **run_reflection())
    if not args.no_adjoint and world == 1:
        line["adjoint"] = dict(workload="24^3 PML mesh (82944 tets), p=3, 8 dipoles, 32 "
                                        "receivers, lognormal eps, receiver-misfit loss; FP32 "
                                        "state, FP64 gradient, sqrt(N) checkpoints",
                               **run_adjoint(args.adjoint_steps, args.adjoint_n))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, sphere, dipole = cpu_reference()
        line["cpu_baseline"] = base
        line["accuracy_vs_oracle"] = replica_accuracy(sphere, dipole)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
