"""CPU tests of the C ABI: the library builds, loads, exports every function
declared in include/dgmax.h, and its host-side setup validates inputs.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_08733_gb300 import build, dgmax
    build.build()
    return dgmax.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dgmax.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dgm_plan_create", "dgm_bind", "dgm_rhs", "dgm_advance", "dgm_energy",
                     "dgm_advance_host", "dgm_set_sources", "dgm_project", "dgm_last_error",
                     "dgm_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_plan_sizes(lib):
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(3, jitter=0.1, seed=1)
    for p, prec, rs in ((1, "fp64", 8), (3, "fp32", 4), (4, "fp64", 8), (5, "fp32", 4)):
        pl = D.Plan(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3, S=3)
        N = W.n_modes(p)
        assert (pl.info.K, pl.info.N, pl.info.S, pl.info.real_size) == (162, N, 3, rs)
        assert pl.info.bytes_fields == 6 * N * 162 * 3 * rs
        assert pl.info.bytes_aux == 0 and pl.info.n_pml == 0
        assert pl.info.bytes_geom % 256 == 0


def test_pml_elements_are_those_outside_the_box(lib):
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(4, lo=(-1, -1, -1), hi=(1, 1, 1))
    pml = dict(lo=(-0.5,) * 3, hi=(0.5,) * 3, thickness=0.5, sigma_max=10.0)
    pl = D.Plan(xyz, tets, 1.0, 1.0, 2, "fp32", "upwind", "lsrk4", 1e-3, pml=pml)
    c = W.centroids(xyz, tets)
    outside = np.any((c < -0.5) | (c > 0.5), axis=1)
    assert np.array_equal(pl.pml_elements(), np.nonzero(outside)[0])


def test_quad_points_lie_in_their_elements(lib):
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(2, jitter=0.1, seed=3)
    pl = D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", "upwind", "lsrk4", 1e-3)
    q = pl.quad_points()
    st = np.sort(tets, axis=1)
    for e in (0, 7, 33):
        V = xyz[st[e]]
        A = (V[1:] - V[0]).T
        lam = np.linalg.solve(A, (q[e] - V[0]).T).T
        assert np.all(lam > -1e-12) and np.all(lam.sum(axis=1) < 1 + 1e-12)


@pytest.mark.parametrize("case", ["repeated", "range", "degenerate", "nonmanifold",
                                  "eps", "order", "leapfrog_upwind", "dt", "columns", "empty"])
def test_invalid_inputs_are_rejected(lib, case):
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(2)
    kw = dict(eps=1.0, mu=1.0, p=2, precision="fp64", flux="upwind", integrator="lsrk4",
              dt=1e-3, S=1)
    expect = D.DgmError
    if case == "repeated":
        tets = tets.copy()
        tets[3, 1] = tets[3, 0]
    elif case == "range":
        tets = tets.copy()
        tets[0, 0] = 10 ** 6
    elif case == "degenerate":
        xyz = xyz.copy()
        xyz[:, 2] = 0.0
    elif case == "nonmanifold":
        tets = np.concatenate([tets, tets[:1]])
    elif case == "eps":
        kw["eps"] = np.where(np.arange(len(tets)) == 5, -1.0, 1.0)
    elif case == "order":
        kw["p"] = 6
    elif case == "leapfrog_upwind":
        kw["integrator"] = "leapfrog"
    elif case == "dt":
        kw["dt"] = 0.0
    elif case == "columns":
        kw["S"] = 0
    elif case == "empty":
        tets = tets[:0]
        kw["eps"] = kw["mu"] = 1.0
    with pytest.raises(expect) as ei:
        D.Plan(xyz, tets, kw.pop("eps"), kw.pop("mu"), kw.pop("p"), **kw)
    codes = {"repeated": 2, "range": 2, "degenerate": 2, "nonmanifold": 2, "eps": 1,
             "order": 3, "leapfrog_upwind": 3, "dt": 1, "columns": 1, "empty": 1}
    assert ei.value.code == codes[case]


def test_energy_noalloc_rejects_bad_output_buffers(lib, monkeypatch):
    """The allocation-free energy writes its output buffer from a kernel, so the
    binding checks it before the call: a numpy array, a CPU tensor, an FP32
    tensor, a short tensor or a non-contiguous one never reach the library."""
    import torch
    from paper_2002_08733_gb300 import dgmax as D

    class FakeCuda:
        """Stands in for a CUDA tensor: only the attributes the check reads."""
        def __init__(self, dtype, numel, index=0, contiguous=True):
            self.dtype, self._n, self._c = dtype, numel, contiguous
            self.is_cuda = True
            self.device = torch.device("cuda", index)

        def numel(self):
            return self._n

        def is_contiguous(self):
            return self._c

    calls = []

    class NoLib:
        def __getattr__(self, name):
            calls.append(name)
            raise AssertionError("library called: " + name)

    monkeypatch.setattr(D, "_lib", NoLib())
    g = D.Solver.__new__(D.Solver)
    g.torch, g.device, g.S, g.N, g.K = torch, torch.device("cuda", 0), 4, 4, 6
    g.dtype = torch.float32
    g.fields = [FakeCuda(torch.float32, 6 * 4 * 6 * 4)] * 2
    g.current = lambda: 0
    monkeypatch.setattr(torch, "is_tensor", lambda t: isinstance(t, (torch.Tensor, FakeCuda)))
    bad = [np.zeros(4), torch.zeros(4, dtype=torch.float64), FakeCuda(torch.float32, 4),
           FakeCuda(torch.float64, 3), FakeCuda(torch.float64, 4, contiguous=False),
           FakeCuda(torch.float64, 4, index=1)]
    for out in bad:
        with pytest.raises(ValueError):
            g.energy_noalloc(out)
    with pytest.raises(ValueError):   # fields of the wrong precision
        g.energy_noalloc(FakeCuda(torch.float64, 4), fields=FakeCuda(torch.float64, 6 * 96))
    assert calls == []


def test_mixed_order_plan_sizes_and_limits(lib):
    """dgm_plan_create_mixed: E of degree p + 1, H of degree p -- field rows
    3 N + 3 N_H; no PML, no leapfrog, p <= 3."""
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(2)
    for p, prec, rs in ((1, "fp64", 8), (2, "fp32", 4), (3, "fp64", 8)):
        pl = D.Plan(xyz, tets, 1.0, 1.0, p, prec, "upwind", "lsrk4", 1e-3, S=2, mixed=True)
        NE, NH = W.n_modes(p + 1), W.n_modes(p)
        assert (pl.info.N, pl.info.N_H) == (NE, NH)
        assert pl.info.bytes_fields == 3 * (NE + NH) * 48 * 2 * rs
        assert pl.info.n_quad == (p + 4) ** 3
    plain = D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", "upwind", "lsrk4", 1e-3)
    assert plain.info.N_H == plain.info.N
    pml = dict(lo=(0.25,) * 3, hi=(0.75,) * 3, thickness=0.25, sigma_max=10.0)
    for kw in (dict(pml=pml), dict(integrator="leapfrog", flux="central"), dict(p=4)):
        args = dict(p=2, precision="fp64", flux="upwind", integrator="lsrk4", dt=1e-3)
        args.update(kw)
        extra = {"pml": args.pop("pml")} if "pml" in args else {}
        with pytest.raises(D.DgmError):
            D.Plan(xyz, tets, 1.0, 1.0, args["p"], args["precision"], args["flux"],
                   args["integrator"], args["dt"], mixed=True, **extra)


def test_incident_faces_are_validated_on_the_host(lib):
    """dgm_set_incident: boundary faces only, each once, a positive bandwidth
    and speed; refused on mixed-order and leapfrog plans; the paired FP32
    variants are refused while incident faces are set.  No CUDA call."""
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(2)
    on_z0 = lambda tri: np.all(np.abs(xyz[list(tri), 2]) < 1e-12)
    bnd, inner = [], []
    from oracle.mesh import Mesh          # face adjacency for choosing the test faces
    m = Mesh(xyz, tets)
    for T in range(m.K):
        for f in range(4):
            tri = np.delete(m.tets[T], f)
            (bnd if m.nbr[T, f] < 0 else inner).append(tri)
    z0 = [t for t in bnd if on_z0(t)]
    assert len(z0) == 8
    wave = dict(E0=(1, 0, 0), direction=(0, 0, 1), speed=1.0, f0=0.0, bw=1.0, t0=0.3)
    pl = D.Plan(xyz, tets, 1.0, 1.0, 3, "fp32", "upwind", "lsrk4", 1e-3)
    pl.set_incident([t[::-1] for t in z0], **wave)          # any vertex order
    for bad in ([inner[0]], [z0[0], z0[0]], [[0, 1, 10 ** 6]]):
        with pytest.raises(D.DgmError):
            pl.set_incident(bad, **wave)
    for kw in (dict(bw=0.0), dict(speed=-1.0), dict(t0=float("nan"))):
        with pytest.raises(D.DgmError):
            pl.set_incident(z0, **{**wave, **kw})
    pl.set_incident(z0, **wave)
    for v in (3, 4):
        assert D.STATUS[lib.dgm_set_variant(pl.handle, v)] == "DGM_EUNSUP"
    assert lib.dgm_set_variant(pl.handle, 0) == 0
    pl.set_incident([], **wave)                              # back to PEC everywhere
    assert lib.dgm_set_variant(pl.handle, 3) == 0
    for plan in (D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", "upwind", "lsrk4", 1e-3, mixed=True),
                 D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", "central", "leapfrog", 1e-3)):
        with pytest.raises(D.DgmError):
            plan.set_incident(z0, **wave)


def test_interior_penalty_plan_sizes_and_limits(lib):
    """dgm_set_sip: interior facets of a Kuhn grid, (4K - 12 n^2) / 2 of them;
    central flux and LSRK4 only, no PML, no mixed orders, alpha >= 0."""
    from paper_2002_08733_gb300 import dgmax as D
    n = 3
    xyz, tets = W.kuhn_mesh(n)
    K = len(tets)
    for p, prec, rs in ((1, "fp64", 8), (3, "fp32", 4)):
        pl = D.Plan(xyz, tets, 1.0, 1.0, p, prec, "central", "lsrk4", 1e-3, S=2, sip=5.0)
        nF = (4 * K - 12 * n * n) // 2
        assert pl.info.n_facets == nF
        assert pl.info.bytes_facets == nF * 2 * 3 * W.n_face_modes(p) * rs
        assert lib.dgm_set_variant(pl.handle, 3 if prec == "fp32" else 0) == (3 if prec == "fp32" else 0)
    assert D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", "central", "lsrk4", 1e-3).info.n_facets == 0
    pml = dict(lo=(0.25,) * 3, hi=(0.75,) * 3, thickness=0.25, sigma_max=10.0)
    for kw in (dict(flux="upwind"), dict(integrator="leapfrog"), dict(mixed=True), dict(pml=pml),
               dict(sip=-1.0)):
        args = dict(flux="central", integrator="lsrk4", sip=5.0)
        args.update(kw)
        with pytest.raises(D.DgmError):
            D.Plan(xyz, tets, 1.0, 1.0, 2, "fp64", args.pop("flux"), args.pop("integrator"), 1e-3,
                   **args)


def test_tile_load_choice_is_validated(lib):
    """dgm_set_tile_loads takes 0 (bulk copies where allowed) or 1 (per-thread
    loads); an unbound plan reports no bulk copies."""
    from paper_2002_08733_gb300 import dgmax as D
    xyz, tets = W.kuhn_mesh(4)
    pl = D.Plan(xyz, tets, 1.0, 1.0, 2, "fp32", "upwind", "lsrk4", 1e-3)
    bulk = ctypes.c_int32(7)
    assert lib.dgm_get_tile_loads(pl.handle, ctypes.byref(bulk)) == 0 and bulk.value == 0
    assert lib.dgm_set_tile_loads(pl.handle, 1) == 0
    assert lib.dgm_set_tile_loads(pl.handle, 0) == 0
    assert lib.dgm_set_tile_loads(pl.handle, 2) == 1          # DGM_EINVAL
    assert lib.dgm_get_tile_loads(pl.handle, None) == 1
