"""Python binding of the dgmax C ABI (include/dgmax.h).

Argument marshalling only: every step of the right-hand side and of the time
stepping runs in the CUDA kernels of libdgmax.so.  PyTorch provides device
memory and the stream.  There is no CPU fallback: if the library is missing
or fails to load, the constructor raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libdgmax.so")

FP64, FP32 = 0, 1
CENTRAL, UPWIND = 0, 1
LEAPFROG, LSRK4 = 0, 1

STATUS = {0: "DGM_OK", 1: "DGM_EINVAL", 2: "DGM_EMESH", 3: "DGM_EUNSUP", 4: "DGM_ECUDA",
          5: "DGM_ETIMEOUT", 6: "DGM_ENAN", 7: "DGM_ESTATE"}


class DgmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("precision", ctypes.c_int32), ("flux", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("n_columns", ctypes.c_int32),
                ("max_receivers", ctypes.c_int32), ("dt", ctypes.c_double)]


class Pml(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("thickness", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("order", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class HaloSizes(ctypes.Structure):
    _fields_ = [("n_owned", ctypes.c_int64), ("n_ghost", ctypes.c_int64),
                ("n_send", ctypes.c_int64), ("n_recv", ctypes.c_int64),
                ("n_peers", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Incident(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double * 3), ("direction", ctypes.c_double * 3),
                ("speed", ctypes.c_double), ("f0", ctypes.c_double), ("bw", ctypes.c_double),
                ("t0", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int64), ("n_pml", ctypes.c_int64), ("N", ctypes.c_int32),
                ("NF", ctypes.c_int32), ("S", ctypes.c_int32), ("real_size", ctypes.c_int32),
                ("bytes_fields", ctypes.c_size_t), ("bytes_aux", ctypes.c_size_t),
                ("bytes_geom", ctypes.c_size_t), ("n_quad", ctypes.c_int32),
                ("N_H", ctypes.c_int32), ("n_facets", ctypes.c_int64),
                ("bytes_facets", ctypes.c_size_t)]


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "dgm_plan_create": [ctypes.POINTER(_P), ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P,
                        ctypes.POINTER(Pml), ctypes.POINTER(Options)],
    "dgm_plan_create_mixed": [ctypes.POINTER(_P), ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P,
                              ctypes.POINTER(Pml), ctypes.POINTER(Options)],
    "dgm_plan_info": [_P, ctypes.POINTER(Info)],
    "dgm_bind": [_P, _P, _P, _P, _P, _P, _P, _P, _P],
    "dgm_set_sources": [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P],
    "dgm_set_receivers": [_P, ctypes.c_int32, _P],
    "dgm_sample_receivers": [_P, _P, _P],
    "dgm_rhs": [_P, _P, _P, _P, _P, ctypes.c_double],
    "dgm_leapfrog_start": [_P, ctypes.c_double],
    "dgm_advance": [_P, ctypes.c_int64, ctypes.c_double],
    "dgm_current": [_P],
    "dgm_advance_host": [_P, _P, _P, ctypes.c_int64, ctypes.c_double],
    "dgm_energy": [_P, _P, _P],
    "dgm_energy_noalloc": [_P, _P, _P],
    "dgm_pml_elements": [_P, _P],
    "dgm_quad_points": [_P, _P],
    "dgm_project": [_P, _P, ctypes.c_int32, _P],
    "dgm_status_check": [_P],
    "dgm_set_materials": [_P, _P, _P],
    "dgm_autotune": [_P, _P, ctypes.c_int32, _P],
    "dgm_autotune_info": [_P, _P, _P],
    "dgm_set_variant": [_P, ctypes.c_int32],
    "dgm_set_index64": [_P, ctypes.c_int32],
    "dgm_set_tile_loads": [_P, ctypes.c_int32],
    "dgm_get_tile_loads": [_P, ctypes.c_void_p],
    "dgm_set_tile_groups": [_P, ctypes.c_int32],
    "dgm_get_tile_groups": [_P, ctypes.c_void_p],
    "dgm_adjoint_workspace": [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)],
    "dgm_forward_record": [_P, ctypes.c_int64, ctypes.c_double, _P, _P],
    "dgm_adjoint": [_P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P],
    "dgm_batch_create": [ctypes.POINTER(_P), _P, ctypes.c_int32, _P],
    "dgm_batch_advance": [_P, ctypes.c_int64, _P],
    "dgm_batch_destroy": [_P],
    "dgm_partition_slabs": [ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int32,
                            ctypes.c_int32, _P],
    "dgm_halo_build": [ctypes.c_int64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                       _P, _P, _P],
    "dgm_set_active": [_P, ctypes.c_int64],
    "dgm_halo_pack": [_P, _P, _P, ctypes.c_int64, _P],
    "dgm_halo_unpack": [_P, _P, _P, ctypes.c_int64, _P],
    "dgm_stage": [_P, ctypes.c_int32, ctypes.c_double],
    "dgm_set_incident": [_P, ctypes.c_int64, _P, ctypes.POINTER(Incident)],
    "dgm_set_sip": [_P, ctypes.c_double],
    "dgm_bind_sip": [_P, _P, _P, _P],
    "dgm_last_error": [],
    "dgm_plan_destroy": [_P],
}


def load_library(path=LIB_PATH):
    """Load libdgmax.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdgmax.so not built (%s); run paper_2002_08733_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.dgm_last_error.restype = ctypes.c_char_p
    lib.dgm_plan_destroy.restype = None
    lib.dgm_batch_destroy.restype = None
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise DgmError(rc, _lib.dgm_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class Plan:
    """Host-side plan (mesh setup, reference matrices); no GPU needed."""

    def __init__(self, xyz, tets, eps, mu, p, precision="fp64", flux="upwind",
                 integrator="lsrk4", dt=1e-3, S=1, pml=None, max_receivers=0, mixed=False,
                 sip=None):
        """mixed=True: E of degree p + 1, H of degree p (dgm_plan_create_mixed);
        sip=alpha: interior penalty with a facet field (dgm_set_sip)."""
        lib = load_library()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int64)
        K = tets.shape[0]
        self.eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (K,)))
        self.mu = np.ascontiguousarray(np.broadcast_to(np.asarray(mu, np.float64), (K,)))
        opt = Options(p=p, precision={"fp64": FP64, "fp32": FP32}[precision],
                      flux={"central": CENTRAL, "upwind": UPWIND}[flux],
                      integrator={"leapfrog": LEAPFROG, "lsrk4": LSRK4}[integrator],
                      n_columns=S, max_receivers=max_receivers, dt=dt)
        pm = None
        if pml is not None:
            pm = Pml()
            pm.lo[:] = list(pml["lo"])
            pm.hi[:] = list(pml["hi"])
            pm.thickness = pml["thickness"]
            pm.sigma_max = pml["sigma_max"]
            pm.order = pml.get("order", 2)
        h = _P()
        create = lib.dgm_plan_create_mixed if mixed else lib.dgm_plan_create
        _check(create(ctypes.byref(h), xyz.shape[0], xyz.ctypes.data, K,
                      tets.ctypes.data, self.eps.ctypes.data, self.mu.ctypes.data,
                      ctypes.byref(pm) if pm is not None else None, ctypes.byref(opt)))
        self.mixed = bool(mixed)
        self.handle = h
        self.opt = opt
        self.precision = precision
        if sip:
            _check(lib.dgm_set_sip(h, float(sip)))
        self.sip = float(sip or 0.0)
        info = Info()
        _check(lib.dgm_plan_info(h, ctypes.byref(info)))
        self.info = info
        self.K, self.N, self.S, self.npml = info.K, info.N, info.S, info.n_pml
        self.NH = info.N_H
        self.p = p
        self.dt = dt

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dgm_plan_destroy(self.handle)
            self.handle = None

    def pml_elements(self):
        """Element ids carrying auxiliary fields, in auxiliary-buffer order."""
        if not hasattr(self, "_pml_el"):
            out = np.zeros(max(self.npml, 1), dtype=np.int64)
            _check(_lib.dgm_pml_elements(self.handle, out.ctypes.data))
            self._pml_el = out[:self.npml]
        return self._pml_el

    def quad_points(self):
        out = np.empty((self.K, self.info.n_quad, 3))
        _check(_lib.dgm_quad_points(self.handle, out.ctypes.data))
        return out

    def set_incident(self, faces, E0=(0.0, 0.0, 0.0), direction=(0.0, 0.0, 1.0), speed=1.0,
                     f0=0.0, bw=1.0, t0=0.0):
        """Incident plane wave E0 g(t - t0 - d.r/speed) entering through the
        boundary faces `faces` [n, 3] (vertex ids); an empty list restores PEC."""
        f = np.ascontiguousarray(np.asarray(faces, dtype=np.int64).reshape(-1, 3))
        w = Incident((ctypes.c_double * 3)(*map(float, E0)),
                     (ctypes.c_double * 3)(*map(float, direction)),
                     float(speed), float(f0), float(bw), float(t0))
        _check(_lib.dgm_set_incident(self.handle, len(f), f.ctypes.data if len(f) else None,
                                     ctypes.byref(w)))


class Solver(Plan):
    """Plan bound to caller-owned torch device buffers on one CUDA device."""

    def __init__(self, *args, device="cuda", stream=None, **kw):
        super().__init__(*args, **kw)
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:   # the current device
            self.device = torch.device("cuda", torch.cuda.current_device())
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        self.dtype = dt
        i = self.info
        # field buffer: rows (component, mode) -- 6 N of them, or 3 N + 3 N_H on a
        # mixed-order plan -- by (element, column)
        shape = (6, self.N, self.K, self.S) if not self.mixed else \
            (3 * (self.N + self.NH), self.K, self.S)
        self.geom = torch.empty(i.bytes_geom + 256, dtype=torch.uint8, device=self.device)
        off = (-self.geom.data_ptr()) % 256
        self.geom_view = self.geom[off:off + i.bytes_geom]
        self.fields = [torch.zeros(shape, dtype=dt, device=self.device) for _ in range(2)]
        self.res = torch.zeros(shape, dtype=dt, device=self.device)
        ashape = (6, self.N, self.npml, self.S)
        if self.npml > 0:
            self.aux = [torch.zeros(ashape, dtype=dt, device=self.device) for _ in range(2)]
            self.aux_res = torch.zeros(ashape, dtype=dt, device=self.device)
        else:
            self.aux = [None, None]
            self.aux_res = None
        self.stream = stream or torch.cuda.current_stream(self.device)
        torch.cuda.synchronize(self.device)   # allocations above ran on torch's stream
        _check(_lib.dgm_bind(self.handle, self.geom_view.data_ptr(), _ptr(self.fields[0]),
                             _ptr(self.fields[1]), _ptr(self.res), _ptr(self.aux[0]),
                             _ptr(self.aux[1]), _ptr(self.aux_res), self.stream.cuda_stream))
        self.hs = [None, None]
        self.hs_res = None
        if self.sip:   # facet field of the interior penalty: [3][NF][facet][column], from rest
            fshape = (3, i.NF, i.n_facets, self.S)
            self.hs = [torch.zeros(fshape, dtype=dt, device=self.device) for _ in range(2)]
            self.hs_res = torch.zeros(fshape, dtype=dt, device=self.device)
            torch.cuda.synchronize(self.device)
            _check(_lib.dgm_bind_sip(self.handle, _ptr(self.hs[self.current()]),
                                     _ptr(self.hs[1 - self.current()]), _ptr(self.hs_res)))

    # -- layout conversion between (K, S, 6, N) and the device layout [6][N][K][S]
    #    (mixed-order plans: H modes l >= N_H of the (K, S, 6, N) array are zero)
    def to_device(self, u):
        u = np.asarray(u)
        if self.mixed and u.shape[2] == 6:
            rows = np.concatenate([u[:, :, 0:3, :].reshape(u.shape[0], u.shape[1], -1),
                                   u[:, :, 3:6, :self.NH].reshape(u.shape[0], u.shape[1], -1)],
                                  axis=2)                               # (K, S, rows)
            t = self.torch.as_tensor(np.ascontiguousarray(np.transpose(rows, (2, 0, 1))))
            return t.to(device=self.device, dtype=self.dtype).contiguous()
        t = self.torch.as_tensor(np.ascontiguousarray(np.transpose(u, (2, 3, 0, 1))))
        return t.to(device=self.device, dtype=self.dtype).contiguous()

    def aux_to_device(self, aux_full):
        """aux given for all K elements (K, S, 6, N) -> compact PML layout."""
        idx = self.pml_elements()
        return self.to_device(np.asarray(aux_full)[idx])

    def from_device(self, t):
        a = t.double().cpu().numpy()
        if a.ndim == 3:   # mixed-order rows -> (K, S, 6, N) with H modes >= N_H zero
            N, NH = self.N, self.NH
            K, S = a.shape[1], a.shape[2]
            out = np.zeros((K, S, 6, N))
            r = np.transpose(a, (1, 2, 0))
            out[:, :, 0:3, :] = r[:, :, :3 * N].reshape(K, S, 3, N)
            out[:, :, 3:6, :NH] = r[:, :, 3 * N:].reshape(K, S, 3, NH)
            return out
        return np.transpose(a, (2, 3, 0, 1)).copy()


    def current(self):
        return _lib.dgm_current(self.handle)

    def set_state(self, u, aux=None):
        self.torch.cuda.synchronize(self.device)
        self.fields[self.current()].copy_(self.to_device(u))
        if aux is not None and self.npml > 0:
            self.aux[self.current()].copy_(aux if self.torch.is_tensor(aux) else self.to_device(aux))
        self.torch.cuda.synchronize(self.device)

    def state(self):
        self.torch.cuda.synchronize(self.device)
        return self.from_device(self.fields[self.current()])

    def facet_state(self):
        """Facet field of the interior penalty -> (n_facets, S, 3, NF) float64."""
        self.torch.cuda.synchronize(self.device)
        return np.transpose(self.hs[self.current()].double().cpu().numpy(), (2, 3, 0, 1)).copy()

    def facet_rhs(self):
        """dh_s/dt written by the last rhs() call -> (n_facets, S, 3, NF)."""
        self.torch.cuda.synchronize(self.device)
        return np.transpose(self.hs_res.double().cpu().numpy(), (2, 3, 0, 1)).copy()

    def set_facet_state(self, hs):
        """hs: (n_facets, S, 3, NF)."""
        self.torch.cuda.synchronize(self.device)
        t = self.torch.as_tensor(np.ascontiguousarray(np.transpose(np.asarray(hs), (2, 3, 0, 1))))
        self.hs[self.current()].copy_(t.to(self.hs[0]))
        self.torch.cuda.synchronize(self.device)

    def rhs(self, u, aux=None, t=0.0):
        """One right-hand-side evaluation; u: (K, S, 6, N) array -> du (same shape)."""
        ud = u if self.torch.is_tensor(u) else self.to_device(u)
        du = self.torch.empty_like(ud)
        ad = dad = None
        if self.npml > 0:
            ad = aux if self.torch.is_tensor(aux) else (
                self.to_device(aux) if aux is not None else self.torch.zeros_like(self.aux[0]))
            dad = self.torch.empty_like(ad)
        _check(_lib.dgm_rhs(self.handle, _ptr(ud), _ptr(ad), _ptr(du), _ptr(dad), t))
        self.torch.cuda.synchronize(self.device)
        if self.npml > 0:
            return du, dad
        return du

    def advance(self, n_steps, t0=0.0):
        _check(_lib.dgm_advance(self.handle, int(n_steps), float(t0)))

    def leapfrog_start(self, t0=0.0):
        _check(_lib.dgm_leapfrog_start(self.handle, float(t0)))

    def advance_host(self, host_in, host_out, n_steps, t0=0.0):
        """End-to-end call from host memory (torch pinned CPU tensors or numpy arrays)."""
        _check(_lib.dgm_advance_host(self.handle, _ptr(host_in), _ptr(host_out), int(n_steps),
                                     float(t0)))

    def energy(self, fields=None):
        f = self.fields[self.current()] if fields is None else fields
        out = np.zeros(self.S)
        _check(_lib.dgm_energy(self.handle, _ptr(f), out.ctypes.data))
        return out

    def energy_noalloc(self, out, fields=None):
        """Allocation-free energy into the device tensor `out` (S doubles) on the
        bound stream; the library's own fixed scratch array holds the partial sums.

        `out` must be a contiguous float64 CUDA tensor on the plan's device with
        at least S elements: the kernel writes it directly, so anything else is
        rejected here, before the library is called."""
        self._check_device_tensor(out, self.torch.float64, self.S, "out")
        f = self.fields[self.current()] if fields is None else fields
        self._check_device_tensor(f, self.dtype, 6 * self.N * self.K * self.S, "fields")
        _check(_lib.dgm_energy_noalloc(self.handle, _ptr(f), _ptr(out)))

    def _check_device_tensor(self, t, dtype, min_numel, name):
        """A buffer the kernels read or write directly: a contiguous torch tensor
        of `dtype` on this plan's CUDA device with at least `min_numel` elements."""
        torch = self.torch
        if not torch.is_tensor(t):
            raise ValueError("%s must be a torch tensor on %s, got %s" % (name, self.device,
                                                                          type(t).__name__))
        if not t.is_cuda or t.device.index != self.device.index:
            raise ValueError("%s must live on %s, got %s" % (name, self.device, t.device))
        if t.dtype != dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() < min_numel:
            raise ValueError("%s needs at least %d elements, got %d" % (name, min_numel,
                                                                         t.numel()))

    def project(self, fn, column=0):
        """L2 projection of fn(points [n,3]) -> [n,6] (E, H) into the current state."""
        pts = self.quad_points()
        vals = np.ascontiguousarray(fn(pts.reshape(-1, 3)).reshape(self.K, -1, 6), dtype=np.float64)
        _check(_lib.dgm_project(self.handle, vals.ctypes.data, column,
                                _ptr(self.fields[self.current()])))

    def set_sources(self, sources):
        """sources: list over columns of dict(pos, dir, f0, bw, t0) or None."""
        cols, pos, dirs, f0, bw, t0 = [], [], [], [], [], []
        for s, rec in enumerate(sources):
            if rec is None:
                continue
            cols.append(s)
            pos.extend(rec["pos"])
            dirs.extend(rec["dir"])
            f0.append(rec["f0"])
            bw.append(rec["bw"])
            t0.append(rec["t0"])
        arr = [np.ascontiguousarray(v, dtype=np.float64) for v in (pos, dirs, f0, bw, t0)]
        c = np.ascontiguousarray(cols, dtype=np.int32)
        _check(_lib.dgm_set_sources(self.handle, len(cols), c.ctypes.data,
                                    *[a.ctypes.data for a in arr]))

    def set_receivers(self, pos):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.n_rec = len(pos)
        _check(_lib.dgm_set_receivers(self.handle, len(pos), pos.ctypes.data))

    def sample_receivers(self, out=None, fields=None):
        """E at the receivers for every column -> device tensor [S, R, 3] (float64)."""
        f = self.fields[self.current()] if fields is None else fields
        if out is None:
            out = self.torch.empty((self.S, self.n_rec, 3), dtype=self.torch.float64,
                                   device=self.device)
        _check(_lib.dgm_sample_receivers(self.handle, _ptr(f), _ptr(out)))
        return out

    def autotune(self, reps=3):
        """Pick the fastest tile shape of the LSRK4 stage kernel; returns (chosen, ms per variant)."""
        nb = 2 * (-(-self.info.bytes_fields // 256) * 256) + 2 * (-(-self.info.bytes_aux // 256) * 256)
        buf = self.torch.empty(nb + 256, dtype=self.torch.uint8, device=self.device)
        off = (-buf.data_ptr()) % 256
        nv, ch = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.dgm_autotune_info(self.handle, ctypes.byref(nv), ctypes.byref(ch)))
        ms = np.zeros(nv.value, dtype=np.float32)
        _check(_lib.dgm_autotune(self.handle, buf.data_ptr() + off, int(reps), ms.ctypes.data))
        _check(_lib.dgm_autotune_info(self.handle, ctypes.byref(nv), ctypes.byref(ch)))
        del buf
        return ch.value, ms

    def set_variant(self, v):
        _check(_lib.dgm_set_variant(self.handle, int(v)))

    def set_tile_groups(self, groups):
        """Tile visiting order of the stage kernels (1: plain order)."""
        _check(_lib.dgm_set_tile_groups(self.handle, int(groups)))

    def tile_groups(self):
        g = ctypes.c_int32()
        _check(_lib.dgm_get_tile_groups(self.handle, ctypes.byref(g)))
        return g.value

    def set_index64(self, force=True):
        """Force 64-bit index arithmetic in the stage kernels (default: automatic)."""
        _check(_lib.dgm_set_index64(self.handle, int(bool(force))))

    def set_tile_loads(self, per_thread=True):
        """Force per-thread tile loads in phase 1 of the stage kernels (default:
        tiled bulk copies where the plan allows them)."""
        _check(_lib.dgm_set_tile_loads(self.handle, int(bool(per_thread))))

    def bulk_tile_loads(self):
        """True when the next stages move their tiles with tiled bulk copies."""
        b = ctypes.c_int32()
        _check(_lib.dgm_get_tile_loads(self.handle, ctypes.byref(b)))
        return bool(b.value)

    def set_materials(self, eps, mu):
        eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (self.K,)))
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(mu, np.float64), (self.K,)))
        _check(_lib.dgm_set_materials(self.handle, eps.ctypes.data, mu.ctypes.data))

    def adjoint_workspace(self, n_steps):
        """Caller-owned device workspace for forward_record / adjoint (256-byte aligned view)."""
        nb = ctypes.c_size_t()
        _check(_lib.dgm_adjoint_workspace(self.handle, int(n_steps), ctypes.byref(nb)))
        buf = self.torch.empty(nb.value + 256, dtype=self.torch.uint8, device=self.device)
        off = (-buf.data_ptr()) % 256
        return buf[off:off + nb.value]

    def forward_record(self, n_steps, t0, workspace):
        """Advance n_steps recording E at the receivers -> device tensor [n, S, R, 3]."""
        rec = self.torch.empty((n_steps, self.S, self.n_rec, 3), dtype=self.torch.float64,
                               device=self.device)
        _check(_lib.dgm_forward_record(self.handle, int(n_steps), float(t0), _ptr(rec),
                                       _ptr(workspace)))
        return rec

    def adjoint(self, n_steps, t0, drecords, workspace):
        """dL/deps, dL/dmu (device float64 [K]) from dL/drecords [n, S, R, 3]."""
        d = drecords.to(device=self.device, dtype=self.torch.float64).contiguous()
        deps = self.torch.empty(self.K, dtype=self.torch.float64, device=self.device)
        dmu = self.torch.empty_like(deps)
        _check(_lib.dgm_adjoint(self.handle, int(n_steps), float(t0), _ptr(d), _ptr(workspace),
                                _ptr(deps), _ptr(dmu)))
        self.torch.cuda.synchronize(self.device)
        return deps, dmu

    def status(self):
        _check(_lib.dgm_status_check(self.handle))

    def set_active(self, n):
        """Update only the first n elements (the rest are halo copies)."""
        _check(_lib.dgm_set_active(self.handle, int(n)))

    def stage(self, k, t):
        """LSRK4 stage k (0..4) of the step starting at time t."""
        _check(_lib.dgm_stage(self.handle, int(k), float(t)))

    def halo_pack(self, idx_device, out=None, fields=None):
        """Coefficients of the elements idx_device (int64 device tensor) -> [6N, n, S]."""
        f = self.fields[self.current()] if fields is None else fields
        n = int(idx_device.numel())
        if out is None:
            out = self.torch.empty((3 * (self.N + self.NH), n, self.S), dtype=self.dtype,
                                   device=self.device)
        _check(_lib.dgm_halo_pack(self.handle, _ptr(f), _ptr(idx_device), n, _ptr(out)))
        return out

    def halo_unpack(self, idx_device, buf, fields=None):
        f = self.fields[self.current()] if fields is None else fields
        _check(_lib.dgm_halo_unpack(self.handle, _ptr(f), _ptr(idx_device), int(idx_device.numel()),
                                    _ptr(buf)))


class Batch:
    """Several bound LSRK4 solvers advanced together by one graph launch per two steps."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        self.stream = stream or torch.cuda.current_stream()
        arr = (_P * len(self.solvers))(*[s.handle for s in self.solvers])
        h = _P()
        _check(_lib.dgm_batch_create(ctypes.byref(h), arr, len(self.solvers),
                                     self.stream.cuda_stream))
        self.handle = h
        self._keep = arr
        self.t = np.zeros(len(self.solvers))

    def advance(self, n_steps, t0=None):
        t = self.t if t0 is None else np.ascontiguousarray(t0, dtype=np.float64)
        _check(_lib.dgm_batch_advance(self.handle, int(n_steps), t.ctypes.data))
        self.t = t + n_steps * np.array([s.dt for s in self.solvers])

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dgm_batch_destroy(self.handle)
            self.handle = None


def receiver_records(solver, eps, mu, n_steps, t0=0.0, u0=None, aux0=None):
    """Receiver records [n, S, R, 3] as a differentiable function of per-element
    eps and mu (torch float64 tensors [K]); backward runs the hand-written
    adjoint kernels with sqrt(N) checkpointing (dgm_forward_record / dgm_adjoint)."""
    import torch

    class _Records(torch.autograd.Function):
        @staticmethod
        def forward(ctx, e, m):
            solver.set_materials(e.detach().cpu().numpy(), m.detach().cpu().numpy())
            if u0 is None:   # start from rest without a host round trip
                solver.torch.cuda.synchronize(solver.device)
                solver.fields[solver.current()].zero_()
            else:
                solver.set_state(u0)
            if solver.npml:
                solver.aux[solver.current()].zero_()
                if aux0 is not None:
                    solver.aux[solver.current()].copy_(solver.aux_to_device(aux0))
            solver.torch.cuda.synchronize(solver.device)   # fills above ran on torch's stream
            ws = solver.adjoint_workspace(n_steps)
            rec = solver.forward_record(n_steps, t0, ws)
            ctx.ws = ws
            return rec

        @staticmethod
        def backward(ctx, grad):
            deps, dmu = solver.adjoint(n_steps, t0, grad, ctx.ws)
            return deps.to(eps.device), dmu.to(mu.device)

    return _Records.apply(eps, mu)



# -- one mesh on several GPUs ------------------------------------------------------------

def partition_slabs(xyz, tets, nparts, axis=2):
    """Part id per element: slabs of nearly equal size along `axis` (dgm_partition_slabs)."""
    lib = load_library()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    part = np.empty(len(tets), dtype=np.int32)
    _check(lib.dgm_partition_slabs(len(xyz), xyz.ctypes.data, len(tets), tets.ctypes.data,
                                   int(axis), int(nparts), part.ctypes.data))
    return part


class Halo:
    """Part `rank` of an element partition: local numbering (owned elements, then
    ghosts, each in ascending global id) and, per peer part, the local ids sent
    to it and received from it (dgm_halo_build).  No GPU needed."""

    def __init__(self, tets, part, nparts, rank):
        lib = load_library()
        tets = np.ascontiguousarray(tets, dtype=np.int64)
        part = np.ascontiguousarray(part, dtype=np.int32)
        sz = HaloSizes()
        _check(lib.dgm_halo_build(len(tets), tets.ctypes.data, part.ctypes.data, int(nparts),
                                  int(rank), ctypes.byref(sz), None, None, None, None, None, None))
        self.n_owned, self.n_ghost, self.rank = sz.n_owned, sz.n_ghost, rank
        self.local_to_global = np.empty(sz.n_owned + sz.n_ghost, dtype=np.int64)
        self.peers = np.empty(max(sz.n_peers, 1), dtype=np.int32)
        sc = np.empty(max(sz.n_peers, 1), dtype=np.int64)
        rc = np.empty(max(sz.n_peers, 1), dtype=np.int64)
        si = np.empty(max(sz.n_send, 1), dtype=np.int64)
        ri = np.empty(max(sz.n_recv, 1), dtype=np.int64)
        _check(lib.dgm_halo_build(len(tets), tets.ctypes.data, part.ctypes.data, int(nparts),
                                  int(rank), ctypes.byref(sz), self.local_to_global.ctypes.data,
                                  self.peers.ctypes.data, sc.ctypes.data, si.ctypes.data,
                                  rc.ctypes.data, ri.ctypes.data))
        self.peers = self.peers[:sz.n_peers]
        so = np.concatenate([[0], np.cumsum(sc[:sz.n_peers])])
        ro = np.concatenate([[0], np.cumsum(rc[:sz.n_peers])])
        self.send = [si[so[q]:so[q + 1]].copy() for q in range(sz.n_peers)]
        self.recv = [ri[ro[q]:ro[q + 1]].copy() for q in range(sz.n_peers)]

    def exchange(self, pack, unpack, isend, irecv, empty_like_recv):
        """One halo refresh: receive buffers posted for every peer, this part's
        send lists packed and sent, then the received coefficients unpacked into
        the ghosts.  pack(q) -> buffer of peer q's send list, unpack(q, buffer),
        isend(buffer, peer) / irecv(buffer, peer) -> request with wait(),
        empty_like_recv(q) -> receive buffer for peer q (e.g. torch.distributed
        isend/irecv over NCCL or gloo)."""
        reqs, bufs = [], []
        for q, peer in enumerate(self.peers):
            b = empty_like_recv(q)
            bufs.append(b)
            reqs.append(irecv(b, int(peer)))
        for q, peer in enumerate(self.peers):
            reqs.append(isend(pack(q), int(peer)))
        for r in reqs:
            r.wait()
        for q in range(len(self.peers)):
            unpack(q, bufs[q])


class PartitionedSolver:
    """This rank's part of a mesh partitioned over ranks (one GPU each): a
    Solver over its owned elements plus their halo, stepping LSRK4 stage by
    stage with a halo exchange after each stage.

    exchange: 'dist' (torch.distributed point-to-point, NCCL on GPUs) or None
    for parts driven together by exchange_local (several parts in one process)."""

    def __init__(self, xyz, tets, eps, mu, p, precision, flux, dt, part, nparts, rank,
                 pml=None, S=1, device="cuda", exchange="dist"):
        import torch
        self.halo = Halo(tets, part, nparts, rank)
        l2g = self.halo.local_to_global
        tets = np.asarray(tets)
        K = len(tets)
        eps = np.broadcast_to(np.asarray(eps, np.float64), (K,))[l2g]
        mu = np.broadcast_to(np.asarray(mu, np.float64), (K,))[l2g]
        self.solver = Solver(xyz, tets[l2g], eps, mu, p, precision, flux, "lsrk4", dt, S=S,
                             pml=pml, device=device)
        self._verts = np.asarray(xyz, np.float64)[tets[l2g]]   # local elements' vertices
        self.solver.set_active(self.halo.n_owned)
        dev = self.solver.device
        self.send_idx = [torch.as_tensor(a, device=dev) for a in self.halo.send]
        self.recv_idx = [torch.as_tensor(a, device=dev) for a in self.halo.recv]
        self.mode = exchange
        self.rank = rank

    def _applies(self, pos, tol=1e-12):
        """Whether this part applies a point source at pos: the lowest global id
        among the local elements containing it (owned and ghosts) is owned."""
        V = self._verts
        A = np.transpose(V[:, 1:] - V[:, :1], (0, 2, 1))          # columns: edges
        lam = np.linalg.solve(A, (np.asarray(pos, np.float64) - V[:, 0])[:, :, None])[:, :, 0]
        inside = np.all(lam >= -tol, axis=1) & (lam.sum(axis=1) <= 1 + tol)
        if not inside.any():
            return False
        loc = np.nonzero(inside)[0]
        return bool(loc[np.argmin(self.halo.local_to_global[loc])] < self.halo.n_owned)

    def set_sources(self, sources):
        """Point dipoles per column (as Solver.set_sources); each is applied by
        the part that owns its element."""
        self.solver.set_sources([rec if rec is not None and self._applies(rec["pos"]) else None
                                 for rec in sources])

    # state in global element ids
    def set_state(self, u_global):
        self.solver.set_state(np.asarray(u_global)[self.halo.local_to_global])

    def owned_state(self):
        """(global ids of the owned elements, their coefficients (n_owned, S, 6, N))."""
        u = self.solver.state()
        n = self.halo.n_owned
        return self.halo.local_to_global[:n], u[:n]

    def refresh_halo(self):
        import torch
        import torch.distributed as dist
        g = self.solver
        torch.cuda.synchronize(g.device)   # this stage's outputs are complete
        self.halo.exchange(
            pack=lambda q: g.halo_pack(self.send_idx[q]),
            unpack=lambda q, b: g.halo_unpack(self.recv_idx[q], b),
            isend=lambda b, peer: dist.isend(b, peer),
            irecv=lambda b, peer: dist.irecv(b, peer),
            empty_like_recv=lambda q: torch.empty((3 * (g.N + g.NH), len(self.halo.recv[q]), g.S),
                                                  dtype=g.dtype, device=g.device))

    def advance(self, n_steps, t0=0.0):
        t = t0
        for _ in range(n_steps):
            for k in range(5):
                self.solver.stage(k, t)
                self.refresh_halo()
            t += self.solver.dt


def exchange_local(parts):
    """Halo refresh of several parts held by one process (one device, or peer
    copies between devices): each part's send list to a peer is packed and
    unpacked straight into that peer's ghosts.  No kernel waits on another."""
    import torch
    by_rank = {pt.rank: pt for pt in parts}
    for pt in parts:
        torch.cuda.synchronize(pt.solver.device)
    for pt in parts:
        for q, peer in enumerate(pt.halo.peers):
            other = by_rank[int(peer)]
            qq = int(np.nonzero(other.halo.peers == pt.rank)[0][0])
            buf = pt.solver.halo_pack(pt.send_idx[q])
            if buf.device != other.solver.device:
                buf = buf.to(other.solver.device)
            other.solver.halo_unpack(other.recv_idx[qq], buf)
    for pt in parts:
        torch.cuda.synchronize(pt.solver.device)


def advance_local(parts, n_steps, t0=0.0):
    """LSRK4 steps of several parts held by one process, halos refreshed after
    every stage (exchange_local)."""
    t = t0
    dt = parts[0].solver.dt
    for _ in range(n_steps):
        for k in range(5):
            for pt in parts:
                pt.solver.stage(k, t)
            exchange_local(parts)
        t += dt
