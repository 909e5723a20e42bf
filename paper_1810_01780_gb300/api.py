"""Torch-level binding of the C ABI (device memory and streams from PyTorch; no compute here).

Every function marshals tensors into the structs of include/rp.h and calls the CUDA
library.  Tensors must live on the current CUDA device; ray arrays are float64 (3, n)
structure-of-arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _abi as A


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_f64(x, shape=None):
    t = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    t = t.contiguous()
    if shape is not None:
        t = t.reshape(shape)
    return t


class Medium:
    """A refractivity model on the device (rp_medium_create / rp_medium_destroy)."""

    def __init__(self, desc: dict, stream=None):
        A.lib()
        d = A.MediumDesc()
        self.desc = desc
        self._keep = None
        if desc["kind"] == "layered":
            layers = desc["layers"]
            if not 1 <= len(layers) <= A.MAX_LAYERS:
                raise ValueError("1..8 layers")
            d.kind = 0
            d.n_layers = len(layers)
            for k, L in enumerate(layers):
                d.layers[k].z_top = float(L.get("z_top", -np.inf)) if k else 0.0
                d.layers[k].n0 = float(L["n0"])
                d.layers[k].dn = float(L.get("dn", 0.0))
                d.layers[k].z0 = float(L.get("z0", 1.0))
                d.layers[k].offset = float(L.get("off", 0.0))
                d.layers[k].absorb = int(bool(L.get("absorb", False)))
            spheres = desc.get("spheres", [])
            if len(spheres) > A.MAX_SPHERES:
                raise ValueError("at most %d spheres" % A.MAX_SPHERES)
            d.n_spheres = len(spheres)
            for j, S in enumerate(spheres):
                for a in range(3):
                    d.spheres[j].center[a] = float(S["center"][a])
                d.spheres[j].radius = float(S["radius"])
                d.spheres[j].n0 = float(S["n0"])
                d.spheres[j].dn = float(S.get("dn", 0.0))
                d.spheres[j].z0 = float(S.get("z0", 1.0))
                d.spheres[j].offset = float(S.get("off", 0.0))
                d.spheres[j].absorb = int(bool(S.get("absorb", False)))
            surfaces = desc.get("surfaces", [])
            if len(surfaces) > A.MAX_LAYERS:
                raise ValueError("at most %d surfaces" % A.MAX_LAYERS)
            d.n_surfaces = len(surfaces)
            keep = []
            for j, srf in enumerate(surfaces):
                q = d.surfaces[j]
                q.layer = int(srf["layer"])
                for a in range(3):
                    q.normal[a] = float(srf.get("normal", (0.0, 0.0, 1.0))[a])
                if srf.get("height") is not None:
                    h = np.ascontiguousarray(srf["height"], dtype=np.float64)  # (ny, nx)
                    q.ny, q.nx = h.shape
                    for a in range(2):
                        q.origin[a] = float(srf["origin"][a])
                        q.spacing[a] = float(srf["spacing"][a])
                    q.height = h.ctypes.data
                    keep.append(h)
            self._keep = keep
        elif desc["kind"] == "grid":
            n = desc["n"]
            if isinstance(n, torch.Tensor):
                n = n.to(device="cuda", dtype=torch.float32).contiguous()
                nz, ny, nx = n.shape
                d.grid_n = n.data_ptr()
            else:
                n = np.ascontiguousarray(n, dtype=np.float32)
                nz, ny, nx = n.shape
                d.grid_n = n.ctypes.data
            self._keep = n
            d.kind = 1
            d.n_layers = 1
            d.nx, d.ny, d.nz = nx, ny, nz
            for a in range(3):
                d.origin[a] = float(desc["origin"][a])
            d.spacing = float(desc["spacing"])
        else:
            raise ValueError(desc["kind"])
        h = C.c_void_p()
        A.check(A.lib().rp_medium_create(C.byref(d), C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self._keep = None
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            A.lib().rp_medium_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(p: dict, precision: str = "fp64") -> A.TraceParams:
    q = A.TraceParams()
    q.tol = p["tol"]
    q.h_min = p["h_min"]
    q.h_max = p["h_max"]
    q.h0 = p.get("h0", p["h_max"])
    q.max_path = p.get("max_path", 0.0)
    q.max_time = p.get("max_time", 0.0)
    q.min_amp = p.get("min_amp", 0.0)
    q.eps_b = p.get("eps_b", 1e-9)
    stop = p.get("stop")
    if stop is not None:
        q.use_stop = 1
        for a in range(3):
            q.stop_n[a] = stop[0][a]
        q.stop_d = stop[1]
    q.max_generation = p.get("max_generation", 3)
    q.precision = A.PRECISION[precision]
    q.polarization = A.POLARIZATION[p.get("polarization", "s")]
    q.rhs_form = A.RHS_FORM[p.get("rhs_form", "projected")]
    q.max_steps = int(p.get("max_steps", 1_000_000))
    # scheduling knobs (0: the library's default); they never change a ray's record
    for k in SCHEDULING_KNOBS:
        setattr(q, k, int(p.get(k, 0)))
    return q


SCHEDULING_KNOBS = ("service_idle", "flush_min", "block", "blocks_per_sm", "ray_order")


RAY_FIELDS_F64 = ("path", "time", "amp")
RAY_FIELDS_I32 = ("status", "generation", "seq", "layer", "n_acc", "n_rej", "n_root", "n_refl",
                  "n_turn")


class TraceBuffers:
    """Preallocated device outputs for repeated rp_trace calls."""

    def __init__(self, capacity: int, hit_capacity: int = 0, fields=None):
        self.capacity = int(capacity)
        self.hit_capacity = int(hit_capacity)
        f = dict(device="cuda")
        want = set(fields) if fields is not None else None

        def need(name):
            return want is None or name in want

        self.t = {"end_pos": torch.empty((3, self.capacity), dtype=torch.float64, **f)}
        if need("end_dir"):
            self.t["end_dir"] = torch.empty((3, self.capacity), dtype=torch.float64, **f)
        for k in RAY_FIELDS_F64:
            if need(k):
                self.t[k] = torch.empty(self.capacity, dtype=torch.float64, **f)
        for k in RAY_FIELDS_I32:
            if need(k):
                self.t[k] = torch.empty(self.capacity, dtype=torch.int32, **f)
        if need("parent"):
            self.t["parent"] = torch.empty(self.capacity, dtype=torch.int64, **f)
        self.out = A.RayOut()
        self.out.capacity = self.capacity
        for name, t in self.t.items():
            setattr(self.out, name, t.data_ptr())
        self.h = {}
        self.hits = None
        if self.hit_capacity > 0:
            hc = self.hit_capacity
            self.h = {
                "ray": torch.empty(hc, dtype=torch.int64, **f),
                "receiver": torch.empty(hc, dtype=torch.int32, **f),
                "time": torch.empty(hc, dtype=torch.float64, **f),
                "path": torch.empty(hc, dtype=torch.float64, **f),
                "amp": torch.empty(hc, dtype=torch.float64, **f),
                "pos": torch.empty((3, hc), dtype=torch.float64, **f),
                "dir": torch.empty((3, hc), dtype=torch.float64, **f),
            }
            self.hits = A.Hits()
            self.hits.capacity = hc
            for name, t in self.h.items():
                setattr(self.hits, name, t.data_ptr())


class PreparedRays:
    """Device copies of a ray batch and its receivers, marshalled once."""

    def __init__(self, pos, dir, amp=None, receivers=None):
        self.pos = _dev_f64(pos, (3, -1))
        self.dir = _dev_f64(dir, (3, -1))
        self.n = self.pos.shape[1]
        self.amp = None if amp is None else _dev_f64(amp)
        self.rays = A.Rays(self.n, self.pos.data_ptr(), self.dir.data_ptr(),
                           0 if self.amp is None else self.amp.data_ptr())
        self.rx = None
        if receivers is not None and len(receivers[1]) > 0:
            if all(isinstance(a, torch.Tensor) and a.is_cuda for a in receivers[:2]):
                self.rx_c = _dev_f64(receivers[0], (-1, 3))
                self.rx_r = _dev_f64(receivers[1])
            else:  # host arrays: the library reads them during each call, no read-back
                self.rx_c = torch.as_tensor(receivers[0], dtype=torch.float64).reshape(-1, 3).contiguous()
                self.rx_r = torch.as_tensor(receivers[1], dtype=torch.float64).contiguous()
            self.rx = A.Receivers(len(self.rx_r), 0, self.rx_c.data_ptr(), self.rx_r.data_ptr())


def trace_into(medium: Medium, rays: PreparedRays, params: A.TraceParams, buf: TraceBuffers,
               stream=None, allow_overflow=False) -> A.Stats:
    """One rp_trace call into preallocated buffers; returns the stats struct."""
    st = A.Stats()
    rc = A.lib().rp_trace(medium.handle, C.byref(rays.rays),
                          C.byref(rays.rx) if rays.rx is not None else None, C.byref(params),
                          C.byref(buf.out), C.byref(buf.hits) if buf.hits is not None else None,
                          C.byref(st), C.c_void_p(_stream_ptr(stream)))
    A.check(rc, allow_overflow=allow_overflow)
    st.rc = rc
    return st


def trace(medium: Medium, pos, dir, amp=None, params: dict | None = None, receivers=None,
          precision: str = "fp64", capacity: int | None = None, hit_capacity: int | None = None,
          stream=None) -> dict:
    """Traces primaries and their secondaries; grows the buffers and retries on overflow.

    Returns {"rays": {field: tensor[:n_rays]}, "hits": {...}, "stats": dict}."""
    rays = PreparedRays(pos, dir, amp, receivers)
    prm = make_params(params, precision)
    cap = capacity or max(16, 4 * rays.n)
    hcap = hit_capacity if hit_capacity is not None else (max(16, rays.n) if rays.rx else 0)
    while True:
        buf = TraceBuffers(cap, hcap)
        st = trace_into(medium, rays, prm, buf, stream, allow_overflow=True)
        if st.rc == A.RP_OK:
            break
        cap = max(cap, int(st.rays) + 16)
        hcap = max(hcap, int(st.hits) + 16)
    n = int(st.rays)
    out = {k: (v[:, :n] if v.dim() == 2 else v[:n]) for k, v in buf.t.items()}
    nh = int(st.hits) if buf.hits is not None else 0
    hits = {k: (v[:, :nh] if v.dim() == 2 else v[:nh]) for k, v in buf.h.items()}
    return {"rays": out, "hits": hits, "stats": st.as_dict()}


SOL_FIELDS = (("type", torch.int32), ("n_iter", torch.int32), ("launch", torch.float64),
              ("receive", torch.float64), ("time", torch.float64), ("path", torch.float64),
              ("amp", torch.float64), ("miss", torch.float64))


class PathBuffers:
    """Device inputs and outputs of rp_find_paths for a batch of pairs."""

    def __init__(self, zs, zr, dist, n_angles, max_sol: int = 4):
        self.zs = _dev_f64(zs)
        self.zr = _dev_f64(zr)
        self.dist = _dev_f64(dist)
        self.n_angles = torch.as_tensor(n_angles, dtype=torch.int32, device="cuda").contiguous()
        self.n = self.zs.numel()
        self.max_sol = int(max_sol)
        self.count = torch.zeros(self.n, dtype=torch.int32, device="cuda")
        self.t = {k: torch.zeros((self.n, self.max_sol), dtype=dt, device="cuda")
                  for k, dt in SOL_FIELDS}
        self.sol = A.Solutions(self.count.data_ptr(), *[self.t[k].data_ptr() for k, _ in SOL_FIELDS])


def make_path_params(p: dict, precision: str = "fp64", hit_tol: float = 0.1, max_iter: int = 60,
                     max_sol: int = 4) -> A.PathParams:
    q = A.PathParams()
    q.trace = make_params(dict(p, max_path=p.get("max_path", 1.0)), precision)
    q.hit_tol = hit_tol
    q.max_iter = max_iter
    q.max_sol = max_sol
    return q


def find_paths_into(medium: Medium, buf: PathBuffers, prm: A.PathParams, stream=None,
                    allow_overflow=False) -> A.Stats:
    st = A.Stats()
    rc = A.lib().rp_find_paths(medium.handle, buf.n, C.c_void_p(buf.zs.data_ptr()),
                               C.c_void_p(buf.zr.data_ptr()), C.c_void_p(buf.dist.data_ptr()),
                               C.c_void_p(buf.n_angles.data_ptr()), C.byref(prm),
                               C.byref(buf.sol), C.byref(st), C.c_void_p(_stream_ptr(stream)))
    A.check(rc, allow_overflow=allow_overflow)
    st.rc = rc
    return st


def find_paths(medium: Medium, zs, zr, dist, n_angles, params: dict, precision: str = "fp64",
               hit_tol: float = 0.1, max_iter: int = 60, max_sol: int = 4, stream=None) -> dict:
    """Batched source-receiver path finding; returns count, per-slot solution fields, stats."""
    buf = PathBuffers(zs, zr, dist, n_angles, max_sol)
    prm = make_path_params(params, precision, hit_tol, max_iter, max_sol)
    st = find_paths_into(medium, buf, prm, stream)
    out = {"count": buf.count}
    out.update(buf.t)
    out["stats"] = st.as_dict()
    return out


class Surrogate:
    """The surrogate network on the device (rp_surrogate_*)."""

    def __init__(self, params=None, seed: int = 0):
        from . import workloads as Wl

        A.lib()
        if params is None:
            params = Wl.mlp_flatten(*Wl.mlp_init(seed))
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != A.lib().rp_surrogate_n_params():
            raise ValueError("parameter vector has the wrong length")
        h = C.c_void_p()
        A.check(A.lib().rp_surrogate_create(C.c_void_p(params.ctypes.data), C.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            A.lib().rp_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(A.lib().rp_surrogate_n_params(), dtype=np.float32)
        A.check(A.lib().rp_surrogate_get_params(self.handle, C.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        A.check(A.lib().rp_surrogate_set_params(self.handle, C.c_void_p(params.ctypes.data)))

    def set_wait_limit(self, cycles: int = 0):
        """Bound on the tensor-core kernels' mbarrier waits [SM cycles]; 0: the default."""
        A.check(A.lib().rp_surrogate_set_wait_limit(self.handle, int(cycles)))

    @staticmethod
    def _f32(x, cols):
        t = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
        return t.reshape(-1, cols)

    def forward(self, x, stream=None):
        x = self._f32(x, 3)
        out = torch.empty((x.shape[0], 12), dtype=torch.float32, device="cuda")
        A.check(A.lib().rp_surrogate_forward(self.handle, x.shape[0], C.c_void_p(x.data_ptr()),
                                             C.c_void_p(out.data_ptr()),
                                             C.c_void_p(_stream_ptr(stream))))
        return out

    def loss_grad(self, x, y, t, stream=None):
        x, y, t = self._f32(x, 3), self._f32(y, 2), self._f32(t, 10)
        g = torch.empty(A.lib().rp_surrogate_n_params(), dtype=torch.float32, device="cuda")
        L = C.c_double()
        A.check(A.lib().rp_surrogate_loss_grad(self.handle, x.shape[0], C.c_void_p(x.data_ptr()),
                                               C.c_void_p(y.data_ptr()), C.c_void_p(t.data_ptr()),
                                               C.byref(L), C.c_void_p(g.data_ptr()),
                                               C.c_void_p(_stream_ptr(stream))))
        return L.value, g

    def train_step(self, x, y, t, lr: float, stream=None) -> float:
        L = C.c_double()
        A.check(A.lib().rp_surrogate_train_step(self.handle, x.shape[0], C.c_void_p(x.data_ptr()),
                                                C.c_void_p(y.data_ptr()),
                                                C.c_void_p(t.data_ptr()), C.c_float(lr),
                                                C.byref(L), C.c_void_p(_stream_ptr(stream))))
        return L.value

    def train(self, x, y, t, epochs: int, batch: int, lr: float, lr_final: float = 0.0,
              seed: int = 0, stream=None) -> float:
        """rp_surrogate_train: the whole schedule on the device; returns the last epoch's loss."""
        x, y, t = self._f32(x, 3), self._f32(y, 2), self._f32(t, 10)
        p = A.TrainParams(int(epochs), int(batch), float(lr), float(lr_final), int(seed))
        L = C.c_double()
        A.check(A.lib().rp_surrogate_train(self.handle, x.shape[0], C.c_void_p(x.data_ptr()),
                                           C.c_void_p(y.data_ptr()), C.c_void_p(t.data_ptr()),
                                           C.byref(p), C.byref(L),
                                           C.c_void_p(_stream_ptr(stream))))
        return L.value

    def save(self, path: str):
        A.check(A.lib().rp_surrogate_save(self.handle, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "Surrogate":
        A.lib()
        h = C.c_void_p()
        A.check(A.lib().rp_surrogate_load(os.fsencode(path), C.byref(h)))
        obj = cls.__new__(cls)
        obj.handle = h
        return obj

    def find_paths_into(self, medium: Medium, buf: PathBuffers, prm: A.PathParams,
                        sprm: A.SurrogateParams, stream=None,
                        allow_overflow=False) -> A.SurrogateStats:
        st = A.SurrogateStats()
        rc = A.lib().rp_surrogate_find_paths(
            self.handle, medium.handle, buf.n, C.c_void_p(buf.zs.data_ptr()),
            C.c_void_p(buf.zr.data_ptr()), C.c_void_p(buf.dist.data_ptr()),
            C.c_void_p(buf.n_angles.data_ptr()), C.byref(prm), C.byref(sprm), C.byref(buf.sol),
            C.byref(st), C.c_void_p(_stream_ptr(stream)))
        A.check(rc, allow_overflow=allow_overflow)
        return st

    def find_paths(self, medium: Medium, zs, zr, dist, n_angles, params: dict,
                   precision: str = "fp32", hit_tol: float = 0.005, max_iter: int = 60,
                   max_sol: int = 4, stream=None, **surrogate) -> dict:
        """rp_surrogate_find_paths; keyword arguments as in make_surrogate_params."""
        buf = PathBuffers(zs, zr, dist, n_angles, max_sol)
        prm = make_path_params(params, precision, hit_tol, max_iter, max_sol)
        st = self.find_paths_into(medium, buf, prm, make_surrogate_params(**surrogate), stream)
        out = {"count": buf.count}
        out.update(buf.t)
        out["stats"] = st.as_dict()
        return out


def make_surrogate_params(conf: float = 0.99, refine_tol: float = 0.005,
                          refine_step: float = 1e-3, max_step: float = 0.05,
                          refine_iters: int = 16, deflate: bool = True) -> A.SurrogateParams:
    return A.SurrogateParams(conf, refine_tol, refine_step, max_step, int(refine_iters),
                             int(bool(deflate)))


def encode(zs, zr, dist, sol=None, stream=None):
    """rp_surrogate_encode: network inputs x (n, 3) and, given path-finder solutions
    (a PathBuffers or the dict of find_paths), targets y (n, 2) and t (n, 10)."""
    zs, zr, dist = _dev_f64(zs), _dev_f64(zr), _dev_f64(dist)
    n = zs.numel()
    x = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    y = t = None
    sref, max_sol = None, 0
    if sol is not None:
        if isinstance(sol, PathBuffers):
            sref, max_sol = sol.sol, sol.max_sol
        else:
            fields = [sol["count"]] + [sol[k] for k, _ in SOL_FIELDS]
            sref = A.Solutions(*[f.data_ptr() for f in fields])
            max_sol = sol["launch"].shape[1]
        y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        t = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    A.check(A.lib().rp_surrogate_encode(
        n, C.c_void_p(zs.data_ptr()), C.c_void_p(zr.data_ptr()), C.c_void_p(dist.data_ptr()),
        C.byref(sref) if sref is not None else None, int(max_sol), C.c_void_p(x.data_ptr()),
        C.c_void_p(y.data_ptr() if y is not None else 0),
        C.c_void_p(t.data_ptr() if t is not None else 0), C.c_void_p(_stream_ptr(stream))))
    return x, y, t


def measure_peaks(stream=None) -> dict:
    """rp_measure_peaks: the FP32 and FP64 FMA rates [TFLOP/s] and the L2 read bandwidth [GB/s]
    of the current device, measured by the library's microkernels."""
    pk = A.Peaks()
    A.check(A.lib().rp_measure_peaks(C.byref(pk), C.c_void_p(_stream_ptr(stream))))
    return pk.as_dict()
