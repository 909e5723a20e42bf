"""Plain FP64 CPU oracle of the RadioPropa ray-propagation method (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library; both sides meet only through the
seeded inputs of ``paper_1810_01780_gb300.workloads``.

The tracer itself is ``rp_oracle.c`` (built with ``-O2 -ffp-contract=off``, no fast-math);
this module compiles it on first use and marshals numpy arrays through ctypes.  The closed
forms for the exponential profile live in ``oracle.analytic`` and the FP64 MLP in
``oracle.mlp``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librp_oracle.so")
SRC = [os.path.join(HERE, "rp_oracle.c")]
HDR = os.path.join(HERE, "rp_oracle.h")

MAX_LAYERS = 8
MAX_SPHERES = 4
RHS = {"projected": 0, "paraxial": 1, "momentum": 2}
POL = {"s": 0, "p": 1, "unpol": 2}
STATUS = {
    "ALIVE": 0, "MAX_PATH": 1, "MAX_TIME": 2, "MIN_AMP": 3, "LEFT_DOMAIN": 4,
    "TRANSMITTED": 5, "REACHED_STOP": 6, "MAX_STEPS": 7,
}
SOL_TYPE = {"DIRECT": 0, "REFRACTED": 1, "REFLECTED": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, strict IEEE double)."""
    newest = max(os.path.getmtime(p) for p in SRC + [HDR])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-Wall", "-fPIC",
           "-shared", "-o", tmp] + SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Medium(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n_layers", C.c_int32),
        ("z_top", C.c_double * MAX_LAYERS), ("n0", C.c_double * MAX_LAYERS),
        ("dn", C.c_double * MAX_LAYERS), ("z0", C.c_double * MAX_LAYERS),
        ("off", C.c_double * MAX_LAYERS), ("absorb", C.c_int32 * MAX_LAYERS),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad", C.c_int32),
        ("origin", C.c_double * 3), ("spacing", C.c_double),
        ("grid4", C.POINTER(C.c_float)),
        ("n_spheres", C.c_int32), ("pad2", C.c_int32),
        ("sph_c", (C.c_double * 3) * MAX_SPHERES), ("sph_R", C.c_double * MAX_SPHERES),
        ("sph_n0", C.c_double * MAX_SPHERES), ("sph_dn", C.c_double * MAX_SPHERES),
        ("sph_z0", C.c_double * MAX_SPHERES), ("sph_off", C.c_double * MAX_SPHERES),
        ("sph_absorb", C.c_int32 * MAX_SPHERES),
        ("srf_on", C.c_int32 * MAX_LAYERS), ("srf_sx", C.c_double * MAX_LAYERS),
        ("srf_sy", C.c_double * MAX_LAYERS), ("hf_nx", C.c_int32 * MAX_LAYERS),
        ("hf_ny", C.c_int32 * MAX_LAYERS), ("hf_ox", C.c_double * MAX_LAYERS),
        ("hf_oy", C.c_double * MAX_LAYERS), ("hf_dx", C.c_double * MAX_LAYERS),
        ("hf_dy", C.c_double * MAX_LAYERS), ("hf", C.POINTER(C.c_double) * MAX_LAYERS),
    ]


class Params(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double), ("h0", C.c_double),
        ("max_path", C.c_double), ("max_time", C.c_double), ("min_amp", C.c_double),
        ("eps_b", C.c_double), ("stop_n", C.c_double * 3), ("stop_d", C.c_double),
        ("use_stop", C.c_int32), ("max_generation", C.c_int32), ("polarization", C.c_int32),
        ("rhs_form", C.c_int32), ("max_steps", C.c_int64),
    ]


RAY_DTYPE = np.dtype([
    ("parent", "<i8"), ("root", "<i8"), ("seq", "<i4"), ("gen", "<i4"), ("status", "<i4"),
    ("layer", "<i4"), ("pos", "<f8", (3,)), ("dir", "<f8", (3,)), ("path", "<f8"),
    ("time", "<f8"), ("amp", "<f8"), ("amp0", "<f8"), ("n_acc", "<i8"), ("n_rej", "<i8"),
    ("n_root", "<i8"), ("n_refl", "<i4"), ("n_turn", "<i4"), ("root_fail", "<i4"),
    ("pad", "<i4"),
])
HIT_DTYPE = np.dtype([
    ("ray", "<i8"), ("receiver", "<i4"), ("pad", "<i4"), ("time", "<f8"), ("path", "<f8"),
    ("amp", "<f8"), ("pos", "<f8", (3,)), ("dir", "<f8", (3,)),
])
SOL_DTYPE = np.dtype([
    ("type", "<i4"), ("n_iter", "<i4"), ("converged", "<i4"), ("pad", "<i4"),
    ("launch", "<f8"), ("receive", "<f8"), ("time", "<f8"), ("path", "<f8"), ("amp", "<f8"),
    ("miss", "<f8"),
])

_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
            L.or_trace.restype = C.c_int64
            L.or_trace.argtypes = [C.POINTER(Medium), C.POINTER(Params), C.c_int64, dp, dp, dp,
                                   C.c_int32, dp, dp, C.c_void_p, C.c_int64, C.c_void_p,
                                   C.c_int64, C.POINTER(C.c_int64)]
            L.or_find_paths.restype = C.c_int32
            L.or_find_paths.argtypes = [C.POINTER(Medium), C.POINTER(Params), C.c_int64, dp, dp,
                                        dp, ip, C.c_double, C.c_int32, C.c_int32, ip,
                                        C.c_void_p]
            L.or_ck_poly_step.argtypes = [dp, C.c_int32, C.c_double, C.c_double, C.c_double,
                                          dp, dp]
            L.or_medium_eval.argtypes = [C.POINTER(Medium), C.c_int32, dp, dp, dp]
            L.or_layer_of.restype = C.c_int32
            L.or_layer_of.argtypes = [C.POINTER(Medium), C.c_double]
            L.or_layer_at.restype = C.c_int32
            L.or_layer_at.argtypes = [C.POINTER(Medium), dp]
            L.or_boundary_depth.restype = C.c_double
            L.or_boundary_depth.argtypes = [C.POINTER(Medium), C.c_int32, C.c_double,
                                            C.c_double, dp, dp]
            L.or_grid_prepare.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32,
                                          C.c_double, C.POINTER(C.c_float)]
            L.or_rhs.argtypes = [C.POINTER(Medium), C.c_int32, C.c_int32, dp, dp]
            L.or_ck_step.restype = C.c_double
            L.or_ck_step.argtypes = [C.POINTER(Medium), C.c_int32, C.c_int32, dp, C.c_double, dp]
            L.or_split_dirs.argtypes = [dp, dp, C.c_double, C.c_double, C.c_int32, dp, dp, dp,
                                        dp, ip]
            L.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                     dp, dp]
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleMedium:
    """Owns the ctypes medium struct plus the arrays it points at."""

    def __init__(self, desc: dict):
        self.desc = desc
        m = Medium()
        if desc["kind"] == "layered":
            layers = desc["layers"]
            if not 1 <= len(layers) <= MAX_LAYERS:
                raise ValueError("1..8 layers")
            m.kind = 0
            m.n_layers = len(layers)
            for k, L in enumerate(layers):
                m.z_top[k] = float(L.get("z_top", -np.inf)) if k else -np.inf
                m.n0[k] = float(L["n0"])
                m.dn[k] = float(L.get("dn", 0.0))
                m.z0[k] = float(L.get("z0", 1.0))
                m.off[k] = float(L.get("off", 0.0))
                m.absorb[k] = int(bool(L.get("absorb", False)))
            spheres = desc.get("spheres", [])
            if len(spheres) > MAX_SPHERES:
                raise ValueError("at most %d spheres" % MAX_SPHERES)
            m.n_spheres = len(spheres)
            for j, S in enumerate(spheres):
                for a in range(3):
                    m.sph_c[j][a] = float(S["center"][a])
                m.sph_R[j] = float(S["radius"])
                m.sph_n0[j] = float(S["n0"])
                m.sph_dn[j] = float(S.get("dn", 0.0))
                m.sph_z0[j] = float(S.get("z0", 1.0))
                m.sph_off[j] = float(S.get("off", 0.0))
                m.sph_absorb[j] = int(bool(S.get("absorb", False)))
            # non-horizontal boundaries: a tilted plane of unit normal N (N_z > 0) through
            # (0, 0, z_top), slopes -N_x / N_z and -N_y / N_z, plus an optional height field
            self.heights = []
            for srf in desc.get("surfaces", []):
                k = int(srf["layer"])
                if not 1 <= k < len(layers):
                    raise ValueError("a surface replaces the boundary of layer 1..n_layers-1")
                N = np.asarray(srf.get("normal", (0.0, 0.0, 1.0)), dtype=np.float64)
                if not N[2] > 0.0:
                    raise ValueError("surface normal needs a positive z component")
                m.srf_on[k] = 1
                m.srf_sx[k] = -N[0] / N[2]
                m.srf_sy[k] = -N[1] / N[2]
                if srf.get("height") is not None:
                    h = np.ascontiguousarray(srf["height"], dtype=np.float64)  # (ny, nx)
                    m.hf_ny[k], m.hf_nx[k] = h.shape
                    m.hf_ox[k], m.hf_oy[k] = (float(v) for v in srf["origin"])
                    m.hf_dx[k], m.hf_dy[k] = (float(v) for v in srf["spacing"])
                    m.hf[k] = _dptr(h)
                    self.heights.append(h)
            self.grid4 = None
        elif desc["kind"] == "grid":
            n = np.ascontiguousarray(desc["n"], dtype=np.float32)  # (nz, ny, nx)
            nz, ny, nx = n.shape
            g4 = np.empty((nz, ny, nx, 4), dtype=np.float32)
            lib().or_grid_prepare(n.ctypes.data_as(C.POINTER(C.c_float)), nx, ny, nz,
                                  float(desc["spacing"]), g4.ctypes.data_as(C.POINTER(C.c_float)))
            self.grid4 = g4
            m.kind = 1
            m.n_layers = 1
            m.nx, m.ny, m.nz = nx, ny, nz
            for a in range(3):
                m.origin[a] = float(desc["origin"][a])
            m.spacing = float(desc["spacing"])
            m.grid4 = g4.ctypes.data_as(C.POINTER(C.c_float))
        else:
            raise ValueError(desc["kind"])
        self.c = m

    def eval(self, r, layer=0):
        r = np.ascontiguousarray(r, dtype=np.float64)
        n = np.zeros(1)
        g = np.zeros(3)
        lib().or_medium_eval(C.byref(self.c), layer, _dptr(r), _dptr(n), _dptr(g))
        return n[0], g

    def layer_of(self, z):
        return lib().or_layer_of(C.byref(self.c), float(z))

    def layer_at(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        return lib().or_layer_at(C.byref(self.c), _dptr(r))

    def boundary_depth(self, k, x, y):
        """(depth, dz/dx, dz/dy) of boundary k at (x, y)."""
        gx, gy = C.c_double(), C.c_double()
        z = lib().or_boundary_depth(C.byref(self.c), int(k), float(x), float(y), C.byref(gx),
                                    C.byref(gy))
        return z, gx.value, gy.value


def make_params(p: dict) -> Params:
    q = Params()
    q.tol = p["tol"]
    q.h_min = p["h_min"]
    q.h_max = p["h_max"]
    q.h0 = p.get("h0", p["h_max"])
    q.max_path = p["max_path"]
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
    q.polarization = POL[p.get("polarization", "s")]
    q.rhs_form = RHS[p.get("rhs_form", "projected")]
    q.max_steps = int(p.get("max_steps", 1_000_000))
    return q


def trace(medium, params: dict, pos, dir, amp=None, receivers=None, out_cap=None,
          hit_cap=None):
    """Trace primaries (pos, dir: (3, n) SoA) and all their secondaries.

    Returns (rays, hits): numpy structured arrays (RAY_DTYPE, HIT_DTYPE).  Primaries occupy
    rays[0:n]; secondaries follow in creation order."""
    med = medium if isinstance(medium, OracleMedium) else OracleMedium(medium)
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(3, -1)
    dir = np.ascontiguousarray(dir, dtype=np.float64).reshape(3, -1)
    n = pos.shape[1]
    amp = np.ones(n) if amp is None else np.ascontiguousarray(amp, dtype=np.float64)
    if receivers is None:
        rc = np.zeros((0, 3))
        rr = np.zeros(0)
    else:
        rc = np.ascontiguousarray(receivers[0], dtype=np.float64).reshape(-1, 3)
        rr = np.ascontiguousarray(receivers[1], dtype=np.float64).reshape(-1)
    prm = make_params(params)
    out_cap = out_cap or max(16, 4 * n)
    hit_cap = hit_cap or max(16, 2 * n)
    while True:
        rays = np.zeros(out_cap, dtype=RAY_DTYPE)
        hits = np.zeros(hit_cap, dtype=HIT_DTYPE)
        nh = C.c_int64(0)
        nr = lib().or_trace(C.byref(med.c), C.byref(prm), n, _dptr(pos), _dptr(dir), _dptr(amp),
                            len(rr), _dptr(rc), _dptr(rr), rays.ctypes.data, out_cap,
                            hits.ctypes.data, hit_cap, C.byref(nh))
        if nr <= out_cap and nh.value <= hit_cap:
            return rays[:nr], hits[: nh.value]
        out_cap = max(out_cap, int(nr))
        hit_cap = max(hit_cap, int(nh.value))


def find_paths(medium, params: dict, zs, zr, dist, n_angles, hit_tol=0.1, max_iter=60,
               max_sol=4):
    """Batched source-receiver path finding; returns (count[n_pairs], sol[n_pairs, max_sol])."""
    med = medium if isinstance(medium, OracleMedium) else OracleMedium(medium)
    zs = np.ascontiguousarray(zs, dtype=np.float64)
    zr = np.ascontiguousarray(zr, dtype=np.float64)
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    na = np.ascontiguousarray(n_angles, dtype=np.int32)
    n = len(zs)
    count = np.zeros(n, dtype=np.int32)
    sol = np.zeros((n, max_sol), dtype=SOL_DTYPE)
    prm = make_params(params)
    lib().or_find_paths(C.byref(med.c), C.byref(prm), n, _dptr(zs), _dptr(zr), _dptr(dist),
                        na.ctypes.data_as(C.POINTER(C.c_int32)), hit_tol, max_iter, max_sol,
                        count.ctypes.data_as(C.POINTER(C.c_int32)), sol.ctypes.data)
    return count, sol


def ck_poly_step(coef, x0, y0, h):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    y5 = np.zeros(1)
    y4 = np.zeros(1)
    lib().or_ck_poly_step(_dptr(coef), len(coef), x0, y0, h, _dptr(y5), _dptr(y4))
    return y5[0], y4[0]


def ck_tableau():
    L = lib()
    c = np.ctypeslib.as_array((C.c_double * 6).in_dll(L, "or_ck_c")).copy()
    a = np.ctypeslib.as_array(((C.c_double * 5) * 6).in_dll(L, "or_ck_a")).copy()
    b5 = np.ctypeslib.as_array((C.c_double * 6).in_dll(L, "or_ck_b5")).copy()
    b4 = np.ctypeslib.as_array((C.c_double * 6).in_dll(L, "or_ck_b4")).copy()
    return c, a, b5, b4


def ck_step(medium, y0, h, layer=0, rhs_form="projected"):
    med = medium if isinstance(medium, OracleMedium) else OracleMedium(medium)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    y5 = np.zeros(7)
    e = lib().or_ck_step(C.byref(med.c), layer, RHS[rhs_form], _dptr(y0), h, _dptr(y5))
    return y5, e


def rhs(medium, y, layer=0, rhs_form="projected"):
    med = medium if isinstance(medium, OracleMedium) else OracleMedium(medium)
    y = np.ascontiguousarray(y, dtype=np.float64)
    k = np.zeros(7)
    lib().or_rhs(C.byref(med.c), layer, RHS[rhs_form], _dptr(y), _dptr(k))
    return k


def split(t, nrm, n1, n2, pol="s"):
    t = np.ascontiguousarray(t, dtype=np.float64)
    nrm = np.ascontiguousarray(nrm, dtype=np.float64)
    tr = np.zeros(3)
    tt = np.zeros(3)
    r = np.zeros(1)
    tau = np.zeros(1)
    tir = np.zeros(1, dtype=np.int32)
    lib().or_split_dirs(_dptr(t), _dptr(nrm), n1, n2, POL[pol], _dptr(tr), _dptr(tt), _dptr(r),
                        _dptr(tau), tir.ctypes.data_as(C.POINTER(C.c_int32)))
    return tr, tt, r[0], tau[0], bool(tir[0])


def fresnel(n1, n2, cos_i, cos_t, pol="s"):
    r = np.zeros(1)
    tau = np.zeros(1)
    lib().or_fresnel(n1, n2, cos_i, cos_t, POL[pol], _dptr(r), _dptr(tau))
    return r[0], tau[0]
