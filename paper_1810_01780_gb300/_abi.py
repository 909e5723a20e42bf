"""ctypes mirror of include/rp.h and the loader of the in-tree CUDA library.

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
Loading fails loudly if the library has not been built or cannot be opened; there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libradiopropa_gb300.so")

RP_OK = 0
ERRORS = {-1: "RP_ERR_INVALID_ARG", -2: "RP_ERR_CUDA", -3: "RP_ERR_OOM", -4: "RP_ERR_OVERFLOW",
          -5: "RP_ERR_UNSUPPORTED", -6: "RP_ERR_TIMEOUT"}
RP_ERR_OVERFLOW = -4
MAX_LAYERS = 8
MAX_SPHERES = 4
MEDIUM_KIND = {"layered": 0, "grid": 1}
PRECISION = {"fp64": 0, "fp32": 1}
POLARIZATION = {"s": 0, "p": 1, "unpol": 2}
RHS_FORM = {"projected": 0, "paraxial": 1, "momentum": 2}
STATUS = {
    "ALIVE": 0, "MAX_PATH": 1, "MAX_TIME": 2, "MIN_AMP": 3, "LEFT_DOMAIN": 4, "TRANSMITTED": 5,
    "REACHED_STOP": 6, "MAX_STEPS": 7, "BAD_INPUT": 8, "QUEUE_FULL": 9,
}
SOL_TYPE = {"DIRECT": 0, "REFRACTED": 1, "REFLECTED": 2}

c_dp = C.POINTER(C.c_double)
c_ip = C.POINTER(C.c_int32)
c_lp = C.POINTER(C.c_int64)


class Layer(C.Structure):
    _fields_ = [("z_top", C.c_double), ("n0", C.c_double), ("dn", C.c_double),
                ("z0", C.c_double), ("offset", C.c_double), ("absorb", C.c_int32),
                ("pad", C.c_int32)]


class Sphere(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("radius", C.c_double), ("n0", C.c_double),
                ("dn", C.c_double), ("z0", C.c_double), ("offset", C.c_double),
                ("absorb", C.c_int32), ("pad", C.c_int32)]


class Surface(C.Structure):
    _fields_ = [("layer", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("pad", C.c_int32),
                ("normal", C.c_double * 3), ("origin", C.c_double * 2),
                ("spacing", C.c_double * 2), ("height", C.c_void_p)]


class MediumDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_layers", C.c_int32), ("layers", Layer * MAX_LAYERS),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double),
                ("grid_n", C.c_void_p), ("n_spheres", C.c_int32), ("pad2", C.c_int32),
                ("spheres", Sphere * MAX_SPHERES), ("n_surfaces", C.c_int32),
                ("pad3", C.c_int32), ("surfaces", Surface * MAX_LAYERS)]


class Rays(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("dir", C.c_void_p), ("amp", C.c_void_p)]


class Receivers(C.Structure):
    _fields_ = [("n", C.c_int32), ("pad", C.c_int32), ("center", C.c_void_p),
                ("radius", C.c_void_p)]


class TraceParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double),
                ("h0", C.c_double), ("max_path", C.c_double), ("max_time", C.c_double),
                ("min_amp", C.c_double), ("eps_b", C.c_double), ("stop_n", C.c_double * 3),
                ("stop_d", C.c_double), ("use_stop", C.c_int32), ("max_generation", C.c_int32),
                ("precision", C.c_int32), ("polarization", C.c_int32), ("rhs_form", C.c_int32),
                ("ray_order", C.c_int32), ("max_steps", C.c_int64), ("service_idle", C.c_int32),
                ("flush_min", C.c_int32), ("block", C.c_int32), ("blocks_per_sm", C.c_int32)]


class RayOut(C.Structure):
    _fields_ = [("capacity", C.c_int64)] + [
        (f, C.c_void_p) for f in ("end_pos", "end_dir", "path", "time", "amp", "status",
                                  "generation", "seq", "layer", "parent", "n_acc", "n_rej",
                                  "n_root", "n_refl", "n_turn")]


class Hits(C.Structure):
    _fields_ = [("capacity", C.c_int64)] + [
        (f, C.c_void_p) for f in ("ray", "receiver", "time", "path", "amp", "pos", "dir")]


class Stats(C.Structure):
    _fields_ = [("rays", C.c_int64), ("hits", C.c_int64), ("secondaries", C.c_int64),
                ("steps_accepted", C.c_int64), ("steps_rejected", C.c_int64),
                ("steps_root", C.c_int64), ("queue_needed", C.c_int64), ("waves", C.c_int32),
                ("flags", C.c_int32), ("kernel_ms", C.c_double), ("wave_ms", C.c_double * 16),
                ("warp_end_ms", C.c_double * 3), ("queue_capacity", C.c_int64),
                ("threads", C.c_int32), ("stack_depth", C.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["wave_ms"] = list(self.wave_ms)[: self.waves]
        d["warp_end_ms"] = list(self.warp_end_ms)
        return d


class PathParams(C.Structure):
    _fields_ = [("trace", TraceParams), ("hit_tol", C.c_double), ("max_iter", C.c_int32),
                ("max_sol", C.c_int32)]


class Solutions(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("count", "type", "n_iter", "launch", "receive", "time",
                                          "path", "amp", "miss")]


class TrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float),
                ("lr_final", C.c_float), ("seed", C.c_uint64)]


class SurrogateParams(C.Structure):
    _fields_ = [("conf", C.c_double), ("refine_tol", C.c_double), ("refine_step", C.c_double),
                ("max_step", C.c_double), ("refine_iters", C.c_int32), ("deflate", C.c_int32)]


class SurrogateStats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("queries", "tasks", "tasks_failed", "fail_end",
                                         "fail_iters", "fail_step", "duplicates",
                                         "deflated", "fallback",
                                         "refine_rays", "refine_steps", "fallback_rays",
                                         "fallback_steps")] + \
               [(f, C.c_float) for f in ("ms_forward", "ms_refine", "ms_fallback", "ms_total",
                                         "ms_fallback_scan")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Peaks(C.Structure):
    _fields_ = [(f, C.c_double) for f in ("fp32_tflops", "fp64_tflops", "l2_gbs", "fp32_ms",
                                          "fp64_ms", "l2_ms", "l2_buffer_bytes")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# every entry point the header declares, with its ctypes signature
SIGNATURES = {
    "rp_medium_create": (C.c_int, [C.POINTER(MediumDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "rp_medium_destroy": (C.c_int, [C.c_void_p]),
    "rp_trace": (C.c_int, [C.c_void_p, C.POINTER(Rays), C.POINTER(Receivers),
                           C.POINTER(TraceParams), C.POINTER(RayOut), C.POINTER(Hits),
                           C.POINTER(Stats), C.c_void_p]),
    "rp_trace_static": (C.c_int, [C.c_void_p, C.POINTER(Rays), C.POINTER(Receivers),
                                  C.POINTER(TraceParams), C.POINTER(RayOut), C.POINTER(Hits),
                                  C.POINTER(Stats), C.c_void_p]),
    "rp_find_paths": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.POINTER(PathParams), C.POINTER(Solutions),
                                C.POINTER(Stats), C.c_void_p]),
    "rp_surrogate_n_params": (C.c_int, []),
    "rp_surrogate_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "rp_surrogate_destroy": (C.c_int, [C.c_void_p]),
    "rp_surrogate_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rp_surrogate_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rp_surrogate_forward": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rp_surrogate_loss_grad": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    "rp_surrogate_train_step": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_float, C.POINTER(C.c_double),
                                          C.c_void_p]),
    "rp_surrogate_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "rp_surrogate_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    "rp_surrogate_train": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(TrainParams), C.POINTER(C.c_double), C.c_void_p]),
    "rp_surrogate_encode": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(Solutions), C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "rp_surrogate_find_paths": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.POINTER(PathParams), C.POINTER(SurrogateParams),
                                          C.POINTER(Solutions), C.POINTER(SurrogateStats),
                                          C.c_void_p]),
    "rp_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "rp_version": (C.c_char_p, []),
    "rp_measure_peaks": (C.c_int, [C.POINTER(Peaks), C.c_void_p]),
    "rp_surrogate_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
}

_lib = None
_lock = threading.Lock()


class RPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded CUDA library (raises if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is not built; run paper_1810_01780_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().rp_last_error(buf, len(buf))
    return buf.value.decode()


def check(code: int, allow_overflow: bool = False) -> int:
    if code == RP_OK or (allow_overflow and code == RP_ERR_OVERFLOW):
        return code
    raise RPError(code, last_error())
