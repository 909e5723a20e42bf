"""Tuning of the tracer's scheduling knobs on the caller's own batch.

rp_trace reads two knobs from the environment at every call (include/rp.h): the idle
lane-iterations after which a warp serves its parked lanes (RP_SERVICE_IDLE in FP32-mixed
mode, RP_SERVICE_IDLE_F64 in FP64) and the number of stacked secondaries a thread hands to the
next launch once the launch's input has run out (RP_FLUSH_MIN, the chunk of the hand-over to
the queue).  They decide which thread traces a ray and when, never a ray's arithmetic, so the
fastest pair for a workload can be found by timing the workload itself.  ``tune_trace`` times
the library's own kernel time (``rp_stats.kernel_ms``) for every candidate pair, leaves the
fastest pair set in the environment for the calls that follow, and returns all timings.
"""
from __future__ import annotations

import os

from . import api

IDLE_CANDIDATES = {"fp32": (128, 192, 256, 384), "fp64": (4, 8, 16, 32)}
FLUSH_CANDIDATES = (1, 2, 4, 8)


def knob_names(precision: str) -> tuple[str, str]:
    """Environment names of the (service idle count, flush chunk) knobs for a precision."""
    if precision not in IDLE_CANDIDATES:
        raise ValueError(f"precision must be one of {sorted(IDLE_CANDIDATES)}")
    return ("RP_SERVICE_IDLE" if precision == "fp32" else "RP_SERVICE_IDLE_F64", "RP_FLUSH_MIN")


def tune_trace(medium, rays, params: dict, buf, precision: str = "fp32", idle=None, flush=None,
               reps: int = 2, stream=None) -> dict:
    """Times rp_trace on (medium, rays, params) into buf for every (idle, flush) pair, one
    untimed call and then the best of `reps` timed calls each, and keeps the fastest pair set.

    Returns {"best": {name: value, ...}, "ms": {(idle, flush): kernel ms}}.  On an error the
    environment is put back as it was and the error propagates."""
    names = knob_names(precision)
    idle = tuple(idle or IDLE_CANDIDATES[precision])
    flush = tuple(flush or FLUSH_CANDIDATES)
    if not idle or not flush or reps < 1 or min(idle) < 1 or min(flush) < 1:
        raise ValueError("need at least one idle and one flush value (>= 1) and reps >= 1")
    prm = api.make_params(params, precision)
    saved = {k: os.environ.get(k) for k in names}
    ms = {}
    try:
        for i in idle:
            for f in flush:
                os.environ[names[0]], os.environ[names[1]] = str(i), str(f)
                api.trace_into(medium, rays, prm, buf, stream)
                ms[(i, f)] = min(float(api.trace_into(medium, rays, prm, buf, stream).kernel_ms)
                                 for _ in range(reps))
    except BaseException:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        raise
    best = min(ms, key=ms.get)
    os.environ[names[0]], os.environ[names[1]] = str(best[0]), str(best[1])
    return {"best": {names[0]: best[0], names[1]: best[1]}, "ms": ms}
