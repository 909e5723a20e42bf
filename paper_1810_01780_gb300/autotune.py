"""Tuning of the tracer's scheduling knobs on the caller's own batch.

rp_trace takes four scheduling knobs in its parameters (include/rp.h, rp_trace_params): the
idle lane-iterations after which a warp serves its parked lanes (``service_idle``), the number
of stacked secondaries a thread hands to the next launch once the launch's input has run out
(``flush_min``), the threads per block of the persistent launches (``block``) and the resident
blocks per SM (``blocks_per_sm``).  They decide which thread traces a ray and when, never a
ray's arithmetic, so the fastest setting for a workload can be found by timing the workload
itself.  ``tune_trace`` times the library's own kernel time (``rp_stats.kernel_ms``) for every
candidate on a grid of the knobs and returns the fastest one as parameter keys to merge into
the caller's parameters; nothing global is changed.
"""
from __future__ import annotations

import itertools

from . import api

IDLE_CANDIDATES = {"fp32": (128, 192, 256, 384), "fp64": (4, 8, 16, 32)}
FLUSH_CANDIDATES = (1, 2, 4, 8)
BLOCK_CANDIDATES = (64, 128, 256)
BLOCKS_PER_SM_CANDIDATES = (0,)  # 0: as many as fit


def tune_trace(medium, rays, params: dict, buf, precision: str = "fp32", idle=None, flush=None,
               block=None, blocks_per_sm=None, reps: int = 2, stream=None) -> dict:
    """Times rp_trace on (medium, rays, params) into buf for every combination of the candidate
    knob values (one untimed call, then the best of `reps` timed calls each).

    Returns {"best": {"service_idle": ..., "flush_min": ..., "block": ...,
    "blocks_per_sm": ...}, "ms": {(idle, flush, block, blocks_per_sm): kernel ms},
    "params": params with the best knobs merged in}."""
    if precision not in IDLE_CANDIDATES:
        raise ValueError(f"precision must be one of {sorted(IDLE_CANDIDATES)}")
    idle = tuple(idle or IDLE_CANDIDATES[precision])
    flush = tuple(flush or FLUSH_CANDIDATES)
    block = tuple(block or BLOCK_CANDIDATES)
    per_sm = tuple(blocks_per_sm if blocks_per_sm is not None else BLOCKS_PER_SM_CANDIDATES)
    if not idle or not flush or not block or not per_sm or reps < 1 or min(idle) < 1 or \
            min(flush) < 1 or min(per_sm) < 0 or any(b < 32 or b > 256 or b % 32 for b in block):
        raise ValueError("need idle and flush values >= 1, blocks of 32..256 threads in steps "
                         "of 32, blocks_per_sm >= 0 and reps >= 1")
    ms = {}
    for i, f, b, o in itertools.product(idle, flush, block, per_sm):
        prm = api.make_params(dict(params, service_idle=i, flush_min=f, block=b,
                                   blocks_per_sm=o), precision)
        api.trace_into(medium, rays, prm, buf, stream)
        ms[(i, f, b, o)] = min(float(api.trace_into(medium, rays, prm, buf, stream).kernel_ms)
                               for _ in range(reps))
    best = min(ms, key=ms.get)
    knobs = dict(zip(api.SCHEDULING_KNOBS, best))
    return {"best": knobs, "ms": ms, "params": dict(params, **knobs)}
