"""GB300-native RadioPropa ray-propagation hot path.

Adaptive Cash-Karp integration of the ray equation in refractivity fields, the boundary
module (reflection, Snell refraction, Fresnel amplitudes, secondary rays), receivers and
source-receiver path finding (RadioPropa, ARENA 2018, Sec. 2), as hand-written CUDA for
sm_103a behind the C ABI of include/rp.h.  This package is the thin Python binding:

    from paper_1810_01780_gb300 import Medium, trace, find_paths, workloads

Importing the package does not load CUDA; the first call does, and fails loudly if the
library is not built (``paper_1810_01780_gb300.build.build()``).
"""
from . import workloads  # noqa: F401  (inputs only)

__all__ = ["Medium", "trace", "trace_into", "TraceBuffers", "PreparedRays", "make_params",
           "find_paths", "workloads"]


def __getattr__(name):
    if name in ("Medium", "trace", "trace_into", "TraceBuffers", "PreparedRays", "make_params",
                "find_paths", "PathBuffers", "find_paths_into", "make_path_params", "Surrogate",
                "make_surrogate_params", "encode", "measure_peaks"):
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
