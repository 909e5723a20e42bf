"""The binding's parameter marshalling (argument marshalling only, no CUDA): every key of the
parameter dicts lands in the field of the same meaning, with the stated defaults."""
import pytest

from paper_1810_01780_gb300 import _abi as A, api, workloads as W


def test_trace_params_fields_and_defaults():
    p = dict(tol=2e-6, h_min=3e-3, h_max=7.0, h0=0.5, max_path=1234.0, max_time=4e-6,
             min_amp=0.05, eps_b=2e-9, stop=((1.0, 0.0, 0.0), 55.0), max_generation=5,
             polarization="unpol", rhs_form="momentum", max_steps=777)
    q = api.make_params(p, "fp64")
    for k in ("tol", "h_min", "h_max", "h0", "max_path", "max_time", "min_amp", "eps_b",
              "max_generation", "max_steps"):
        assert getattr(q, k) == p[k], k
    assert list(q.stop_n) == [1.0, 0.0, 0.0] and q.stop_d == 55.0 and q.use_stop == 1
    assert q.precision == A.PRECISION["fp64"] and q.polarization == A.POLARIZATION["unpol"]
    assert q.rhs_form == A.RHS_FORM["momentum"]
    d = api.make_params(dict(tol=1e-6, h_min=1e-3, h_max=10.0), "fp32")
    assert d.h0 == 10.0 and d.eps_b == 1e-9 and d.max_generation == 3 and d.use_stop == 0
    assert d.max_time == 0.0 and d.min_amp == 0.0 and d.max_steps == 1_000_000
    assert d.precision == A.PRECISION["fp32"] and d.polarization == A.POLARIZATION["s"]
    assert d.rhs_form == A.RHS_FORM["projected"]
    # scheduling knobs: 0 (the library's defaults) unless given
    assert (d.service_idle, d.flush_min, d.block, d.blocks_per_sm) == (0, 0, 0, 0)
    k = api.make_params(dict(W.TRACE_DEFAULTS, service_idle=9, flush_min=3, block=64,
                             blocks_per_sm=2), "fp32")
    assert (k.service_idle, k.flush_min, k.block, k.blocks_per_sm) == (9, 3, 64, 2)
    with pytest.raises(KeyError):
        api.make_params(W.TRACE_DEFAULTS, "fp16")


def test_path_and_surrogate_params():
    q = api.make_path_params(W.paths(4)["params"], "fp32", hit_tol=0.005, max_iter=80, max_sol=3)
    assert q.hit_tol == 0.005 and q.max_iter == 80 and q.max_sol == 3
    assert q.trace.max_path == 10000.0 and q.trace.max_generation == 0
    assert q.trace.precision == A.PRECISION["fp32"]
    # the path finder sets each ray's path budget itself; a placeholder keeps the struct valid
    assert api.make_path_params(dict(tol=1e-6, h_min=1e-3, h_max=10.0)).trace.max_path == 1.0
    s = api.make_surrogate_params(conf=0.9, refine_tol=0.01, refine_step=2e-3, max_step=0.1,
                                  refine_iters=12, deflate=False)
    assert (s.conf, s.refine_tol, s.refine_step, s.max_step, s.refine_iters, s.deflate) == \
        (0.9, 0.01, 2e-3, 0.1, 12, 0)
