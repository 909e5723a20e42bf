"""The scheduling-knob tuner: on CPU with the library call replaced by a fake whose kernel time
depends on the knobs it finds in the environment; on the GPU on a batch of the batched
workload."""
import os

import numpy as np
import pytest

from paper_1810_01780_gb300 import autotune, workloads as W


class _Stats:
    def __init__(self, ms):
        self.kernel_ms = ms


def test_tuner_picks_the_fastest_pair_and_keeps_it(monkeypatch):
    from paper_1810_01780_gb300 import api

    seen = []

    def fake(medium, rays, prm, buf, stream=None):
        i, f = int(os.environ["RP_SERVICE_IDLE"]), int(os.environ["RP_FLUSH_MIN"])
        seen.append((i, f))
        return _Stats(abs(i - 192) / 64.0 + abs(f - 4) + 1.0)

    monkeypatch.setattr(api, "trace_into", fake)
    monkeypatch.setenv("RP_SERVICE_IDLE", "7")
    monkeypatch.delenv("RP_FLUSH_MIN", raising=False)
    r = autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp32", reps=3)
    assert r["best"] == {"RP_SERVICE_IDLE": 192, "RP_FLUSH_MIN": 4}
    assert os.environ["RP_SERVICE_IDLE"] == "192" and os.environ["RP_FLUSH_MIN"] == "4"
    assert len(r["ms"]) == 16 and r["ms"][(192, 4)] == 1.0
    assert len(seen) == 16 * 4  # one untimed and three timed calls per pair
    # FP64 tunes its own idle knob
    monkeypatch.setattr(api, "trace_into", lambda *a, **k: _Stats(
        float(os.environ["RP_SERVICE_IDLE_F64"])))
    r = autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp64", flush=(2,), reps=1)
    assert r["best"] == {"RP_SERVICE_IDLE_F64": 4, "RP_FLUSH_MIN": 2}


def test_tuner_restores_the_environment_on_error(monkeypatch):
    from paper_1810_01780_gb300 import api

    def boom(*a, **k):
        raise RuntimeError("device error")

    monkeypatch.setattr(api, "trace_into", boom)
    monkeypatch.setenv("RP_SERVICE_IDLE", "300")
    monkeypatch.delenv("RP_FLUSH_MIN", raising=False)
    with pytest.raises(RuntimeError):
        autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp32")
    assert os.environ["RP_SERVICE_IDLE"] == "300" and "RP_FLUSH_MIN" not in os.environ
    with pytest.raises(ValueError):
        autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp16")
    with pytest.raises(ValueError):
        autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp32", flush=(0,))


@pytest.mark.gpu
def test_tuner_on_the_gpu(monkeypatch):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp

    for k in ("RP_SERVICE_IDLE", "RP_FLUSH_MIN"):
        monkeypatch.setenv(k, "1")  # monkeypatch puts the caller's values back afterwards
    cfg = W.batched(n=20_000)
    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"], receivers=cfg["receivers"])
    buf = rp.TraceBuffers(int(5.5 * rays.n), 4096)
    r = autotune.tune_trace(med, rays, cfg["params"], buf, "fp32", idle=(64, 256),
                            flush=(1, 2), reps=1)
    assert set(r["ms"]) == {(64, 1), (64, 2), (256, 1), (256, 2)}
    assert all(np.isfinite(v) and v > 0 for v in r["ms"].values())
    best = min(r["ms"], key=r["ms"].get)
    assert os.environ["RP_SERVICE_IDLE"] == str(best[0])
    assert os.environ["RP_FLUSH_MIN"] == str(best[1])
