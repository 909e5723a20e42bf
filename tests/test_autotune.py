"""The scheduling-knob tuner: on CPU with the library call replaced by a fake whose kernel time
depends on the knobs it finds in the parameters it is given; on the GPU on a batch of the
batched workload, where the tuned knobs must leave every record unchanged."""
import numpy as np
import pytest

from paper_1810_01780_gb300 import autotune, workloads as W


class _Stats:
    def __init__(self, ms):
        self.kernel_ms = ms


def test_tuner_picks_the_fastest_knobs_and_returns_them(monkeypatch):
    from paper_1810_01780_gb300 import api

    seen = []

    def fake(medium, rays, prm, buf, stream=None):
        i, f, b = prm.service_idle, prm.flush_min, prm.block
        seen.append((i, f, b, prm.blocks_per_sm))
        return _Stats(abs(i - 192) / 64.0 + abs(f - 4) + abs(b - 64) / 64.0 + 1.0)

    monkeypatch.setattr(api, "trace_into", fake)
    prm = dict(W.TRACE_DEFAULTS, max_path=100.0)
    r = autotune.tune_trace(None, None, prm, None, "fp32", reps=3)
    assert r["best"] == {"service_idle": 192, "flush_min": 4, "block": 64, "blocks_per_sm": 0}
    assert len(r["ms"]) == 16 * 3 and r["ms"][(192, 4, 64, 0)] == 1.0
    assert len(seen) == 16 * 3 * 4  # one untimed and three timed calls per combination
    assert r["params"] == dict(prm, service_idle=192, flush_min=4, block=64, blocks_per_sm=0)
    assert "service_idle" not in prm  # the caller's dict is left as it was
    # FP64 tunes over its own idle candidates; explicit candidate lists are honoured
    monkeypatch.setattr(api, "trace_into", lambda m, r_, p, b, s=None: _Stats(
        float(p.service_idle) + p.block / 1000.0 + p.blocks_per_sm))
    r = autotune.tune_trace(None, None, prm, None, "fp64", flush=(2,), block=(128, 256),
                            blocks_per_sm=(0, 1), reps=1)
    assert r["best"] == {"service_idle": 4, "flush_min": 2, "block": 128, "blocks_per_sm": 0}
    assert len(r["ms"]) == 4 * 1 * 2 * 2


def test_tuner_rejects_bad_candidates_and_propagates_errors(monkeypatch):
    from paper_1810_01780_gb300 import api

    def boom(*a, **k):
        raise RuntimeError("device error")

    monkeypatch.setattr(api, "trace_into", boom)
    with pytest.raises(RuntimeError):
        autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, "fp32")
    for bad in (dict(precision="fp16"), dict(flush=(0,)), dict(block=(96, 300)),
                dict(block=(100,)), dict(blocks_per_sm=(-1,)), dict(reps=0)):
        kw = dict(precision="fp32")
        kw.update(bad)
        with pytest.raises(ValueError):
            autotune.tune_trace(None, None, W.TRACE_DEFAULTS, None, **kw)


@pytest.mark.gpu
def test_tuner_on_the_gpu():
    """Tunes all four knobs on 20,000 primaries of the batched workload; the tuned parameters
    reproduce the default run's records bit for bit (matched by split tree)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp
    from parity import gpu_rays, match

    cfg = W.batched(n=20_000)
    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"], receivers=cfg["receivers"])
    buf = rp.TraceBuffers(int(5.5 * rays.n), 4096)
    r = autotune.tune_trace(med, rays, cfg["params"], buf, "fp32", idle=(64, 256),
                            flush=(1, 2), block=(64, 128, 256), blocks_per_sm=(0, 2), reps=1)
    assert len(r["ms"]) == 2 * 2 * 3 * 2
    assert all(np.isfinite(v) and v > 0 for v in r["ms"].values())
    best = min(r["ms"], key=r["ms"].get)
    assert tuple(r["best"].values()) == best
    base = gpu_rays(rp.trace(med, *cfg["rays"], params=cfg["params"],
                             receivers=cfg["receivers"], precision="fp32"))
    tuned = gpu_rays(rp.trace(med, *cfg["rays"], params=r["params"],
                              receivers=cfg["receivers"], precision="fp32"))
    gi, bi, only_g, only_b = match(tuned, base)
    assert not only_g and not only_b
    for k in ("pos", "dir", "path", "time", "amp", "status", "n_acc", "n_rej"):
        np.testing.assert_array_equal(tuned[k][gi], base[k][bi], err_msg=k)
