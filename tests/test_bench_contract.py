"""The JSON line of bench.py on CPU: the reference arm runs for real on a tiny sample; the
GPU arm runs its host logic with the CUDA calls, the library and the clock sampler replaced
by fakes (a first clock record with a hardware slowdown, so that the re-measure path runs)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e"}

_FAKE_GPU_ARM = r'''
import argparse, contextlib, os, sys, types
import numpy as np
import torch
import torch.distributed as dist

torch.cuda.set_device = lambda *a, **k: None
torch.cuda.synchronize = lambda *a, **k: None


class Stream:
    def __init__(self, *a, **k):
        pass

    def wait_event(self, event):
        pass


torch.cuda.Stream = Stream
torch.cuda.current_stream = lambda *a, **k: Stream()
torch.cuda.stream = lambda s: contextlib.nullcontext()


class Event:
    def __init__(self, **k):
        pass

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 10.0


torch.cuda.Event = Event
_empty, _tensor = torch.empty, torch.tensor


def _host(fn):
    def f(*a, **k):
        k.pop("device", None)
        return fn(*a, **k)
    return f


torch.empty, torch.tensor = _host(_empty), _host(_tensor)
torch.Tensor.pin_memory = lambda self: self

import bench

_init = dist.init_process_group
dist.init_process_group = lambda backend, **k: _init("gloo", **k)
THROTTLED_RANK = int(os.environ.get("THROTTLED_RANK", "0"))


class Sampler:
    calls = 0

    def __init__(self, index):
        pass

    def __enter__(self):
        Sampler.calls += 1
        return self

    def __exit__(self, *exc):
        pass

    def summary(self):
        # sampled regions: the peak microkernels, then the timed region (throttled once)
        first = Sampler.calls == 2 and int(os.environ.get("RANK", "0")) == THROTTLED_RANK
        r = ["hw_slowdown"] if first else ["sw_power_cap"]
        return {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": r, "samples": 5}


bench.ClockSampler = Sampler


class Stats:
    def __init__(self, n):
        self.steps_accepted, self.steps_rejected, self.steps_root = 300 * n, 30 * n, 5 * n
        self.rays, self.kernel_ms = 2 * n, 9.0


class Rays:
    def __init__(self, pos, d, a=None, receivers=None):
        self.n = pos.shape[1]
        self.pos, self.dir, self.amp = (torch.as_tensor(np.ascontiguousarray(x)).clone()
                                        for x in (pos, d, a))


class Buffers:
    def __init__(self, cap, hits=0, fields=None):
        self.t = {k: _empty((3, cap) if k == "end_pos" else (cap,),
                            dtype=torch.int32 if k == "status" else torch.float64).zero_()
                  for k in ("end_pos", "path", "time", "amp", "status")}


import paper_1810_01780_gb300 as pkg
import paper_1810_01780_gb300.build as B

B.build = lambda *a, **k: None
pkg.Medium = lambda desc: object()
pkg.PreparedRays = Rays
pkg.make_params = lambda p, prec: (p, prec)
pkg.TraceBuffers = Buffers
pkg.trace_into = lambda med, rays, prm, buf, stream=None: Stats(rays.n)
import paper_1810_01780_gb300.api as api

api.trace_into = pkg.trace_into  # the tuner's calls
pkg.measure_peaks = lambda stream=None: {"fp32_tflops": 70.0, "fp64_tflops": 1.2, "l2_gbs": 2e4,
                                         "fp32_ms": 9.0, "fp64_ms": 9.0, "l2_ms": 9.0,
                                         "l2_buffer_bytes": 33554432.0}

off = dict(no_fp64=True, no_grid=True, no_paths=True, no_surrogate=True, no_fig1=True,
           no_spheres=True, no_surfaces=True, no_cpu_baseline=True)
bench.run_gpu(argparse.Namespace(gpus=int(os.environ.get("WORLD_SIZE", "1")), steps=2, warmup=3,
                                 impl="ours", paths_steps=1,
                                 rays=4096, sur_train=0, sur_queries=0, sur_check=0,
                                 grid_steps=1, fp64_steps=1, cpu_sample=0, ref_sample=0,
                                 no_tune=False, grid_rays=4_194_304, **off))
'''


def _last_json(out):
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def _run(args, **kw):
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600, **kw)
    assert p.returncode == 0, p.stderr[-3000:]
    return _last_json(p.stdout)


def test_reference_arm_line():
    d = _run(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
              "--ref-sample", "32"])
    assert BASE_KEYS <= d.keys()
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["host"].endswith("logical CPUs")
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_gpu_arm_line_with_fakes():
    d = _run(["-c", "import sys; sys.path.insert(0, '.'); exec(sys.stdin.read())"],
             input=_FAKE_GPU_ARM)
    assert BASE_KEYS <= d.keys()
    assert "impl" not in d and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["scaling"] == "weak" and d["data"] == "synthetic" and d["vs_baseline"] is None
    # 4,096 primaries x 300 accepted steps per 10 ms step
    assert abs(d["value"] - 4096 * 300 / 10e-3) <= 1e-6 * d["value"]
    e = d["e2e"]
    assert e["unit"] == d["unit"] and e["value"] > 0
    assert e["h2d_bytes_per_step"] == 4096 * 7 * 8  # pos, dir (3 x f64) and amp (f64)
    assert e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    c = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= c.keys()
    assert c["remeasured_after"] == "hw_slowdown" and c["reasons"] == ["sw_power_cap"]
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= r.keys()
    assert r["bound"] == "alu" and abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-12
    # the peak is the measured FP32 rate (sampled at 2000 MHz, as the run) at the run's clock
    assert d["measured_peaks"]["fp32_tflops"] == 70.0 and abs(r["peak"] - 70.0) <= 1e-9
    assert d["modes"]["fp32_mixed"]["roofline"] == r
    k = d["tuned_knobs"]
    assert k["candidates"] == 27 and k["block"] in (64, 128, 256) and k["service_idle"] > 0
    # 364 flops per attempted step (335 per primary) over the 9 ms kernel time
    assert abs(r["achieved"] - 364 * 335 * 4096 / 9e-3 / 1e12) <= 1e-9 * r["achieved"]
    assert r["traffic"] is None  # measured for the full-size workload only
    assert "workload" in d["config"]


def test_gpu_arm_two_ranks_with_fakes():
    """Two replicas (gloo in place of NCCL): the value sums both ranks' steps over the slowest
    rank's time, the CPU baseline is skipped, and a throttled clock record on rank 1 alone
    makes both ranks measure again."""
    import socket

    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), THROTTLED_RANK="1")
        procs.append(subprocess.Popen(
            [sys.executable, "-c", "import sys; sys.path.insert(0, '.'); exec(sys.stdin.read())"],
            cwd=ROOT, env=env, stdin=subprocess.PIPE, stdout=subprocess.PIPE,
            stderr=subprocess.PIPE, text=True))
    for p in procs:  # both ranks get their script before either is waited on
        p.stdin.write(_FAKE_GPU_ARM)
        p.stdin.close()
    try:
        outs = [(p.stdout.read(), p.stderr.read()) for p in procs]
        for p in procs:
            p.wait(timeout=600)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-3000:]
    assert not [ln for ln in outs[1][0].splitlines() if ln.startswith("{")]  # rank 1 is silent
    d = _last_json(outs[0][0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak"
    assert abs(d["value"] - 2 * 4096 * 300 / 10e-3) <= 1e-6 * d["value"]
    assert d["cpu_baseline"] is None
    assert d["clocks"]["remeasured_after"] == "a throttled clock record on another rank"
