"""Benchmark of the ray-propagation hot path on GB300 (one JSON line on stdout).

Workload: the batched two-layer-ice scenario -- 1,048,576 isotropic rays from sources at
50..1500 m depth, exponential ice n(z) = 1.788 - 0.463 exp(-z / 75 m), an internal boundary
at 100 m (+0.02), the ice-air surface at 0 m, secondaries up to generation 3 through the
device work queue, 64 receiver spheres, Cash-Karp tol 1e-6, steps 1e-3..10 m, 3 km paths.
One step = one rp_trace call over the whole batch (every generation, every receiver test).

Headline value: accepted Cash-Karp ray-steps per second of the FP32-mixed path (FP32 stages,
float-float position and direction, FP64 travel time and path length); the FP64 path, rays/s
and the FP32-vs-FP64 error are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-fp64]

--impl reference times the plain FP64 CPU oracle on the host cores (bounded sample of the
same workload).  Under torchrun each rank traces its own batch (weak scaling, no data-path
collective); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-steps/s and rays/s on 1 GB300: FP64 vs FP32 vs surrogate at stated error"
WORKLOAD = ("batched two-layer ice: 1,048,576 isotropic rays, sources 50-1500 m, internal "
            "boundary at 100 m (+0.02), surface reflection, secondaries to generation 3, "
            "64 receivers, tol 1e-6, h 1e-3..10 m, 3 km paths")
N_RAYS = 1_048_576
# Algorithmic FP32 flops of one attempted Cash-Karp step of the FP32-mixed path in a layered
# analytic medium, counted from trace_core.cuh (ck_step_vgrad and the step's control, event
# test and commit; FMA = 2, a sum of m products = 2m - 1): stage combinations 75, stage states
# 30, medium 30, projection 36, fifth-order sums 35, error sums 36, increments 16, error norms
# 13, control 3, event tests 10, float-float state update 80.  The 6 exp, 6 reciprocals and
# the pow of the step control are not counted.
FLOPS_PER_ATTEMPT_F32 = 364
# The same Runge-Kutta step in FP64 (trace_core.cuh, PrecF64): stage combinations 75, stage
# states 30, medium 30, projection 36, fifth-order sums 35, error sums 36, increments 10, error
# norms 13, control 3, event tests 10, state update 13 (position, direction, travel time and
# arc length sums and the direction's renormalisation); 6 exp, 6 divisions and 3 square roots
# not counted.
FLOPS_PER_ATTEMPT_F64 = 291
# Eq. 1 as written on p = n t (ck_step_momentum, FP64): stage combinations 150, stage states 60,
# medium 30, |p| 30, momentum 3, fifth-order sums 49, error sums 54, increments and their norms
# 24, control 3, event tests 10, state update 13; 22 divisions, 9 square roots, 6 exp not
# counted.
FLOPS_PER_ATTEMPT_MOMENTUM = 432
# Spheres (FP32-mixed): the layered step plus, per attempted step, the float-float distance to
# each of the workload's two spheres from the candidate end point (91 flops each: the
# difference, its square and sum in float-float, (|w|^2 - R^2) / (|w| + R)); FP64: 13 each.
FLOPS_PER_ATTEMPT_SPHERES_F32 = 364 + 2 * 91
FLOPS_PER_ATTEMPT_SPHERES_F64 = 291 + 2 * 13
SM_COUNT_NOMINAL = 152  # GB300, for the nominal comparison only
# Non-horizontal boundaries: the layered step plus the surface event tests, evaluated in FP64 in
# both precisions (the vertical offset from a tilted plane: 12 flops, counted twice per step;
# the height field's bilinear evaluations are not counted); FP32-mixed counts its FP32 flops.
FLOPS_PER_ATTEMPT_SURFACES_F32 = 364
FLOPS_PER_ATTEMPT_SURFACES_F64 = 291 + 2 * 12
# Gridded medium: 8 float4 corner samples (128 B) per medium evaluation, 6 evaluations per
# attempted step.
BYTES_PER_ATTEMPT_GRID = 768


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(
        os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ----------------------------------------------------------------------------------------

def _oracle_chunk(args):
    lo, hi, seed = args
    import oracle
    from paper_1810_01780_gb300 import workloads as W

    cfg = W.batched(N_RAYS, seed)
    rays = W.subsample(cfg["rays"], np.arange(lo, hi))
    t0 = time.perf_counter()
    out, hits = oracle.trace(cfg["medium"], cfg["params"], *rays, receivers=cfg["receivers"])
    dt = time.perf_counter() - t0
    return int(out["n_acc"].sum()), int(len(out)), dt


def oracle_sample(n_primaries: int, seed: int = 2, cores: int | None = None):
    """Trace the first n_primaries rays of the workload with the oracle on `cores` processes.
    Returns (ray_steps, rays, wall_seconds, cores)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = cores or os.cpu_count() or 1
    cores = max(1, min(cores, n_primaries))
    bounds = np.linspace(0, n_primaries, cores + 1).astype(int)
    chunks = [(int(bounds[i]), int(bounds[i + 1]), seed) for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(0, 1, seed)] * cores)  # warm the workers
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, chunks)
        wall = time.perf_counter() - t0
    return sum(r[0] for r in res), sum(r[1] for r in res), wall, cores


def host_cpu() -> str:
    """Architecture and CPU model of this host (lscpu's model name where it reports one)."""
    import platform
    import subprocess

    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{platform.machine()}{', ' + model if model else ''}, {os.cpu_count()} logical CPUs"


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    sample = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(max(16, sample // 8))
    steps_tot = rays_tot = wall_tot = 0.0
    cores = 1
    for _ in range(args.steps):
        s, r, w, cores = oracle_sample(sample)
        steps_tot += s
        rays_tot += r
        wall_tot += w
    v = steps_tot / wall_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ray-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "rays_per_s": rays_tot / wall_tot,
        "config": {"workload": WORKLOAD, "rays": N_RAYS, "precision": "fp64 (CPU oracle)",
                   "sample": f"first {sample} primaries (+ their secondaries) per step",
                   "device": f"{cores} host cores on rank 0; the launch's GPUs are not used"},
        "cpu_baseline": {"value": v, "unit": "ray-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} primaries of the workload, all secondaries",
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": "ray-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------

class ClockSampler:
    """SM clock and clock-event reasons of this process's GPU, sampled every 5 ms by a thread
    through NVML (read-only queries) while the timed region runs."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int):
        self.cuda_index = cuda_index
        self.samples, self.max_mhz, self.err, self.how = [], None, None, None

    def _handle(self, nv):
        import ctypes as C
        import torch

        h = C.c_void_p()
        uuid = getattr(torch.cuda.get_device_properties(self.cuda_index), "uuid", None)
        if uuid is not None:
            key = ("GPU-" + str(uuid)).encode()
            if nv.nvmlDeviceGetHandleByUUID(key, C.byref(h)) == 0:
                self.how = "uuid"
                return h
        if nv.nvmlDeviceGetHandleByIndex_v2(self.cuda_index, C.byref(h)) == 0:
            self.how = "index"
            return h
        raise OSError("no NVML handle")

    def __enter__(self):
        import ctypes as C
        import threading

        self.stop = threading.Event()
        self.thread = None
        try:
            nv = C.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = self._handle(nv)
            mx = C.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0:  # 1: SM clock
                self.max_mhz = float(mx.value)
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError) as e:
            self.err = str(e)
            return self

        def run():
            clk, rs = C.c_uint(), C.c_ulonglong()
            while not self.stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and \
                        get_reasons(h, C.byref(rs)) == 0:
                    self.samples.append((float(clk.value), int(rs.value)))
                self.stop.wait(0.005)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz,
                    "reasons": ["unsampled" + (f": {self.err}" if self.err else "")], "samples": 0}
        reasons = sorted({nm for _, r in self.samples for bit, nm in self.REASONS.items()
                          if r & bit})
        return {"sm_mhz": statistics.median(c for c, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(self.samples),
                "source": f"NVML every 5 ms during the timed region (device by {self.how})"}


# a clock record with one of these active rejects the timing it was taken over
THROTTLE_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_reject(clocks):
    """Why a clock record rejects the timing taken under it, or None: a hardware or thermal
    slowdown was active, or the median SM clock sat below 85 % of its maximum with no reason
    active (a clock left locked).  A power cap alone keeps the timing."""
    bad = [r for r in clocks.get("reasons") or [] if r in THROTTLE_REASONS]
    if bad:
        return "+".join(bad)
    mhz, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    if mhz and mx and mhz < 0.85 * mx and not clocks.get("reasons"):
        return f"SM clock {mhz:.0f} of {mx:.0f} MHz with no reason active"
    return None


def any_rank(flag, device):
    """True on every rank when the flag is set on any rank (one rank: the flag itself)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return bool(flag)
    t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return bool(t.item())


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


MLP_FLOPS_FWD = 2 * (3 * 256 + 3 * 256 * 256 + 256 * 12)  # per row, multiply-adds x 2

# DRAM bytes (read + write) of the four k_trace_wave<PrecF32, MediumLayered> launches of one
# step of the 1,048,576-ray batched workload, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the current kernel (profiles/k_trace_wave_f32_layered_1M_dram.md)
TRACE_DRAM_BYTES_PER_STEP = 1_966_933_248


def peaks_leg(rp, local):
    """The roofline denominators of this GPU measured by the library's microkernels
    (rp_measure_peaks), with the SM clock sampled while they run."""
    with ClockSampler(local) as clk:
        pk = rp.measure_peaks()
    pk["clocks"] = clk.summary()
    pk["how"] = ("rp_measure_peaks: FP32 / FP64 FMA chains (8 independent per thread, 1,024 "
                 "threads per SM) and 16-byte L1-bypassing loads over a 32 MiB L2-resident "
                 "buffer; best of 3 timed launches each")
    return pk


def at_clock(rate, pk, sm_mhz):
    """A measured peak rate moved to the SM clock of the run it is the denominator for (the
    microkernels and the run may see different clocks under the power cap)."""
    mhz = (pk.get("clocks") or {}).get("sm_mhz")
    return rate * (sm_mhz / mhz) if (mhz and sm_mhz) else rate


def alu_roofline(flops_per_attempt, attempts, ms, peak, kernel, basis):
    achieved = flops_per_attempt * attempts / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "kernel": kernel,
            "flops_per_attempted_step": flops_per_attempt, "peak_basis": basis}


def _sync_time(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def surrogate_leg(rp, W, args, rank, flush):
    import torch

    scfg = W.surrogate(n_train=args.sur_train, n_query=args.sur_queries, seed=5 + 16 * rank)
    med = rp.Medium(scfg["medium"])
    P, tr, q = scfg["params"], scfg["train"], scfg["queries"]
    t_lab, lab = _sync_time(lambda: rp.find_paths(
        med, tr["zs"], tr["zr"], tr["dist"], tr["n_angles"], P, "fp32",
        hit_tol=scfg["label_hit_tol"], max_iter=scfg["max_iter"], max_sol=scfg["max_sol"]))
    x, y, t = rp.encode(tr["zs"], tr["zr"], tr["dist"], lab)
    del lab
    net = rp.Surrogate(seed=0)
    sch = scfg["schedule"]
    t_train, loss = _sync_time(lambda: net.train(x, y, t, epochs=sch["epochs"], batch=sch["batch"],
                                                 lr=sch["lr"], lr_final=sch["lr_final"],
                                                 seed=sch["seed"]))
    n_steps = sch["epochs"] * (len(tr["zs"]) // sch["batch"])
    del x, y, t
    buf = rp.PathBuffers(q["zs"], q["zr"], q["dist"], q["n_angles"], scfg["max_sol"])
    pprm = rp.make_path_params(P, "fp32", scfg["hit_tol"], scfg["max_iter"], scfg["max_sol"])
    sprm = rp.make_surrogate_params(**scfg["infer"])
    net.find_paths_into(med, buf, pprm, sprm)  # warm-up (sizes the buffers)
    t_inf, n_sol, agg = [], 0, {}
    for _ in range(args.paths_steps):
        flush.fill_(1.0)
        dt, st = _sync_time(lambda: net.find_paths_into(med, buf, pprm, sprm))
        t_inf.append(dt)
        n_sol += int(buf.count.sum())
        for k, v in st.as_dict().items():
            agg[k] = agg.get(k, 0) + v
    sur = {k: buf.t[k][:args.sur_check].cpu().numpy() for k in ("launch", "time")}
    sur_count = buf.count[:args.sur_check].cpu().numpy()
    sec = sum(t_inf)
    sol_s = n_sol / sec
    # the plain path finder on the same queries, same tolerance
    flush.fill_(1.0)
    t_plain, _ = _sync_time(lambda: rp.find_paths_into(med, buf, pprm))
    plain_sol_s = int(buf.count.sum()) / t_plain
    # error against the FP64 path finder (0.1 mm) on the first queries; count mismatches
    # decided by an 8192-angle FP64 scan
    m = args.sur_check
    truth = rp.find_paths(med, q["zs"][:m], q["zr"][:m], q["dist"][:m], q["n_angles"][:m], P,
                          "fp64", hit_tol=1e-4, max_iter=80, max_sol=scfg["max_sol"])
    tc = truth["count"].cpu().numpy()
    tl, tt = truth["launch"].cpu().numpy(), truth["time"].cpu().numpy()
    bad = np.nonzero(sur_count != tc)[0]
    adj = tc.copy()
    if len(bad):
        fine = rp.find_paths(med, q["zs"][bad], q["zr"][bad], q["dist"][bad],
                             np.full(len(bad), 8192, np.int32), P, "fp64", hit_tol=1e-4,
                             max_iter=80, max_sol=scfg["max_sol"])
        adj[bad] = fine["count"].cpu().numpy()
    errs = []
    for i in np.nonzero((sur_count > 0) & (tc > 0))[0]:
        for j in range(sur_count[i]):
            k = int(np.argmin(np.abs(tl[i, :tc[i]] - sur["launch"][i, j])))
            errs.append(abs(sur["time"][i, j] - tt[i, k]))
    errs = np.array(errs) if errs else np.zeros(1)
    # the network on its own, before any refinement trace: predicted existence and launch angle
    # of the two earliest solutions against the FP64 path finder on the same queries
    xq, _, _ = rp.encode(q["zs"][:m], q["zr"][:m], q["dist"][:m])
    pred = net.forward(xq).cpu().numpy().astype(np.float64)
    two = tc <= 2
    exist_ok, ang = [], []
    for k in range(2):
        said = pred[:, 6 * k] > 0.0  # the existence logit: sigmoid > 1/2 exactly when it is > 0
        has = tc > k
        exist_ok.append((said == has)[two])
        both = two & has & said
        ang.append(np.abs((pred[both, 6 * k + 1] + 1.0) * (np.pi / 2) - tl[both, k]))
    ang = np.concatenate(ang) if ang else np.zeros(1)
    network_alone = {
        "vs": f"FP64 path finder on the first {m:,} queries with at most two solutions",
        "existence_accuracy": float(np.concatenate(exist_ok).mean()),
        "launch_angle_error_rad": {"p50": float(np.median(ang)), "p99": float(np.percentile(ang, 99)),
                                   "max": float(ang.max())},
        "note": "the refinement starts from these angles; each returned solution is a traced ray"}
    nq = len(q["zs"]) * len(t_inf)
    return {
        "workload": f"MLP 3-256x4-12 trained on {len(tr['zs']):,} path-finder-labelled pairs; "
                    f"inference on {len(q['zs']):,} queries, secant/Illinois refinement to a "
                    "5 mm receiver miss, fallback to the path finder",
        "solutions_per_s": sol_s, "pairs_per_s": nq / sec,
        "plain_path_finder_solutions_per_s": plain_sol_s, "gain_vs_plain": sol_s / plain_sol_s,
        "ms_per_step": 1e3 * sec / len(t_inf),
        "fallback_fraction": agg["fallback"] / agg["queries"],
        "refine_rays_per_query": agg["refine_rays"] / agg["queries"],
        "ray_steps_per_s": (agg["refine_steps"] + agg["fallback_steps"]) / sec,
        "ms_phases": {k: agg[k] / len(t_inf) for k in ("ms_forward", "ms_refine", "ms_fallback",
                                                       "ms_fallback_scan")},
        "mlp_forward_tflops": MLP_FLOPS_FWD * len(q["zs"]) / (agg["ms_forward"] / len(t_inf) / 1e3)
                              / 1e12,
        "error": {"vs": f"FP64 path finder (0.1 mm) on the first {m:,} queries",
                  "time_s": {"p50": float(np.median(errs)), "p99": float(np.percentile(errs, 99)),
                             "max": float(errs.max())},
                  "count_agreement_adjudicated": float((sur_count == adj).mean()),
                  "count_agreement_vs_coarse_scan": float((sur_count == tc).mean())},
        "network_alone": network_alone,
        "training": {"label_s": t_lab, "train_s": t_train, "adam_steps": n_steps,
                     "batch": sch["batch"], "epochs": sch["epochs"], "final_loss": loss,
                     "train_tflops": 3 * MLP_FLOPS_FWD * sch["batch"] * n_steps / t_train / 1e12},
    }


def reduce_over_ranks(total_ms, counts, device):
    """Whole-job figures of a timed region: the slowest rank's time (every rank's work counts
    only when all are done) and the sums of the ranks' work counters.  One rank: unchanged."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), [float(v) for v in c]


def fp32_fp64_leg(rp, cfg, flush, steps, flops, peaks, workload, tune=True):
    """One trace workload in both precisions: ray-steps/s and rays/s (kernel time, L2 flushed
    before each call), each precision's ALU roofline (flops[prec] per attempted step against
    peaks[prec], TFLOP/s) and the FP32-mixed end points of the primaries against FP64.  The
    FP32-mixed scheduling knobs (speed only, never a record) are tuned on the workload first."""
    from paper_1810_01780_gb300 import autotune

    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"])
    buf = rp.TraceBuffers(3 * rays.n, 0, fields=("end_pos", "path", "time", "status"))
    leg, ends = {"workload": workload}, {}
    params = {"fp32": dict(cfg["params"]), "fp64": dict(cfg["params"])}
    if tune:
        t = autotune.tune_trace(med, rays, cfg["params"], buf, "fp32", idle=(256, 512),
                                flush=(1, 2), block=(128, 256), reps=1)
        params["fp32"] = t["params"]
        leg["tuned_knobs_fp32"] = t["best"]
    for prec in ("fp32", "fp64"):
        prm = rp.make_params(params[prec], prec)
        rp.trace_into(med, rays, prm, buf)  # warm-up
        ts, acc, att, nr = [], 0, 0, 0
        for _ in range(steps):
            flush.fill_(1.0)
            st = rp.trace_into(med, rays, prm, buf)
            ts.append(st.kernel_ms)
            acc += st.steps_accepted
            att += st.steps_accepted + st.steps_rejected + st.steps_root
            nr += st.rays
        sec = sum(ts) / 1e3
        name = "fp32_mixed" if prec == "fp32" else "fp64"
        leg[name] = {
            "ray_steps_per_s": acc / sec, "rays_per_s": nr / sec, "ms_per_step": 1e3 * sec / len(ts),
            "roofline": alu_roofline(flops[prec], att, 1e3 * sec, peaks[prec][0],
                                     "k_trace_wave<%s, %s>" % (
                                         "PrecF32" if prec == "fp32" else "PrecF64",
                                         cfg.get("kernel_medium", "MediumLayered")),
                                     peaks[prec][1])}
        ends[prec] = (buf.t["end_pos"][:, :rays.n].clone(), buf.t["time"][:rays.n].clone())
    dpos = (ends["fp32"][0] - ends["fp64"][0]).norm(dim=0)
    dt = (ends["fp32"][1] - ends["fp64"][1]).abs()
    leg["error_fp32_vs_fp64"] = {
        "primaries": rays.n, "pos_m_p99": float(dpos.double().quantile(0.99)),
        "time_s_p99": float(dt.double().quantile(0.99)),
        "within_1mm_10ps": float(((dpos <= 1e-3) & (dt <= 1e-11)).double().mean())}
    return leg


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    # CPU baseline first (spawned pool), before this process does heavy GPU work; one GPU only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s, r, w, cores = oracle_sample(args.cpu_sample)
        cpu = {"value": s / w, "unit": "ray-steps/s", "cores": cores, "kind": "oracle",
               "host": host_cpu(),
               "sample": f"first {args.cpu_sample} primaries of the workload with all their "
                         f"secondaries ({r} rays, {s} accepted steps, {w:.2f} s wall)"}

    from paper_1810_01780_gb300 import build as B

    B.build()
    import paper_1810_01780_gb300 as rp
    from paper_1810_01780_gb300 import workloads as W

    from paper_1810_01780_gb300 import autotune

    # roofline denominators of this GPU, measured before anything else runs
    peaks = peaks_leg(rp, local)
    mp = _peaks()

    n_rays = args.rays
    seed = 2 + rank  # weak scaling: every rank traces its own batch
    cfg = W.batched(n_rays, seed)
    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"], receivers=cfg["receivers"])
    cap = int(5.5 * n_rays)
    buf = rp.TraceBuffers(cap, 4096)
    stream = torch.cuda.current_stream()
    # the scheduling knobs (speed only, never a record) tuned on this batch
    t0 = time.perf_counter()
    if args.no_tune:
        tuned = {"best": dict.fromkeys(("service_idle", "flush_min", "block", "blocks_per_sm"), 0),
                 "ms": {}, "params": dict(cfg["params"])}
    else:
        tuned = autotune.tune_trace(med, rays, cfg["params"], buf, "fp32", idle=(192, 256, 384),
                                    flush=(1, 2, 4), block=(64, 128, 256), reps=1)
    tune_s = time.perf_counter() - t0
    prm32 = rp.make_params(tuned["params"], "fp32")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(prm, b):
        flush.fill_(1.0)  # evict the L2 (129 MB) between steps, outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = rp.trace_into(med, rays, prm, b, stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), st

    def timed_region():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        times, kern, acc, att, nrays = [], [], 0, 0, 0
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                ms, st = one_step(prm32, buf)
                times.append(ms)
                kern.append(st.kernel_ms)
                acc += st.steps_accepted
                att += st.steps_accepted + st.steps_rejected + st.steps_root
                nrays += st.rays
            torch.cuda.synchronize()
        return times, kern, acc, att, nrays, clk.summary()

    for _ in range(args.warmup):
        one_step(prm32, buf)
    times, kern, acc, att, nrays, clocks = timed_region()
    why = clocks_reject(clocks)
    if any_rank(why is not None, "cuda"):  # a throttled or clock-locked run: measured once more
        times, kern, acc, att, nrays, clocks = timed_region()
        clocks["remeasured_after"] = why or "a throttled clock record on another rank"
    total_ms_max, (acc_all, rays_all) = reduce_over_ranks(sum(times), [acc, nrays], "cuda")
    value = acc_all / (total_ms_max / 1e3)

    # primary end points of the FP32 run for the stated error against FP64
    end32 = buf.t["end_pos"][:, :n_rays].clone()
    t32 = buf.t["time"][:n_rays].clone()
    s32 = buf.t["status"][:n_rays].clone()

    # e2e: host (pinned) -> device -> rp_trace -> host, through the same C ABI call
    hp = torch.from_numpy(np.ascontiguousarray(cfg["rays"][0])).pin_memory()
    hd = torch.from_numpy(np.ascontiguousarray(cfg["rays"][1])).pin_memory()
    ha = torch.from_numpy(np.ascontiguousarray(cfg["rays"][2])).pin_memory()
    out_fields = ("end_pos", "path", "time", "amp", "status")
    host_out = {k: torch.empty(buf.t[k].shape, dtype=buf.t[k].dtype).pin_memory()
                for k in out_fields}
    h2d_b = hp.numel() * 8 + hd.numel() * 8 + ha.numel() * 8

    def upload(r):
        r.pos.copy_(hp, non_blocking=True)
        r.dir.copy_(hd, non_blocking=True)
        r.amp.copy_(ha, non_blocking=True)

    def download(b, n_out):
        for k in out_fields:
            src = b.t[k]
            # one contiguous copy per component row of the (3, capacity) arrays: a strided
            # slice copy of all three rows at once runs at a fraction of the link's bandwidth
            for r in (range(src.shape[0]) if src.dim() == 2 else (None,)):
                d, s_ = (host_out[k], src) if r is None else (host_out[k][r], src[r])
                d[:n_out].copy_(s_[:n_out], non_blocking=True)
        return sum(b.t[k][..., :n_out].numel() * b.t[k].element_size() for k in out_fields)

    # serial: each step uploads, traces and reads back before the next one starts
    e2e_ms, d2h_b = [], 0
    for it in range(max(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upload(rays)
        st = rp.trace_into(med, rays, prm32, buf, stream)
        d2h_b = download(buf, int(st.rays))
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    serial_val = acc / len(times) / (statistics.median(e2e_ms) / 1e3)
    # pipelined, as a serving loop runs it: two input and two output buffers; step k + 1's
    # inputs go up and step k's records come back on a copy stream while the next step traces.
    # The timed region holds every step's upload, trace and read-back, from the first upload
    # to the last read-back.
    rays_b = [rays, rp.PreparedRays(*cfg["rays"], receivers=cfg["receivers"])]
    buf_b = [buf, rp.TraceBuffers(cap, 4096)]
    cst = torch.cuda.Stream()
    k_pipe = max(4, args.steps)
    pipe_ms = []
    for rep in range(2):  # the first pass warms the second buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(cst):
            upload(rays_b[0])
            up = torch.cuda.Event()
            up.record(cst)
        for k in range(k_pipe):
            nxt = None
            if k + 1 < k_pipe:
                with torch.cuda.stream(cst):  # buffer (k + 1) % 2: its last trace has returned
                    upload(rays_b[(k + 1) % 2])
                    nxt = torch.cuda.Event()
                    nxt.record(cst)
            stream.wait_event(up)
            st = rp.trace_into(med, rays_b[k % 2], prm32, buf_b[k % 2], stream)
            with torch.cuda.stream(cst):  # recorded after upload k + 1: trace k + 2 waits for it
                download(buf_b[k % 2], int(st.rays))
            up = nxt
        torch.cuda.synchronize()
        pipe_ms.append((time.perf_counter() - t0) * 1e3 / k_pipe)
    e2e_val = acc / len(times) / (pipe_ms[-1] / 1e3)

    # FP64 path on the same batch (fewer steps; FP64 issue rate on GB300 is low)
    modes = {"fp32_mixed": {"ray_steps_per_s": value, "rays_per_s": rays_all / (total_ms_max / 1e3),
                            "ms_per_step": total_ms_max / args.steps}}
    err = None
    pk32 = at_clock(peaks["fp32_tflops"], peaks, clocks["sm_mhz"])
    basis32 = ("rp_measure_peaks FP32 FMA rate %.1f TFLOP/s at %s MHz, moved to the run's median "
               "SM clock" % (peaks["fp32_tflops"], (peaks["clocks"] or {}).get("sm_mhz")))
    pk64 = at_clock(peaks["fp64_tflops"], peaks, clocks["sm_mhz"])
    basis64 = ("rp_measure_peaks FP64 FMA rate %.3f TFLOP/s at %s MHz, moved to the run's median "
               "SM clock" % (peaks["fp64_tflops"], (peaks["clocks"] or {}).get("sm_mhz")))
    if not args.no_fp64:
        prm64 = rp.make_params(cfg["params"], "fp64")
        one_step(prm64, buf)
        t64, k64 = [], []
        acc64 = rays64 = att64 = 0
        for _ in range(args.fp64_steps):
            ms, st = one_step(prm64, buf)
            t64.append(ms)
            k64.append(st.kernel_ms)
            acc64 += st.steps_accepted
            att64 += st.steps_accepted + st.steps_rejected + st.steps_root
            rays64 += st.rays
        modes["fp64"] = {"ray_steps_per_s": acc64 / (sum(t64) / 1e3),
                         "rays_per_s": rays64 / (sum(t64) / 1e3), "ms_per_step": sum(t64) / len(t64),
                         "roofline": alu_roofline(FLOPS_PER_ATTEMPT_F64, att64, sum(k64), pk64,
                                                  "k_trace_wave<PrecF64, MediumLayered>", basis64)}
        end64 = buf.t["end_pos"][:, :n_rays].clone()
        t64e = buf.t["time"][:n_rays].clone()
        s64 = buf.t["status"][:n_rays].clone()
        # conditioning: the FP64 run again with every launch direction tilted by 1e-7 rad; a
        # primary whose FP64 result moves by more than 1 mm / 10 ps (or changes status) under
        # the tilt is ill-conditioned (grazing or critical incidence, an amplitude at its
        # threshold)
        trays = rp.PreparedRays(cfg["rays"][0], W.tilted_dirs(cfg["rays"][1], 1e-7, 9),
                                cfg["rays"][2], receivers=cfg["receivers"])
        rp.trace_into(med, trays, prm64, buf, stream)
        sens = (((end64 - buf.t["end_pos"][:, :n_rays]).norm(dim=0) > 1e-3) |
                ((t64e - buf.t["time"][:n_rays]).abs() > 1e-11) |
                (s64 != buf.t["status"][:n_rays]))
        del trays
        d = (end32 - end64).norm(dim=0)
        dT = (t32 - t64e).abs()
        outside = (d > 1e-3) | (dT > 1e-11) | (s32 != s64)
        err = {"vs": f"FP64 GPU path, all {n_rays:,} primary end points",
               "within_1mm_10ps": float((~outside).double().mean()),
               "outside_1mm_10ps": int(outside.sum()),
               "outside_and_not_tilt_sensitive": int((outside & ~sens).sum()),
               "tilt_sensitive_fraction": float(sens.double().mean()),
               "conditioning": "FP64 end point moves > 1 mm / 10 ps or changes status under a "
                               "1e-7 rad launch tilt",
               "pos_m": {"p50": float(d.quantile(0.5)), "p99": float(d.double().quantile(0.99)),
                         "max": float(d.max())},
               "time_s": {"p50": float(dT.quantile(0.5)), "p99": float(dT.quantile(0.99)),
                          "max": float(dT.max())}}
        # Eq. 1 integrated as written (momentum form, FP64 only): the same batch, end points
        # against the projected FP64 run just made
        prmm = rp.make_params(dict(cfg["params"], rhs_form="momentum"), "fp64")
        one_step(prmm, buf)
        tm, km, accm, raysm, attm = [], [], 0, 0, 0
        for _ in range(args.fp64_steps):
            ms, st = one_step(prmm, buf)
            tm.append(ms)
            km.append(st.kernel_ms)
            accm += st.steps_accepted
            attm += st.steps_accepted + st.steps_rejected + st.steps_root
            raysm += st.rays
        dm = (end64 - buf.t["end_pos"][:, :n_rays]).norm(dim=0)
        dTm = (t64e - buf.t["time"][:n_rays]).abs()
        modes["fp64_momentum"] = {
            "ray_steps_per_s": accm / (sum(tm) / 1e3), "rays_per_s": raysm / (sum(tm) / 1e3),
            "ms_per_step": sum(tm) / len(tm),
            "roofline": alu_roofline(FLOPS_PER_ATTEMPT_MOMENTUM, attm, sum(km), pk64,
                                     "k_trace_wave<PrecF64, MediumLayered> (momentum form)",
                                     basis64),
            "vs_projected_fp64": {"pos_m_p99": float(dm.double().quantile(0.99)),
                                  "time_s_p99": float(dTm.double().quantile(0.99)),
                                  "within_1mm_10ps": float(((dm <= 1e-3) & (dTm <= 1e-11))
                                                           .double().mean())}}

    # gridded medium: 256 x 256 x 512 FP32 grid, 4,194,304 rays (FP32-mixed), its own
    # figures (memory-bound path: algorithmic bytes = 8 float4 corner samples per medium
    # evaluation, 6 evaluations per attempted step)
    if not args.no_grid:
        gcfg = W.gridded(per_src=args.grid_rays // 16)
        gmed = rp.Medium(gcfg["medium"])
        grays = rp.PreparedRays(*gcfg["rays"])
        gbuf = rp.TraceBuffers(grays.n + 16, 0, fields=("end_pos", "path", "time", "status"))
        gprm = rp.make_params(gcfg["params"], "fp32")
        rp.trace_into(gmed, grays, gprm, gbuf)  # warm-up
        gt, gatt, gacc, gr = [], 0, 0, 0
        for _ in range(args.grid_steps):
            flush.fill_(1.0)
            st = rp.trace_into(gmed, grays, gprm, gbuf)
            gt.append(st.kernel_ms)
            gacc += st.steps_accepted
            gatt += st.steps_accepted + st.steps_rejected + st.steps_root
            gr += st.rays
        gsec = sum(gt) / 1e3
        bytes_alg = float(BYTES_PER_ATTEMPT_GRID) * gatt
        gbs = bytes_alg / gsec / 1e9
        modes["grid_fp32_mixed"] = {
            "workload": "256x256x512 FP32 grid (4 m), %d rays from 16 sources, tol 1e-5" % grays.n,
            "ray_steps_per_s": gacc / gsec, "rays_per_s": gr / gsec,
            "ms_per_step": 1e3 * gsec / len(gt),
            "roofline": {"bound": "l2", "achieved": gbs, "peak": peaks["l2_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["l2_gbs"],
                         "kernel": "k_trace_wave<PrecF32, MediumGrid>",
                         "bytes_per_attempted_step": BYTES_PER_ATTEMPT_GRID,
                         "peak_basis": "rp_measure_peaks L2-resident read bandwidth",
                         "hbm_peak": mp.get("hbm_gbs"),
                         "frac_of_hbm": gbs / mp["hbm_gbs"] if mp.get("hbm_gbs") else None},
        }
        del gmed, grays, gbuf

    # the paper's Fig. 1 example as a 1,048,576-ray fan: firn layer over ice, 5 us, A/A0 cut
    if not args.no_fig1:
        modes["fig1"] = fp32_fp64_leg(
            rp, W.fig1(), flush, args.grid_steps,
            {"fp32": FLOPS_PER_ATTEMPT_F32, "fp64": FLOPS_PER_ATTEMPT_F64},
            {"fp32": (pk32, basis32), "fp64": (pk64, basis64)},
            "Fig. 1 example: 1,048,576 rays from 240 m in the x-z plane, 10 m of n = 1.5 over "
            "exponential ice (z0 = 71.4 m), 5 us, A/A0 < 0.05 discarded, generations <= 8",
            tune=not args.no_tune)
    # curved boundaries: two spherical inclusions in the ice, 1,048,576 isotropic rays
    if not args.no_spheres:
        modes["spheres"] = fp32_fp64_leg(
            rp, dict(W.spheres(), kernel_medium="MediumSpheres"), flush, args.grid_steps,
            {"fp32": FLOPS_PER_ATTEMPT_SPHERES_F32, "fp64": FLOPS_PER_ATTEMPT_SPHERES_F64},
            {"fp32": (pk32, basis32), "fp64": (pk64, basis64)},
            "spherical inclusions: 1,048,576 isotropic rays around a denser-ice lens (R 40 m) "
            "and an air pocket (R 25 m) in the surface-bounded ice, 2 km, A/A0 < 0.05, "
            "generations <= 3", tune=not args.no_tune)

    # non-horizontal boundaries: a tilted ice surface carrying a height field of undulations and
    # a tilted internal boundary, 1,048,576 isotropic rays
    if not args.no_surfaces:
        modes["surfaces"] = fp32_fp64_leg(
            rp, dict(W.surfaces(), kernel_medium="MediumSurfaces"), flush, args.grid_steps,
            {"fp32": FLOPS_PER_ATTEMPT_SURFACES_F32, "fp64": FLOPS_PER_ATTEMPT_SURFACES_F64},
            {"fp32": (pk32, basis32), "fp64": (pk64, basis64)},
            "non-horizontal boundaries: 1,048,576 isotropic rays under a 2-degree tilted ice "
            "surface with a 0.3 m height field of undulations (256 x 256 nodes at 2 m) and a "
            "1-degree tilted internal boundary at 100 m, 2 km, A/A0 < 0.05, generations <= 3",
            tune=not args.no_tune)

    # source-receiver path finding: 65,536 pairs, 32..512 scan angles each, FP64 bisection
    if not args.no_paths:
        pcfg = W.paths()
        P = pcfg["pairs"]
        pbuf = rp.PathBuffers(P["zs"], P["zr"], P["dist"], P["n_angles"], pcfg["max_sol"])
        pprm = rp.make_path_params(pcfg["params"], "fp32", pcfg["hit_tol"], pcfg["max_iter"],
                                   pcfg["max_sol"])
        rp.find_paths_into(med_paths := rp.Medium(pcfg["medium"]), pbuf, pprm)  # warm-up
        pt, nsol, prays, pacc, patt = [], 0, 0, 0, 0
        for _ in range(args.paths_steps):
            flush.fill_(1.0)
            st = rp.find_paths_into(med_paths, pbuf, pprm)
            pt.append(st.kernel_ms)
            nsol += int(pbuf.count.sum())
            prays += st.rays
            pacc += st.steps_accepted
            patt += st.steps_accepted + st.steps_rejected + st.steps_root
        psec = sum(pt) / 1e3
        modes["paths_fp32_mixed"] = {
            "workload": "65,536 source-receiver pairs, 32..512 scan angles, FP64 bisection to "
                        "0.1 m, up to 4 solutions per pair",
            "solutions_per_s": nsol / psec, "pairs_per_s": len(P["zs"]) * len(pt) / psec,
            "rays_per_s": prays / psec, "ray_steps_per_s": pacc / psec,
            "ms_per_step": 1e3 * psec / len(pt),
            "roofline": alu_roofline(FLOPS_PER_ATTEMPT_F32, patt, 1e3 * psec, pk32,
                                     "k_scan / k_bisect<PrecF32> (the tracing step of the path "
                                     "finder; all its launches timed)", basis32),
        }

    # learned surrogate of the path finder: labels from the FP32 path finder, native training,
    # inference on 1,048,576 queries with refinement and fallback, against the plain path
    # finder at the same 5 mm receiver tolerance and the FP64 path finder on a sample
    if not args.no_surrogate:
        sur = surrogate_leg(rp, W, args, rank, flush)
        bf16_burst, bf16_sus = mp.get("bf16_tflops"), mp.get("bf16_tflops_sustained")
        tr = sur["training"]["train_tflops"]
        sur["training"]["roofline"] = {
            "bound": "tensor", "achieved": tr, "peak": bf16_sus, "unit": "TFLOP/s",
            "frac": tr / bf16_sus if bf16_sus else None,
            "kernel": "the whole Adam step (k_train_fwd, k_train_bwd, k_tc_wgrad, k_adam_pack)",
            "peak_basis": "MEASURED_PEAKS bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"}
        fw = sur["mlp_forward_tflops"]
        sur["forward_roofline"] = {
            "bound": "tensor", "achieved": fw, "peak": bf16_burst, "unit": "TFLOP/s",
            "frac": fw / bf16_burst if bf16_burst else None, "kernel": "k_mlp_fused",
            "peak_basis": "MEASURED_PEAKS bf16_tflops (cuBLAS bf16 burst)"}
        modes["surrogate"] = sur

    # roofline of the dominant kernel (the FP32 tracing launches): FP32 ALU bound, against the
    # FP32 FMA rate measured on this GPU (moved to the run's clock)
    kern_ms = sum(kern)
    roof = alu_roofline(FLOPS_PER_ATTEMPT_F32, att, kern_ms, pk32,
                        "k_trace_wave<PrecF32, MediumLayered>", basis32)
    roof.update({"traffic": TRACE_DRAM_BYTES_PER_STEP if n_rays == N_RAYS else None,
                 "traffic_unit": "bytes per step (all launches of the step)",
                 "attempted_steps_per_launch_set": att / len(times),
                 "nominal_peak": SM_COUNT_NOMINAL * 128 * 2 * (clocks["sm_mhz"] or 2070.0) / 1e6,
                 "frac_of_nominal": None})
    roof["frac_of_nominal"] = roof["achieved"] / roof["nominal_peak"]
    modes["fp32_mixed"]["roofline"] = roof

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ray-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 accumulators)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays": n_rays, "precision": "fp32_mixed",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "flushed (512 MB write) before every step",
                       "rays_traced_per_step": nrays / len(times)},
            "rays_per_s": rays_all / (total_ms_max / 1e3),
            "modes": modes, "error": err,
            "e2e": {"value": e2e_val, "unit": "ray-steps/s", "h2d_bytes_per_step": h2d_b,
                    "d2h_bytes_per_step": d2h_b, "ms_per_step": pipe_ms[-1],
                    "pipelined": "two buffers: step k + 1 uploads and step k reads back on a "
                                 "copy stream while the next step traces; %d steps" % k_pipe,
                    "serial": {"value": serial_val, "ms_per_step": statistics.median(e2e_ms)}},
            "gpu_launches": args.steps * (1 + 4 + 3),
            "clocks": clocks, "roofline": roof, "cpu_baseline": cpu,
            "measured_peaks": peaks,
            "tuned_knobs": dict(tuned["best"], tune_s=tune_s, candidates=len(tuned["ms"])),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-grid", action="store_true")
    ap.add_argument("--no-paths", action="store_true")
    ap.add_argument("--paths-steps", type=int, default=3)
    ap.add_argument("--rays", type=int, default=N_RAYS,
                    help="primaries of the batched workload (the bench workload is 1,048,576)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-fig1", action="store_true")
    ap.add_argument("--no-spheres", action="store_true")
    ap.add_argument("--no-surfaces", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default scheduling knobs (for profiling runs)")
    ap.add_argument("--grid-rays", type=int, default=4_194_304,
                    help="rays of the gridded leg (the workload is 4,194,304)")
    ap.add_argument("--sur-train", type=int, default=4_194_304)
    ap.add_argument("--sur-queries", type=int, default=1_048_576)
    ap.add_argument("--sur-check", type=int, default=16_384)
    ap.add_argument("--grid-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=65536)
    ap.add_argument("--ref-sample", type=int, default=16384)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
