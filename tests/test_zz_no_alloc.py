"""rp_trace_static -- the allocation-free variant of rp_trace -- against rp_trace.

Callers that cannot allocate device memory while they trace (their device memory is owned
by another allocator's pool, or allocation is banned after start-up because cudaMalloc and
cudaFree can synchronise the device) use rp_trace_static, whose scratch space is a fixed
device array inside the library.  This file checks, through the C ABI, that two calls in a
row give the same rays and receiver hits as rp_trace.  It is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from parity import errors, gpu_rays, match
from paper_1810_01780_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static_call(rp, A, med, rays, prm, cap, hcap):
    import torch

    buf = rp.TraceBuffers(cap, hcap)
    st = A.Stats()
    rc = A.lib().rp_trace_static(med.handle, C.byref(rays.rays), C.byref(rays.rx), C.byref(prm),
                                 C.byref(buf.out), C.byref(buf.hits), C.byref(st),
                                 C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    assert rc == A.RP_OK, A.last_error()
    n, nh = int(st.rays), int(st.hits)
    res = {"rays": {k: (v[:, :n] if v.dim() == 2 else v[:n]) for k, v in buf.t.items()},
           "hits": {k: (v[:, :nh] if v.dim() == 2 else v[:nh]) for k, v in buf.h.items()}}
    return res, st


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_scratch_entry_matches_rp_trace(precision):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp
    from paper_1810_01780_gb300 import _abi as A

    cfg = W.batched()
    pos, d, a = W.subsample(cfg["rays"], np.arange(20000))
    c, r = cfg["receivers"]
    receivers = (c, r * 25.0)
    med = rp.Medium(cfg["medium"])
    ref = rp.trace(med, pos, d, a, params=cfg["params"], receivers=receivers, precision=precision)
    g_ref = gpu_rays(ref)
    rays = rp.PreparedRays(pos, d, a, receivers)
    prm = rp.make_params(cfg["params"], precision)
    cap = len(g_ref["path"]) + 64
    hcap = int(ref["stats"]["hits"]) + 64
    for call in range(2):
        res, st = _static_call(rp, A, med, rays, prm, cap, hcap)
        g = gpu_rays(res)
        assert int(st.rays) == len(g_ref["path"]) and int(st.hits) == int(ref["stats"]["hits"])
        gi, oi, only_s, only_r = match(g, g_ref)
        assert not only_s and not only_r
        assert np.array_equal(g["status"][gi], g_ref["status"][oi])
        assert np.array_equal(g["n_acc"][gi], g_ref["n_acc"][oi])
        dp, dd, ds, dT, dA = errors(g, g_ref, gi, oi)
        # the same kernels on the same inputs: each ray's arithmetic is identical
        assert dp.max() <= 1e-9 and dd.max() <= 1e-12 and ds.max() <= 1e-9
        assert dT.max() <= 1e-18 and dA.max() <= 1e-12
        hs = sorted(zip(res["hits"]["receiver"].cpu().numpy().tolist(),
                        np.round(res["hits"]["time"].cpu().numpy(), 15).tolist()))
        hr = sorted(zip(ref["hits"]["receiver"].cpu().numpy().tolist(),
                        np.round(ref["hits"]["time"].cpu().numpy(), 15).tolist()))
        assert len(hs) == len(hr) > 0
        for x, y in zip(hs, hr):
            assert x[0] == y[0] and abs(x[1] - y[1]) <= 1e-15


def test_static_scratch_rejects_oversized_input():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp
    from paper_1810_01780_gb300 import _abi as A

    cfg = W.small(8)
    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"])
    big = A.Rays((1 << 20) + 1, rays.rays.pos, rays.rays.dir, rays.rays.amp)
    buf = rp.TraceBuffers(16)
    st = A.Stats()
    rc = A.lib().rp_trace_static(med.handle, C.byref(big), None, C.byref(rp.make_params(cfg["params"])),
                                 C.byref(buf.out), None, C.byref(st), None)
    assert rc == -1 and "exceed" in A.last_error()


def test_static_scratch_at_its_ray_limit():
    """rp_trace_static with RP_STATIC_MAX_RAYS (2^20) primaries -- the whole batched workload
    with its 64 receivers, FP32-mixed.  Either every ray and hit equals rp_trace's, or the call
    returns RP_ERR_OVERFLOW because the fixed queue is too small, with rp_stats holding the
    queue records needed, the records it had room for and the rays and hits found."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_01780_gb300 import build

    build.build()
    import paper_1810_01780_gb300 as rp
    from paper_1810_01780_gb300 import _abi as A

    cfg = W.batched()
    assert cfg["rays"][0].shape[1] == 1 << 20
    med = rp.Medium(cfg["medium"])
    rays = rp.PreparedRays(*cfg["rays"], receivers=cfg["receivers"])
    prm = rp.make_params(cfg["params"], "fp32")
    ref = rp.TraceBuffers(int(5.5 * rays.n), 1 << 16)
    st_ref = rp.trace_into(med, rays, prm, ref)
    buf = rp.TraceBuffers(int(5.5 * rays.n), 1 << 16)
    st = A.Stats()
    rc = A.lib().rp_trace_static(med.handle, C.byref(rays.rays), C.byref(rays.rx), C.byref(prm),
                                 C.byref(buf.out), C.byref(buf.hits), C.byref(st),
                                 C.c_void_p(int(torch.cuda.current_stream().cuda_stream)))
    print("rp_trace_static at 2^20 primaries: rc %d, queue needed %d of %d, %d threads, stack "
          "depth %d; rays %d (rp_trace %d)" % (rc, st.queue_needed, st.queue_capacity, st.threads,
                                              st.stack_depth, st.rays, st_ref.rays))
    assert st.threads > 0 and st.stack_depth >= 1 and st.queue_capacity > 0
    if rc == A.RP_ERR_OVERFLOW:
        assert st.flags & 4 and st.queue_needed > st.queue_capacity
        assert st.rays >= rays.n and st.rays <= st_ref.rays
        return
    assert rc == A.RP_OK, A.last_error()
    assert st.rays == st_ref.rays and st.hits == st_ref.hits
    assert st.queue_needed <= st.queue_capacity
    n = int(st.rays)
    g = gpu_rays({"rays": {k: (v[:, :n] if v.dim() == 2 else v[:n]) for k, v in buf.t.items()}})
    r = gpu_rays({"rays": {k: (v[:, :n] if v.dim() == 2 else v[:n]) for k, v in ref.t.items()}})
    gi, oi, only_s, only_r = match(g, r)
    assert not only_s and not only_r
    for k in ("pos", "dir", "path", "time", "amp", "status", "n_acc", "n_rej"):
        np.testing.assert_array_equal(g[k][gi], r[k][oi], err_msg=k)
