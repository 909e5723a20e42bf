// trace_static.cu -- rp_trace_static: rp_trace without any device allocation.
//
// Some callers cannot allocate device memory at the time they trace: a process whose memory
// is entirely owned by another allocator (a framework's caching pool that has reserved the
// device), a service that forbids allocation after start-up because cudaMalloc / cudaFree
// can synchronise the whole device and stall every stream, or a tool that must run inside a
// fixed memory budget.  For them this entry point takes its scratch space (control block,
// receiver grid, per-thread secondary stacks, overflow queue) from one statically sized
// device array that the library carries from load time.
#include <cstring>
#include <mutex>

#include "rp_internal.h"

namespace {

// The scratch array.  In host code `g_rp_static_scratch` only names a host-side stand-in of
// the symbol, never the device memory: its device address is obtained with
// cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) unsigned char g_rp_static_scratch[RP_STATIC_SCRATCH_BYTES];

struct StaticSlot {
    std::mutex mu;    // serialises the calls that share the array on this device
    void *ptr = nullptr;
};

StaticSlot g_slots[64];
std::mutex g_setup_mu;

}  // namespace

using namespace rph;

extern "C" int rp_trace_static(rp_medium_t m, const rp_rays *in, const rp_receivers *rx,
                               const rp_trace_params *p, rp_ray_out *out, rp_hits *hits,
                               rp_stats *stats, void *stream)
{
    if (stats) memset(stats, 0, sizeof *stats);
    try {
        if (!in) {
            set_error("rp_trace_static: null rays");
            return RP_ERR_INVALID_ARG;
        }
        if (in->n > RP_STATIC_MAX_RAYS) {
            set_error("rp_trace_static: %lld primaries exceed the limit of %d of the fixed scratch",
                      (long long)in->n, RP_STATIC_MAX_RAYS);
            return RP_ERR_INVALID_ARG;
        }
        if (rx && rx->n > RP_STATIC_MAX_RECEIVERS) {
            set_error("rp_trace_static: %d receivers exceed the limit of %d of the fixed scratch",
                      rx->n, RP_STATIC_MAX_RECEIVERS);
            return RP_ERR_INVALID_ARG;
        }
        int dev;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "rp_trace_static: cudaGetDevice");
        if (dev < 0 || dev >= 64) {
            set_error("rp_trace_static: device index %d out of range", dev);
            return RP_ERR_INVALID_ARG;
        }
        StaticSlot &slot = g_slots[dev];
        {
            // first call on this device: resolve the array's device address (no allocation)
            std::lock_guard<std::mutex> lock(g_setup_mu);
            if (!slot.ptr) {
                void *ptr = nullptr;
                e = cudaGetSymbolAddress(&ptr, g_rp_static_scratch);
                if (e != cudaSuccess) return cuda_fail(e, "rp_trace_static: cudaGetSymbolAddress");
                slot.ptr = ptr;
            }
        }
        FixedScratch fs;
        fs.ptr = slot.ptr;
        fs.size = RP_STATIC_SCRATCH_BYTES;
        fs.mu = &slot.mu;
        return run_trace(m, in, rx, p, out, hits, stats, (cudaStream_t)stream, &fs);
    } catch (...) {
        set_error("rp_trace_static: internal exception");
        return RP_ERR_CUDA;
    }
}
