// rp_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "rp.h"
#include "trace_core.cuh"

struct rp_medium_s {
    int device;
    int kind;
    rpk::MediumLayered layered;
    rpk::MediumGrid grid;
    float4 *grid_dev;
};

namespace rph {

// thread-local last-error message
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define RP_CUDA_TRY(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return rph::cuda_fail(_e, #expr);  \
    } while (0)

// Grow-only device workspace, one per device; the lock serialises calls on that device.
struct Workspace {
    std::mutex mu;
    void *ptr = nullptr;
    size_t size = 0;
    void *host_ctrl = nullptr;  // pinned copy of the control block
    void *host_clock = nullptr; // pinned copy of the per-warp clocks
    size_t host_clock_size = 0;
};
Workspace &workspace(int device);
int ensure_workspace(Workspace &w, size_t bytes);
int ensure_host_clock(Workspace &w, size_t bytes);

int sm_count(int device);

// Splits a double into the float-float pair used by the FP32 path.
inline rpk::PlaneC plane_const(double d)
{
    rpk::PlaneC c;
    c.d = d;
    c.hi = (float)d;
    c.lo = (float)(d - (double)c.hi);
    return c;
}

int validate_params(const rp_trace_params *p, bool path_finding);

// A caller-provided device scratch region used instead of the grow-only workspace.
struct FixedScratch {
    void *ptr;
    size_t size;
    std::mutex *mu;  // serialises the calls that share the region
};

// Tracing driver (trace.cu).  fs == nullptr: the grow-only workspace of the device.
int run_trace(rp_medium_t m, const rp_rays *in, const rp_receivers *rx, const rp_trace_params *p,
              rp_ray_out *out, rp_hits *hits, rp_stats *stats, cudaStream_t st,
              const FixedScratch *fs = nullptr);

// Path-finding driver (pathfind.cu).
int run_find_paths(rp_medium_t m, int64_t n_pairs, const double *zs, const double *zr,
                   const double *dist, const int32_t *n_angles, const rp_path_params *p,
                   rp_solutions *sol, rp_stats *stats, cudaStream_t st);

// Grid gradient precompute (medium.cu).
int build_grid(rp_medium_s *m, const float *n_src, double spacing, cudaStream_t st);

}  // namespace rph
