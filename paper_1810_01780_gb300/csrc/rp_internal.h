// rp_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <mutex>
#include <utility>

#include "rp.h"
#include "trace_core.cuh"

#include <cuda_bf16.h>

struct rp_surrogate_s {
    int device;
    long long step;
    float *p, *m, *v, *grad;
    __nv_bfloat16 *pb;
    // training buffers for a batch of up to `cap` rows, per 128-row tile: gelu'(z) of the
    // pre-activations z0..z2 (BF16, tiled, 64 KB per tile), the activations H1..H4 and the
    // gradients g0..g3 as BF16 operand images (64 KB per tile; H[0] unused), and x and g4 as
    // 16-column images (4 KB per tile)
    long long cap;
    unsigned char *Z[3];
    unsigned char *H[5], *gl[4];
    unsigned char *ximg, *g4img;
    double *loss;
    void *pipe;  // buffers of the surrogate path-finding pipeline (pathfind.cu)
    // inference operands for the fused kernel (mlp_fused.cu), rebuilt when the weights change
    unsigned char *pack;
    unsigned char *pack_t;  // training: W1..W3 as the backward pass's B images (mlp_train_tc.cu)
    long long version, pack_version;
    int *fflag;  // set by a tensor-core kernel when a bounded wait gave up
    long long wait;  // SM cycles a tensor-core kernel waits on an mbarrier; 0: the default
    bool clean;      // the gradient and the batch loss are zero (as the fused Adam step leaves them)
};

struct rp_medium_s {
    int device;
    int kind;
    rpk::MediumSpheres layered;  // n_sph = 0: a plain layered medium
    rpk::MediumGrid grid;
    float4 *grid_dev;
    // non-horizontal boundaries (n_surf > 0: the medium is traced as rpk::MediumSurfaces)
    int n_surf;
    rpk::SurfB surf[RP_MAX_LAYERS];
    double *surf_dev;  // the height fields, one allocation
    float *surf_dev_f; // the same in FP32 (the FP32-mixed event tests)
};

// Which instantiation of the tracer a medium takes.
enum { VARIANT_LAYERED = 0, VARIANT_SPHERES = 1, VARIANT_SURFACES = 2, VARIANT_GRID = 3 };
inline int medium_variant(const rp_medium_s *m)
{
    if (m->kind != RP_MEDIUM_LAYERED) return VARIANT_GRID;
    if (m->layered.n_sph > 0) return VARIANT_SPHERES;
    return m->n_surf > 0 ? VARIANT_SURFACES : VARIANT_LAYERED;
}
inline rpk::MediumSurfaces surfaces_of(const rp_medium_s *m)
{
    rpk::MediumSurfaces s;
    static_cast<rpk::MediumLayered &>(s) = static_cast<const rpk::MediumLayered &>(m->layered);
    for (int k = 0; k < RP_MAX_LAYERS; ++k) s.B[k] = m->surf[k];
    return s;
}

namespace rph {

// thread-local last-error message
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define RP_CUDA_TRY(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return rph::cuda_fail(_e, #expr);  \
    } while (0)

// Launches k on st as a programmatic dependent launch: k may be scheduled while the kernel
// before it in the stream still runs, and must call tc::chain_wait_release() in every thread
// before it touches global memory that earlier work in the stream writes or reads.
template <typename... P, typename... A>
int launch_chained(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    RP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...));
    return RP_OK;
}

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

// Service-phase batching (see k_trace_wave): a warp services its waiting lanes once the idle
// lane-iterations summed since its last service reach this threshold.  An FP64 step costs far
// more than an FP32-mixed one against the same service phase, so FP64 lanes wait less.  Once a
// wave's input has run out, a thread hands the rest of its secondary stack to the next launch
// when at least kFlushMinDefault records remain below the one it takes.  rp_trace_params
// overrides both (0 keeps the default).  A lane whose ray has split kHotSplits times already
// is served at its next boundary without waiting for the threshold.
constexpr int kServiceIdleF32 = 256, kServiceIdleF64 = 8, kFlushMinDefault = 2;
constexpr int kHotSplits = 4;
constexpr int kBlockDefault = 128, kBlockMax = 256;

template <class P>
inline rpk::StepParams<P> step_params(const rp_trace_params *p, int axis, float dir)
{
    rpk::StepParams<P> sp;
    sp.tol = (typename P::R)p->tol;
    sp.inv_tol = (typename P::R)(1.0 / p->tol);
    sp.inv_tol2 = (typename P::R)std::min(1.0 / (p->tol * p->tol), 1e30);
    sp.h_min = (typename P::R)p->h_min;
    sp.h_max = (typename P::R)p->h_max;
    double eps = p->eps_b;
    if (P::kFF && eps < 2e-6) eps = 2e-6;
    sp.eps_b = (typename P::R)eps;
    sp.max_path = p->max_path;
    sp.max_time = p->max_time;
    sp.min_amp = p->min_amp;
    sp.mp = plane_const(p->max_path);
    sp.mt = plane_const(p->max_time);
    sp.use_max_time = p->max_time > 0.0;
    sp.use_min_amp = p->min_amp > 0.0;
    sp.rhs_form = p->rhs_form;
    sp.polarization = p->polarization;
    sp.max_generation = p->max_generation;
    sp.use_stop = p->use_stop;
    sp.stop_axis = axis;
    sp.stop_dir = dir;
    sp.max_steps = p->max_steps;
    sp.service_idle = (unsigned int)(p->service_idle > 0 ? p->service_idle
                                     : (P::kFF ? kServiceIdleF32 : kServiceIdleF64));
    sp.flush_min = p->flush_min > 0 ? p->flush_min : kFlushMinDefault;
    return sp;
}


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

// Operands of the fused kernels (built by mlp.cu, read by mlp_fused.cu and
// mlp_train_fused.cu): the hidden layers' weights W1..W3 as three BF16 B images of kPackW bytes
// (layout: bimg_off), then kPackF floats: W0 (3 x 256,
// BF16-rounded) at PF_W0, b0 at PF_B0, b1..b3 from PF_B1 (256 each), W4 (256 x 12,
// BF16-rounded) at PF_W4, b4 at PF_B4 (12, padded to 16).
constexpr long long kPackW = 256LL * 256 * 2;
// Byte offset of element (k, n) (K index k, N index n) in a 256 x 256 BF16 B image: the two
// halves of the N columns one after the other (64 KB each, so a CTA that computes one half
// copies it whole), each in the no-swizzle K-major layout of 8 x 8 core matrices of 128 bytes,
// core (k / 8, (n % 128) / 8) at ((k / 8) * 16 + (n % 128) / 8) * 128 (K-direction stride
// 2048 B, 8-column stride 128 B).
__host__ __device__ constexpr long long bimg_off(int k, int n)
{
    return (long long)(n >> 7) * 65536 + ((k >> 3) * 16 + ((n & 127) >> 3)) * 128 + (n & 7) * 16 +
           (k & 7) * 2;
}
constexpr int kPackF = 768 + 4 * 256 + 3072 + 16;
enum { PF_W0 = 0, PF_B0 = 768, PF_B1 = 1024, PF_W4 = 1792, PF_B4 = 4864 };
// Then the last layer's weights as two BF16 tensor-core images (8 KB each, outputs zero-padded
// from 12 to 16), for training: at kPackW4F the forward B image B[o][k] = W4[k][o] (K = 256
// hidden inputs, N = 16; core (k / 8, o / 8) at ((k / 8) * 2 + o / 8) * 128), at kPackW4B the
// backward one B[n][o] = W4[n][o] (K = 16, N = 256; core (o / 8, n / 8) at
// ((o / 8) * 32 + n / 8) * 128).
constexpr long long kPackW4F = 3 * kPackW + 4LL * kPackF;
constexpr long long kPackW4B = kPackW4F + 8192;
// Then the first layer's weights as a BF16 B image for training, B[n][k] = W0[k][n] (K = 3
// inputs zero-padded to 16, N = 256), half-major like the hidden layers' (4 KB per half; core
// (k / 8, (n % 128) / 8) at ((k / 8) * 16 + (n % 128) / 8) * 128 within its half).
constexpr long long kPackW0 = kPackW4B + 8192;
constexpr long long kPackBytes = kPackW0 + 8192;
static_assert(kPackW4F % 16 == 0, "bulk-copy alignment");
__host__ __device__ constexpr long long w4f_off(int k, int o)
{
    return ((k >> 3) * 2 + (o >> 3)) * 128 + (o & 7) * 16 + (k & 7) * 2;
}
__host__ __device__ constexpr long long w4b_off(int n, int o)
{
    return ((o >> 3) * 32 + (n >> 3)) * 128 + (n & 7) * 16 + (o & 7) * 2;
}
__host__ __device__ constexpr long long w0_off(int k, int n)
{
    return (long long)(n >> 7) * 4096 + ((k >> 3) * 16 + ((n & 127) >> 3)) * 128 + (n & 7) * 16 +
           (k & 7) * 2;
}

// Surrogate network (mlp.cu) and its path-finding pipeline buffers (pathfind.cu).
int ensure_acts(rp_surrogate_s *s, long long n);
void free_pipe(rp_surrogate_s *s);
int ensure_pack(rp_surrogate_s *s, cudaStream_t st);
int forward_fused(rp_surrogate_s *s, long long n, const float *x, float *out, cudaStream_t st);
int fused_status(rp_surrogate_s *s, cudaStream_t st);  // syncs st; RP_ERR_TIMEOUT if flagged
// training on the tensor cores: the fused forward pass with the loss and the last layer's
// backward data pass, and the hidden layers' backward data chain (mlp_train_fused.cu; they add
// the bias gradients to db0..db4); the weight gradients of all five layers (mlp_train_tc.cu)
int train_fwd(rp_surrogate_s *s, long long n, const float *x, const float *y, const float *t,
              float *db3, float *db4, cudaStream_t st);
int train_bwd(rp_surrogate_s *s, long long n, float *db2, float *db1, float *db0, cudaStream_t st);
int tc_pack_backward(const float *p, unsigned char *img, long long w1, long long w2, long long w3,
                     cudaStream_t st);
// One weight-gradient product D = A^T B over the rows of a batch (k_tc_wgrad): A the operand
// images of a layer's 256 input columns (M, two halves), B those of its N output columns (256,
// or 16 for the thin layers' zero-padded images), D added to dW as `out` says.
enum { WG_OUT_SQUARE = 0, WG_OUT_LAST = 1, WG_OUT_FIRST_T = 2 };
struct WgradJob {
    const unsigned char *A, *B;
    float *dW;
    int32_t n;       // N: 256 or 16
    int32_t out;     // WG_OUT_SQUARE: dW[m * 256 + c]; WG_OUT_LAST: dW[m * 12 + c] (c < 12);
                     // WG_OUT_FIRST_T: dW[c * 256 + m] (c < 3, the first layer's W0 transposed)
    int32_t shares;  // CTAs that split this job's tiles among them
    int32_t pad;
};
struct WgradArgs {
    WgradJob job[5];  // the hidden layers 1..3, the last layer, the first layer (transposed)
};
// Launches the five jobs of `a` (their shares filled in here) over n rows.
int tc_wgrad(WgradArgs &a, long long n, int *flag, long long wait, cudaStream_t st);
// the mbarrier wait limit of the surrogate's tensor-core kernels [SM cycles]
long long wait_cycles(const rp_surrogate_s *s);
int run_surrogate_paths(rp_surrogate_s *s, rp_medium_t m, int64_t n, const double *zs,
                        const double *zr, const double *dist, const int32_t *n_angles,
                        const rp_path_params *p, const rp_surrogate_params *sp,
                        rp_solutions *sol, rp_surrogate_stats *stats, cudaStream_t st);
int run_surrogate_encode(int64_t n, const double *zs, const double *zr, const double *dist,
                         const rp_solutions *sol, int max_sol, float *x, float *y, float *t,
                         cudaStream_t st);

// Grid gradient precompute (medium.cu).
int build_grid(rp_medium_s *m, const float *n_src, double spacing, cudaStream_t st);

}  // namespace rph
