// trace.cu -- persistent tracing launches (rp_trace).
//
// Every thread of a launch claims rays from a global counter (warp-aggregated atomics),
// traces its ray with the lane state machine of trace_core.cuh and claims the next one as soon
// as it finishes, so rays with very different step counts keep all lanes busy.  Secondaries
// cast at boundaries (Sec. 2, boundary module) go on the thread's own stack and are traced by
// the same thread, depth first, before it claims new input.  Once the launch's input has run
// out, new secondaries and the rest of a thread's stack go to a device work queue instead; the
// queue segment written by launch w is the input of launch w + 1.  Every queued record is at
// least one generation younger than the launch that wrote it, so max_generation + 1 launches
// on one stream trace everything, and no launch ever waits for work that another thread has
// still to produce: there are no spin waits anywhere.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rp_internal.h"

namespace cg = cooperative_groups;
using namespace rpk;

namespace rph {

struct WaveIn {
    const double *pos, *dir, *amp;
    long long n;
    PlaneC stop;
    double h0;
    float h0f;
    const uint32_t *ord;  // primary taken up k-th: ray ord[k] (null: ray k)
};

// Coherent order of the primaries (rp_trace_params.ray_order == RP_ORDER_COHERENT): a counting
// sort on a 16-bit key, the launch direction's z component in 256 bins over [-1, 1] (high
// bits) and the start depth in 256 bins over the batch's range (low bits).  Rays that start
// near one another in nearly the same direction follow similar paths -- the same boundaries,
// the same step sizes -- so the lanes of a warp that take them up together stay in step
// (coarser bins leave more spread within a warp; a full sort on direction and depth lines up
// rays of equal direction but scattered depths).  A batch with a single start depth gives all
// 16 bits to the direction.  Four launches: the depth range, the keys
// with their histogram, its exclusive scan (two launches), the scatter (within a key the
// order follows the atomics; no record depends on it).
constexpr int kOrderAxis = 256, kOrderBins = kOrderAxis * kOrderAxis;
__device__ __forceinline__ uint32_t ordered_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__global__ void k_order_range(const double *__restrict__ z, long long n, uint32_t *range)
{
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float f = (float)z[i];
        if (isfinite(f)) {
            const uint32_t u = ordered_bits(f);
            lo = min(lo, u);
            hi = max(hi, u);
        }
    }
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
}
__global__ void k_order_keys(const double *__restrict__ pos, const double *__restrict__ dir,
                             long long n, const uint32_t *range, uint16_t *key, uint32_t *hist)
{
    const float z0 = range[1] >= range[0] ? from_ordered_bits(range[0]) : 0.0f;
    const float z1 = range[1] >= range[0] ? from_ordered_bits(range[1]) : 0.0f;
    // no depth spread (one start depth): all 16 bits of the key for the direction
    const bool flat = !(z1 > z0);
    const float half = 0.5f * (float)(flat ? kOrderBins : kOrderAxis);
    const float scale = flat ? 0.0f : (float)kOrderAxis / (z1 - z0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float dx = (float)dir[i], dy = (float)dir[n + i], dz = (float)dir[2 * n + i];
        const float q = dx * dx + dy * dy + dz * dz;
        const float tz = q > 0.0f ? dz * rsqrtf(q) : 0.0f;
        const float ft = (tz + 1.0f) * half, fz = ((float)pos[2 * n + i] - z0) * scale;
        const int zb = fz >= 0.0f ? min(kOrderAxis - 1, (int)fz) : 0;  // NaN -> bin 0
        const uint32_t k = flat ? (uint32_t)(ft >= 0.0f ? min(kOrderBins - 1, (int)ft) : 0)
                                : (uint32_t)((ft >= 0.0f ? min(kOrderAxis - 1, (int)ft) : 0) *
                                                 kOrderAxis + zb);
        key[i] = (uint16_t)k;
        atomicAdd(&hist[k], 1u);
    }
}
// Exclusive scan of the histogram in place, in two launches of kOrderBins / 1024 blocks: each
// block scans its 1,024 bins (one per thread) and leaves its total in sums[block]; then each
// block adds the totals of the blocks before it.
constexpr int kOrderScanBlocks = kOrderBins / 1024;
__global__ void __launch_bounds__(1024) k_order_scan(uint32_t *hist, uint32_t *sums)
{
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x, i = blockIdx.x * 1024 + t;
    const uint32_t v = hist[i];
    part[t] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan
        const uint32_t add = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    hist[i] = part[t] - v;
    if (t == 1023) sums[blockIdx.x] = part[1023];
}
__global__ void __launch_bounds__(1024) k_order_offsets(uint32_t *hist, const uint32_t *sums)
{
    __shared__ uint32_t before;
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int b = 0; b < (int)blockIdx.x; ++b) s += sums[b];
        before = s;
    }
    __syncthreads();
    hist[blockIdx.x * 1024 + threadIdx.x] += before;
}
__global__ void k_order_scatter(const uint16_t *__restrict__ key, long long n, uint32_t *cursor,
                                uint32_t *ord)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        ord[atomicAdd(&cursor[key[i]], 1u)] = (uint32_t)i;
}

__device__ __forceinline__ long long claim_index(unsigned long long *counter)
{
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    return (long long)(base + g.thread_rank());
}

template <class P, class M>
__device__ __forceinline__ void lane_reset(Lane<P> &L, const M &med, const StepParams<P> &sp,
                                           const PlaneC &stop)
{
    load_layer<P>(L.lc, med, L.layer);
    L.mode = MODE_NORMAL;
    L.ev = EV_NONE;
    L.side = 0;
    L.it = 0;
    L.n_acc = L.n_rej = L.n_root = L.n_refl = L.n_turn = L.root_fail = 0;
    L.status = RP_ST_ALIVE;
    L.pend = 0;
    L.stop = stop;
    L.stop_axis = sp.stop_axis;
    L.mp = sp.mp;
    init_stop(L, sp);
    set_trial(L, sp);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Starts fetching the inputs of ray k (claimed ahead of time) into L1.
__device__ __forceinline__ void prefetch_ray(const Sinks &sk, const WaveIn &in, int wave,
                                             unsigned long long base, long long k)
{
    if (wave == 0) {
        const long long n = in.n;
        if (in.ord) k = (long long)__ldg(&in.ord[k]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            prefetch_l1(&in.pos[a * n + k]);
            prefetch_l1(&in.dir[a * n + k]);
        }
        if (in.amp) prefetch_l1(&in.amp[k]);
    } else {
        const char *q = (const char *)&sk.queue[base + k];
        prefetch_l1(q);
        prefetch_l1(q + sizeof(QRec) - 1);
    }
}

// Copies a queued record (a secondary cast at a boundary, or a finished record to write out)
// into the lane; the lane's per-ray state is reset by the caller.
template <class P>
__device__ __forceinline__ void load_record(Lane<P> &L, const QRec &Q)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P::set(L.r, a, Q.r[a]);
        P::set(L.t, a, Q.t[a]);
    }
    L.A = Q.A;
    L.A0 = Q.A0;
    P::sset(L.T, Q.T);
    P::sset(L.s, Q.s);
    L.h = P::from_d(Q.h);
    L.id = Q.id;
    L.parent = Q.parent;
    L.gen = Q.gen;
    L.seq = Q.seq;
    L.layer = Q.layer;
    L.status = Q.status;  // RP_ST_ALIVE, or a record that only has to be written out
}

// Fills the lane with primary k of the input.  Sets L.status to RP_ST_ALIVE, or to
// RP_ST_BAD_INPUT (and the launch's flag) for a non-finite position or a zero, non-finite
// direction; such a ray is written out as it is.
template <class P, class M>
__device__ __forceinline__ void load_primary(Lane<P> &L, const M &med, const Sinks &sk,
                                             const WaveIn &in, long long k)
{
    const long long n = in.n;
    if (in.ord) k = (long long)__ldg(&in.ord[k]);  // the ray taken up k-th
    L.A = in.amp ? in.amp[k] : 1.0;
    L.A0 = L.A;
    L.id = k;
    L.parent = -1;
    L.gen = 0;
    L.seq = 0;
    L.status = RP_ST_ALIVE;
    if constexpr (P::kFF) {
        // FP32-mixed: every conversion on the integer/FP32 pipes
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            P::set(L.r, a, in.pos[a * n + k]);
            P::set(L.t, a, in.dir[a * n + k]);
        }
        L.T.hi = L.T.lo = 0.0f;
        L.s.hi = L.s.lo = 0.0f;
        L.h = in.h0f;
        if constexpr (has_spheres_v<M>) {
            const double r0[3] = {in.pos[k], in.pos[n + k], in.pos[2 * n + k]};
            L.layer = region_of(med, r0);
        } else if constexpr (has_surfaces_v<M>) {
            const double r0[3] = {in.pos[k], in.pos[n + k], in.pos[2 * n + k]};
            L.layer = layer_at(med, r0);
        } else if constexpr (is_layered_v<M>) {
            L.layer = layer_of_ff(med, L.r.hi[2], L.r.lo[2]);
        } else {
            L.layer = 0;
        }
        const float q2 = L.t.hi[0] * L.t.hi[0] + L.t.hi[1] * L.t.hi[1] + L.t.hi[2] * L.t.hi[2];
        const bool pos_ok = isfinite(L.r.hi[0]) && isfinite(L.r.hi[1]) && isfinite(L.r.hi[2]);
        if (!(q2 > 0.0f) || !isfinite(q2) || !pos_ok) {
            L.status = RP_ST_BAD_INPUT;
            atomicOr(&sk.ctrl->flags, (unsigned)FLAG_BAD_INPUT);
            return;
        }
        if (fabsf(q2 - 1.0f) > 1e-5f) {
            // far from unit: a coarse FP64 normalisation first (rare)
            double t[3] = {in.dir[k], in.dir[n + k], in.dir[2 * n + k]};
            const double q = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) P::set(L.t, a, t[a] / q);
        }
        ff_renormalise(L.t);  // exact unit length in float-float
    } else {
        double r[3], t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r[a] = in.pos[a * n + k];
            t[a] = in.dir[a * n + k];
        }
        P::sset(L.T, 0.0);
        P::sset(L.s, 0.0);
        L.h = P::from_d(in.h0);
        if constexpr (has_spheres_v<M>)
            L.layer = region_of(med, r);
        else if constexpr (has_surfaces_v<M>)
            L.layer = layer_at(med, r);
        else if constexpr (is_layered_v<M>)
            L.layer = layer_of(med, r[2]);
        else
            L.layer = 0;
        const double q2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        const bool pos_ok = isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) P::set(L.r, a, r[a]);
        if (!(q2 > 0.0) || !isfinite(q2) || !pos_ok) {
#pragma unroll
            for (int a = 0; a < 3; ++a) P::set(L.t, a, t[a]);
            L.status = RP_ST_BAD_INPUT;
            atomicOr(&sk.ctrl->flags, (unsigned)FLAG_BAD_INPUT);
            return;
        }
        // normalised as the FP64 reference does
        const double q = sqrt(q2);
#pragma unroll
        for (int a = 0; a < 3; ++a) P::set(L.t, a, t[a] / q);
    }
}

// Moves m records of a thread's stack to the global queue, which the next launch drains with
// all its threads; false (nothing moved) when the queue has no room for them.  The room is
// reserved with a bounded compare-and-swap loop: each failed attempt means another thread's
// reservation succeeded, and after 64 the records simply stay on the stack.
__device__ __forceinline__ bool flush_to_queue(const Sinks &sk, const QRec *src, int m)
{
    unsigned long long cur = *(volatile unsigned long long *)&sk.ctrl->q_tail, q = 0;
    bool ok = false;
    for (int attempt = 0; attempt < 64 && cur + (unsigned long long)m <= sk.q_cap; ++attempt) {
        const unsigned long long old = atomicCAS(&sk.ctrl->q_tail, cur, cur + (unsigned long long)m);
        if (old == cur) {
            q = cur;
            ok = true;
            break;
        }
        cur = old;
    }
    if (!ok) return false;
    static_assert(sizeof(QRec) % sizeof(long long) == 0, "QRec copies by 8-byte words");
    constexpr int kWords = (int)(sizeof(QRec) / sizeof(long long));
    const long long *from = (const long long *)src;
    long long *to = (long long *)&sk.queue[q];
    for (int w = 0; w < m * kWords; ++w) to[w] = from[w];
    return true;
}

enum { NEXT_NONE = 0, NEXT_TRACE = 1, NEXT_RECORD = 2 };

// Next ray of this wave for the calling lane: NEXT_TRACE, NEXT_RECORD (a finished record to
// write out: a ray refracted into air, or an invalid input) or NEXT_NONE when the wave's
// input is exhausted.  `ahead` holds a ray index claimed one ray in advance, so that the
// claim's atomic and the input loads overlap the tracing of the current ray.
template <class P, class M>
__device__ int next_ray(Lane<P> &L, const M &med, const StepParams<P> &sp, const Sinks &sk,
                        const WaveIn &in, int wave, unsigned long long base,
                        unsigned long long count, long long &ahead)
{
    // the wave's input has run out once the shared claim counter has passed its end (this
    // thread's own look-ahead claim can be old: a thread working through its stack claims
    // nothing)
    bool input_out = ahead >= (long long)count;
    if (!input_out)
        input_out = *(volatile const unsigned long long *)&sk.ctrl->claim[wave] >= count;
    // once the input has run out, a ray this lane claimed but has not started (nobody else can
    // take it) starts now, and the lane's stack goes to the next launch: taken depth first, the
    // stack would hold the claimed ray back and make it the launch's last
    if (L.stk > 0 && input_out && ahead < (long long)count &&
        flush_to_queue(sk, thread_stack(sk), L.stk))
        L.stk = 0;
    if (L.stk > 0) {
        // depth first: the secondaries this thread cast itself come before new input
        const int top = --L.stk;
        const QRec *stk = thread_stack(sk);
        // once the input has run out, the rest of the stack (at least sp.flush_min records)
        // goes to the next launch, where all threads share it: a primary that cast many
        // secondaries would otherwise keep this one thread busy for all of them while the
        // others idle
        if (top >= sp.flush_min && input_out && flush_to_queue(sk, stk, top)) L.stk = 0;
        load_record<P>(L, stk[top]);
    } else {
        const long long k = ahead;
        if (k >= (long long)count) return NEXT_NONE;
        ahead = claim_index(&sk.ctrl->claim[wave]);
        if (ahead < (long long)count) prefetch_ray(sk, in, wave, base, ahead);
        if (wave != 0)
            load_record<P>(L, sk.queue[base + k]);
        else
            load_primary<P, M>(L, med, sk, in, k);
    }
    const int32_t st = L.status;
    lane_reset<P, M>(L, med, sp, in.stop);
    L.status = st;
    L.tail = input_out || ahead >= (long long)count;
    return st == RP_ST_ALIVE ? NEXT_TRACE : NEXT_RECORD;
}

// Launched with any block of up to kBlockMax threads (a multiple of 32); the bounds keep the
// register budget of P::kMinBlocks blocks of 128 threads per SM.
template <class P, class M>
__global__ void __launch_bounds__(kBlockMax, P::kMinBlocks * 128 / kBlockMax) k_trace_wave(const M med, const StepParams<P> sp,
                                                    const Sinks sk, const WaveIn in, int wave)
{
    unsigned long long base = 0, count;
    if (wave == 0) {
        count = (unsigned long long)in.n;
    } else {
        base = sk.ctrl->seg_begin[wave];
        count = sk.ctrl->seg_end[wave] - base;
    }
    const unsigned long long t_start = global_ns();
    Lane<P> L;
    L.stk = 0;
    unsigned int acc = 0, rej = 0, root = 0;
    long long ahead = claim_index(&sk.ctrl->claim[wave]);
    // fetch: the lane wants its next ray (its first one comes from the first service phase,
    // so that next_ray is inlined once)
    bool active = false, done = false, fetch = true;
    unsigned int idle = 0;  // waiting lane-iterations since the last service phase
    // Warp-synchronous loop.  Every iteration runs one Runge-Kutta step on each lane whose
    // ray is stepping.  The rare, long code paths -- a boundary split with its secondary,
    // writing a finished ray and loading the next one -- are parked and serviced together:
    // once the lane-iterations spent waiting since the last service reach sp.service_idle
    // (many waiting lanes are served soon, a single one waits longer), when no lane can step,
    // or at once for a ray bouncing in a duct; so they run seldom, with many lanes at once,
    // and stay out of the hot loop's instruction working set.
    while (__any_sync(0xffffffffu, active || done || fetch)) {
        __syncwarp();
        const bool stepping = active && L.pend == 0;
        if (stepping && advance<P, M>(med, L, sp, sk)) {
            active = false;
            done = true;
        }
        const bool waits = done || fetch || (active && L.pend != 0);
        const unsigned int wait = __ballot_sync(0xffffffffu, waits);
        const unsigned int step_mask = __ballot_sync(0xffffffffu, active && L.pend == 0);
        // a ray that has already split kHotSplits times is bouncing in a duct: it reaches the
        // next boundary within a few steps, and made to wait for the batch at every bounce it
        // would outlast the launch
        const bool hot = __any_sync(0xffffffffu, active && L.pend != 0 && L.n_refl >= kHotSplits);
        idle += (unsigned int)__popc(wait);
        if (wait != 0u && (idle >= sp.service_idle || step_mask == 0u || hot)) {
            idle = 0;
            if (active && L.pend != 0 && finish_split<P>(med, L, sp, sk)) {
                active = false;
                done = true;
            }
            while (done || fetch) {
                if (done) {
                    acc += (unsigned int)L.n_acc;
                    rej += (unsigned int)L.n_rej;
                    root += (unsigned int)L.n_root;
                    write_ray<P>(sk.out, L.id, L, sk.ctrl);
                }
                const int nx = next_ray<P, M>(L, med, sp, sk, in, wave, base, count, ahead);
                fetch = false;
                active = nx == NEXT_TRACE;
                done = nx == NEXT_RECORD;
            }
        }
    }
    // per-warp totals; no block-wide barrier, so finished warps simply retire
    acc = __reduce_add_sync(0xffffffffu, acc);
    rej = __reduce_add_sync(0xffffffffu, rej);
    root = __reduce_add_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0) {
        if (wave == 0) {
            const size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
            sk.warp_clock[2 * w] = t_start;
            sk.warp_clock[2 * w + 1] = global_ns();
        }
        atomicAdd(&sk.ctrl->steps_acc, (unsigned long long)acc);
        atomicAdd(&sk.ctrl->steps_rej, (unsigned long long)rej);
        atomicAdd(&sk.ctrl->steps_root, (unsigned long long)root);
    }
}

__global__ void k_init_ctrl(Ctrl *ctrl, long long n)
{
    ctrl->out_count = (unsigned long long)n;
}

// Input segment of wave w: the queue records written by wave w - 1.
__global__ void k_prep_wave(Ctrl *ctrl, int w, unsigned long long q_cap)
{
    const unsigned long long tail = ctrl->q_tail < q_cap ? ctrl->q_tail : q_cap;
    ctrl->seg_begin[w] = (w == 1) ? 0ull : ctrl->seg_end[w - 1];
    ctrl->seg_end[w] = tail;
}

// Resident blocks per SM of k_trace_wave<P, M> at `block` threads (cached per block size),
// capped at `want` when 0 < want.
template <class P, class M>
static int occupancy_grid(int block, int want)
{
    static int cached[kBlockMax / 32 + 1] = {0};
    const int slot = block / 32;
    int occ = cached[slot];
    if (occ == 0) {
        RP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_wave<P, M>,
                                                                  block, 0));
        occ = occ > 0 ? occ : 1;
        cached[slot] = occ;
    }
    return (want > 0 && want < occ) ? want : occ;
}

static int trace_blocks(int variant, int precision, int block, int want)
{
    const bool f64 = precision == RP_FP64;
    switch (variant) {
    case VARIANT_SPHERES:
        return f64 ? occupancy_grid<PrecF64, MediumSpheres>(block, want)
                   : occupancy_grid<PrecF32, MediumSpheres>(block, want);
    case VARIANT_SURFACES:
        return f64 ? occupancy_grid<PrecF64, MediumSurfaces>(block, want)
                   : occupancy_grid<PrecF32, MediumSurfaces>(block, want);
    case VARIANT_LAYERED:
        return f64 ? occupancy_grid<PrecF64, MediumLayered>(block, want)
                   : occupancy_grid<PrecF32, MediumLayered>(block, want);
    default:
        return f64 ? occupancy_grid<PrecF64, MediumGrid>(block, want)
                   : occupancy_grid<PrecF32, MediumGrid>(block, want);
    }
}

template <class P, class M>
static int launch_waves(const M &med, const StepParams<P> &sp, const Sinks &sk, const WaveIn &in,
                        int n_waves, int grid, int block, cudaStream_t st, cudaEvent_t *ev)
{
    for (int w = 0; w < n_waves; ++w) {
        if (w > 0) k_prep_wave<<<1, 1, 0, st>>>(sk.ctrl, w, sk.q_cap);
        k_trace_wave<P, M><<<grid, block, 0, st>>>(med, sp, sk, in, w);
        RP_CUDA_TRY(cudaEventRecord(ev[w + 1], st));
    }
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

// Stop plane stop_n . r = stop_d with stop_n = +/- a coordinate axis.
int stop_axis_of(const rp_trace_params *p, int *axis, float *dir, double *offset)
{
    *axis = 0;
    *dir = 1.0f;
    *offset = 0.0;
    if (!p->use_stop) return RP_OK;
    int nz = 0;
    for (int a = 0; a < 3; ++a) {
        if (p->stop_n[a] == 0.0) continue;
        if (p->stop_n[a] != 1.0 && p->stop_n[a] != -1.0) nz = 9;
        *axis = a;
        *dir = (float)p->stop_n[a];
        ++nz;
    }
    if (nz != 1) {
        set_error("stop plane normal must be +/- a coordinate axis");
        return RP_ERR_INVALID_ARG;
    }
    *offset = p->stop_d * (double)*dir;  // the plane is r[axis] = dir * stop_d
    return RP_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// A receiver set binned into a uniform grid of cells (Receivers in trace_core.cuh), with the
// receivers and the h_max it was built for.
struct RxGrid {
    bool valid = false;
    long long version = 0;  // bumped by every rebuild
    double h_max = 0.0;
    std::vector<double> c, rad;
    std::vector<SphereC> spheres;
    std::vector<int2> cells;  // per cell: [first, last) in items
    std::vector<int> items;   // receiver indices, ascending within a cell
    float org[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, inv = 1.0f;
    int dims[3] = {1, 1, 1};
    // device copies (spheres, cells, items), one per device, current while version matches
    struct DevCopy {
        char *ptr = nullptr;
        size_t bytes = 0;
        long long version = -1;
    };
    static constexpr int kDevices = 16;
    DevCopy dev[kDevices];
};

// The device copy of grid g on device `d` (uploaded on `st` when the grid was rebuilt since):
// spheres at *ps, cells at *pz, items at *pb.  No kernel of an earlier call can still read a
// copy being replaced, as every call drains its stream before it returns.
static int rx_device_copy(RxGrid &g, int d, cudaStream_t st, const char **ps, const char **pz,
                          const char **pb)
{
    const size_t o_z = align_up(sizeof(SphereC) * g.spheres.size());
    const size_t o_b = o_z + align_up(sizeof(int2) * g.cells.size());
    const size_t bytes = o_b + align_up(sizeof(int) * std::max<size_t>(g.items.size(), 1));
    RxGrid::DevCopy &c = g.dev[d];
    if (c.version != g.version) {
        if (c.bytes < bytes) {
            if (c.ptr) cudaFree(c.ptr);
            c.ptr = nullptr;
            c.bytes = 0;
            RP_CUDA_TRY(cudaMalloc(&c.ptr, bytes));
            c.bytes = bytes;
        }
        RP_CUDA_TRY(cudaMemcpyAsync(c.ptr, g.spheres.data(), sizeof(SphereC) * g.spheres.size(),
                                    cudaMemcpyHostToDevice, st));
        RP_CUDA_TRY(cudaMemcpyAsync(c.ptr + o_z, g.cells.data(), sizeof(int2) * g.cells.size(),
                                    cudaMemcpyHostToDevice, st));
        if (!g.items.empty())
            RP_CUDA_TRY(cudaMemcpyAsync(c.ptr + o_b, g.items.data(), sizeof(int) * g.items.size(),
                                        cudaMemcpyHostToDevice, st));
        c.version = g.version;
    }
    *ps = c.ptr;
    *pz = c.ptr + o_z;
    *pb = c.ptr + o_b;
    return RP_OK;
}

// Bins receivers (centres c, 3 per receiver; radii rad) for steps of at most h_max: each
// sphere is listed in every cell that its centre box, inflated by R + h_max / 2 and a rounding
// pad, overlaps; cells are at least twice the inflation wide, so a sphere meets at most two
// cells per axis.  A counting sort over the cells keeps each cell's receivers in ascending
// order.
static int bin_receivers(const std::vector<double> &c, const std::vector<double> &rad,
                         double h_max, RxGrid &g)
{
    const int n_rx = (int)rad.size();
    g.spheres.assign(n_rx, SphereC{});
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, r_max = 0.0;
    for (int j = 0; j < n_rx; ++j) {
        if (!(rad[j] > 0.0)) {
            set_error("rp_trace: receiver radius must be > 0");
            return RP_ERR_INVALID_ARG;
        }
        for (int a = 0; a < 3; ++a) {
            g.spheres[j].c[a] = plane_const(c[3 * j + a]);
            lo[a] = std::min(lo[a], c[3 * j + a]);
            hi[a] = std::max(hi[a], c[3 * j + a]);
        }
        g.spheres[j].R = rad[j];
        g.spheres[j].Rf = (float)rad[j];
        g.spheres[j].idx = j;
        r_max = std::max(r_max, rad[j]);
    }
    // inflation: radius + half the longest chord + a pad far above FP32 rounding
    double amax = 0.0;
    for (int a = 0; a < 3; ++a) amax = std::max(amax, std::max(std::fabs(lo[a]), std::fabs(hi[a])));
    const double infl = r_max + 0.5 * h_max + 1e-2 + 1e-6 * amax;
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        lo[a] -= infl;
        hi[a] += infl;
        ext = std::max(ext, hi[a] - lo[a]);
    }
    const double cell = std::max(2.0 * infl, ext / 64.0);
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = std::max(1, std::min(64, (int)std::ceil((hi[a] - lo[a]) / cell)));
        g.org[a] = (float)lo[a];
        g.hi[a] = (float)(lo[a] + cell * g.dims[a]);
    }
    g.inv = (float)(1.0 / cell);
    const size_t n_cells = (size_t)g.dims[0] * g.dims[1] * g.dims[2];
    // the cells a receiver's box spans, in (z, y, x) order
    auto span = [&](int j, int (&i0)[3], int (&i1)[3]) {
        for (int a = 0; a < 3; ++a) {
            i0[a] = std::max(0, (int)std::floor((c[3 * j + a] - infl - lo[a]) / cell));
            i1[a] = std::min(g.dims[a] - 1, (int)std::floor((c[3 * j + a] + infl - lo[a]) / cell));
        }
    };
    auto cell_of = [&](int x, int y, int z) { return ((size_t)z * g.dims[1] + y) * g.dims[0] + x; };
    std::vector<int> start(n_cells + 1, 0);
    for (int j = 0; j < n_rx; ++j) {
        int i0[3], i1[3];
        span(j, i0, i1);
        for (int z = i0[2]; z <= i1[2]; ++z)
            for (int y = i0[1]; y <= i1[1]; ++y)
                for (int x = i0[0]; x <= i1[0]; ++x) ++start[cell_of(x, y, z) + 1];
    }
    for (size_t q = 0; q < n_cells; ++q) start[q + 1] += start[q];
    g.cells.resize(n_cells);
    for (size_t q = 0; q < n_cells; ++q) g.cells[q] = make_int2(start[q], start[q + 1]);
    g.items.assign((size_t)start[n_cells], 0);
    for (int j = 0; j < n_rx; ++j) {  // ascending j: each cell's list in receiver order
        int i0[3], i1[3];
        span(j, i0, i1);
        for (int z = i0[2]; z <= i1[2]; ++z)
            for (int y = i0[1]; y <= i1[1]; ++y)
                for (int x = i0[0]; x <= i1[0]; ++x) g.items[start[cell_of(x, y, z)]++] = j;
    }
    g.c = c;
    g.rad = rad;
    g.h_max = h_max;
    g.valid = true;
    ++g.version;
    return RP_OK;
}

int run_trace(rp_medium_t m, const rp_rays *in, const rp_receivers *rx, const rp_trace_params *p,
              rp_ray_out *out, rp_hits *hits, rp_stats *stats, cudaStream_t st,
              const FixedScratch *fs)
{
    if (!m || !in || !p || !out) {
        set_error("rp_trace: null medium, rays, params or output");
        return RP_ERR_INVALID_ARG;
    }
    if (in->n < 0 || (in->n > 0 && (!in->pos || !in->dir))) {
        set_error("rp_trace: bad ray arrays");
        return RP_ERR_INVALID_ARG;
    }
    if (!out->end_pos || out->capacity < in->n) {
        set_error("rp_trace: output capacity %lld < n %lld or end_pos null",
                  (long long)out->capacity, (long long)in->n);
        return RP_ERR_INVALID_ARG;
    }
    int rc = validate_params(p, false);
    if (rc) return rc;
    int axis;
    float sdir;
    double soff;
    if ((rc = stop_axis_of(p, &axis, &sdir, &soff))) return rc;
    if (hits && hits->capacity > 0 && (!hits->ray || !hits->receiver)) {
        set_error("rp_trace: hits need ray and receiver arrays");
        return RP_ERR_INVALID_ARG;
    }
    int n_rx = (rx && rx->n > 0) ? rx->n : 0;
    if (n_rx && (!rx->center || !rx->radius)) {
        set_error("rp_trace: receiver arrays are null");
        return RP_ERR_INVALID_ARG;
    }
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device) {
        set_error("rp_trace: medium lives on device %d, current device is %d", m->device, dev);
        return RP_ERR_INVALID_ARG;
    }

    // receivers: bin into a uniform cell grid on the host (each sphere listed in every cell
    // its centre box, inflated by R + h_max / 2, overlaps); the calling thread keeps the last
    // receiver set, its grid and the grid's device copy, so that a call with the same
    // receivers and h_max skips the binning and the upload (a call with a fixed scratch
    // copies the grid into the scratch instead)
    static thread_local RxGrid rxg;
    if (n_rx) {
        std::vector<double> c(3 * (size_t)n_rx), rad(n_rx);
        // host arrays are read directly; device arrays are read back (a stream synchronisation)
        auto on_host = [](const void *q) {
            cudaPointerAttributes attr;
            memset(&attr, 0, sizeof attr);
            const bool dev = cudaPointerGetAttributes(&attr, q) == cudaSuccess &&
                             (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            return !dev;
        };
        if (on_host(rx->center) && on_host(rx->radius)) {
            std::memcpy(c.data(), rx->center, c.size() * sizeof(double));
            std::memcpy(rad.data(), rx->radius, rad.size() * sizeof(double));
        } else {
            RP_CUDA_TRY(cudaMemcpyAsync(c.data(), rx->center, c.size() * sizeof(double),
                                        cudaMemcpyDefault, st));
            RP_CUDA_TRY(cudaMemcpyAsync(rad.data(), rx->radius, rad.size() * sizeof(double),
                                        cudaMemcpyDefault, st));
            RP_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (!(rxg.valid && rxg.h_max == p->h_max && rxg.c == c && rxg.rad == rad)) {
            rxg.valid = false;
            if ((rc = bin_receivers(c, rad, p->h_max, rxg))) return rc;
        }
    }
    const std::vector<SphereC> &spheres = rxg.spheres;
    const std::vector<int2> &cells = rxg.cells;
    const std::vector<int> &items = rxg.items;
    const float *g_org = rxg.org, *g_hi = rxg.hi;
    const float g_inv = n_rx ? rxg.inv : 1.0f;
    const int g_dims[3] = {n_rx ? rxg.dims[0] : 1, n_rx ? rxg.dims[1] : 1, n_rx ? rxg.dims[2] : 1};

    const int block = p->block > 0 ? p->block : kBlockDefault;
    const int variant = medium_variant(m);
    const int per_sm = trace_blocks(variant, p->precision, block, p->blocks_per_sm);
    if (per_sm < 0) return per_sm;
    const int grid = sm_count(dev) * per_sm;
    const int threads = grid * block;
    // scratch layout: control block, receivers, per-thread stacks, warp clocks, queue last
    long long q_cap = out->capacity - in->n;
    int depth = kStackDepth;
    const size_t off_ctrl = 0;
    const size_t off_s = align_up(sizeof(Ctrl));
    const size_t off_z = off_s + align_up(sizeof(SphereC) * (size_t)std::max(n_rx, 1));
    const size_t n_cells = n_rx ? cells.size() : 0, n_items = n_rx ? items.size() : 0;
    const size_t off_b = off_z + align_up(sizeof(int2) * std::max<size_t>(n_cells, 1));
    const size_t off_k = off_b + align_up(sizeof(int) * std::max<size_t>(n_items, 1));
    const size_t clk_bytes = align_up(sizeof(unsigned long long) * 2 * (size_t)(threads / 32));
    if (fs) {
        // fixed scratch: at most half of it for the stacks, the rest (after the fixed parts)
        // for the queue
        if (off_k + clk_bytes + align_up(sizeof(QRec) * (size_t)threads) + 4096 > fs->size) {
            set_error("rp_trace_static: the %zu-byte fixed scratch cannot hold the control block, "
                      "the cell table of %d receivers (%zu bytes) and one %zu-byte stack record "
                      "for each of the %d threads of the launch (%d SMs x %d blocks x %d); "
                      "fewer blocks_per_sm or receivers fit",
                      fs->size, n_rx, off_k - off_s, sizeof(QRec), threads, sm_count(dev),
                      per_sm, block);
            return RP_ERR_INVALID_ARG;
        }
        while (depth > 1 && off_k + clk_bytes + sizeof(QRec) * (size_t)threads * depth > fs->size / 2)
            --depth;
    }
    const size_t off_w = off_k + align_up(sizeof(QRec) * (size_t)threads * depth);
    // the coherent order of the primaries (not with the fixed scratch): order, keys, the
    // histogram and the depth range
    const long long n_in = in->n;
    const bool order = !fs && p->ray_order == RP_ORDER_COHERENT && n_in > 1;
    const size_t ord_keys = align_up(sizeof(uint32_t) * (size_t)n_in);
    const size_t ord_hist = ord_keys + align_up(sizeof(uint16_t) * (size_t)n_in);
    const size_t ord_bytes =
        order ? ord_hist + align_up(sizeof(uint32_t) * (kOrderBins + 2 + kOrderScanBlocks)) : 0;
    const size_t off_o = off_w + clk_bytes;
    const size_t off_q = off_o + ord_bytes;
    if (fs) {
        const long long fit = (long long)((fs->size - off_q) / sizeof(QRec));
        q_cap = std::min(q_cap, fit);
    }
    const size_t total = off_q + align_up(sizeof(QRec) * (size_t)std::max(q_cap, 1LL));

    Workspace &ws = workspace(dev);
    std::unique_lock<std::mutex> lock(fs ? *fs->mu : ws.mu);
    if (!fs && (rc = ensure_workspace(ws, total))) return rc;
    // Declared after the lock, so destroyed before it is released: on every return from here
    // on, the work already queued on `st` (which reads and writes the scratch) has drained
    // before another call may reuse the scratch, and the timing events are released.
    struct Drain {
        cudaStream_t st;
        cudaEvent_t ev[RP_MAX_WAVES + 1];
        bool queued = false;
        ~Drain()
        {
            if (queued) cudaStreamSynchronize(st);
            for (cudaEvent_t e : ev)
                if (e) cudaEventDestroy(e);
        }
    } drain{st, {}};
    char *base = fs ? (char *)fs->ptr : (char *)ws.ptr;
    Ctrl *ctrl = (Ctrl *)(base + off_ctrl);

    Sinks sk;
    memset(&sk, 0, sizeof sk);
    sk.ctrl = ctrl;
    sk.queue = (QRec *)(base + off_q);
    sk.q_cap = (unsigned long long)q_cap;
    sk.stack = (QRec *)(base + off_k);
    sk.stack_depth = depth;
    sk.warp_clock = (unsigned long long *)(base + off_w);
    sk.out = *out;
    if (hits) sk.hits = *hits;
    sk.has_rx = n_rx > 0;
    // the receiver grid: the calling thread's device copy, or (fixed scratch, which allocates
    // nothing) a copy in the scratch made by every call
    const bool rx_cached = n_rx && !fs && dev < RxGrid::kDevices;
    sk.rx.s = (const SphereC *)(base + off_s);
    sk.rx.cell = (const int2 *)(base + off_z);
    sk.rx.items = (const int *)(base + off_b);
    sk.rx.n = n_rx;
    sk.rx.nx = g_dims[0];
    sk.rx.ny = g_dims[1];
    sk.rx.nz = g_dims[2];
    for (int a = 0; a < 3; ++a) {
        sk.rx.org[a] = g_org[a];
        sk.rx.hi[a] = g_hi[a];
    }
    sk.rx.inv_cell = g_inv;

    drain.queued = true;
    RP_CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    if (rx_cached) {
        const char *ps, *pz, *pb;
        if ((rc = rx_device_copy(rxg, dev, st, &ps, &pz, &pb))) return rc;
        sk.rx.s = (const SphereC *)ps;
        sk.rx.cell = (const int2 *)pz;
        sk.rx.items = (const int *)pb;
    } else if (n_rx) {
        RP_CUDA_TRY(cudaMemcpyAsync(base + off_s, spheres.data(), sizeof(SphereC) * n_rx,
                                    cudaMemcpyHostToDevice, st));
        RP_CUDA_TRY(cudaMemcpyAsync(base + off_z, cells.data(), sizeof(int2) * cells.size(),
                                    cudaMemcpyHostToDevice, st));
        if (!items.empty())
            RP_CUDA_TRY(cudaMemcpyAsync(base + off_b, items.data(), sizeof(int) * items.size(),
                                        cudaMemcpyHostToDevice, st));
    }
    k_init_ctrl<<<1, 1, 0, st>>>(ctrl, in->n);

    WaveIn wi;
    wi.pos = in->pos;
    wi.dir = in->dir;
    wi.amp = in->amp;
    wi.n = in->n;
    wi.stop = plane_const(soff);
    wi.h0 = p->h0;
    wi.h0f = (float)p->h0;

    const int n_waves = p->max_generation + 1;  // launches: the stacks' overflow needs at most this
    cudaEvent_t *ev = drain.ev;
    for (int w = 0; w <= n_waves; ++w) RP_CUDA_TRY(cudaEventCreate(&ev[w]));
    RP_CUDA_TRY(cudaEventRecord(ev[0], st));
    wi.ord = nullptr;
    if (order) {  // inside the timed region
        uint32_t *ord = (uint32_t *)(base + off_o);
        uint16_t *key = (uint16_t *)(base + off_o + ord_keys);
        uint32_t *hist = (uint32_t *)(base + off_o + ord_hist), *range = hist + kOrderBins;
        // histogram and the range's maximum start at 0, its minimum at all ones
        RP_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (kOrderBins + 2), st));
        RP_CUDA_TRY(cudaMemsetAsync(range, 0xFF, sizeof(uint32_t), st));
        const unsigned g = (unsigned)std::min<long long>((n_in + 255) / 256, 8LL * sm_count(dev));
        k_order_range<<<g, 256, 0, st>>>(in->pos + 2 * n_in, n_in, range);
        k_order_keys<<<g, 256, 0, st>>>(in->pos, in->dir, n_in, range, key, hist);
        k_order_scan<<<kOrderScanBlocks, 1024, 0, st>>>(hist, range + 2);
        k_order_offsets<<<kOrderScanBlocks, 1024, 0, st>>>(hist, range + 2);
        k_order_scatter<<<g, 256, 0, st>>>(key, n_in, hist, ord);
        RP_CUDA_TRY(cudaGetLastError());
        wi.ord = ord;
    }
    const bool f64 = p->precision == RP_FP64;
    const StepParams<PrecF64> sp64 = step_params<PrecF64>(p, axis, sdir);
    const StepParams<PrecF32> sp32 = step_params<PrecF32>(p, axis, sdir);
    switch (variant) {
    case VARIANT_SPHERES:
        rc = f64 ? launch_waves<PrecF64, MediumSpheres>(m->layered, sp64, sk, wi, n_waves, grid,
                                                        block, st, ev)
                 : launch_waves<PrecF32, MediumSpheres>(m->layered, sp32, sk, wi, n_waves, grid,
                                                        block, st, ev);
        break;
    case VARIANT_SURFACES: {
        const MediumSurfaces ms = surfaces_of(m);
        rc = f64 ? launch_waves<PrecF64, MediumSurfaces>(ms, sp64, sk, wi, n_waves, grid, block,
                                                         st, ev)
                 : launch_waves<PrecF32, MediumSurfaces>(ms, sp32, sk, wi, n_waves, grid, block,
                                                         st, ev);
        break;
    }
    case VARIANT_LAYERED:
        rc = f64 ? launch_waves<PrecF64, MediumLayered>(m->layered, sp64, sk, wi, n_waves, grid,
                                                        block, st, ev)
                 : launch_waves<PrecF32, MediumLayered>(m->layered, sp32, sk, wi, n_waves, grid,
                                                        block, st, ev);
        break;
    default:
        rc = f64 ? launch_waves<PrecF64, MediumGrid>(m->grid, sp64, sk, wi, n_waves, grid, block,
                                                     st, ev)
                 : launch_waves<PrecF32, MediumGrid>(m->grid, sp32, sk, wi, n_waves, grid, block,
                                                     st, ev);
    }
    // read-back: pinned buffers of the workspace, or (fixed scratch) pageable host memory and
    // no warp clocks, so that nothing is allocated
    Ctrl ctrl_local;
    Ctrl *hc = fs ? &ctrl_local : (Ctrl *)ws.host_ctrl;
    const size_t n_clk = fs ? 0 : 2 * (size_t)(threads / 32);
    if (!rc && !fs) rc = ensure_host_clock(ws, n_clk * sizeof(unsigned long long));
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && n_clk)
            e = cudaMemcpyAsync(ws.host_clock, sk.warp_clock, n_clk * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "rp_trace: control block read-back");
    }
    const unsigned long long *wclk = (const unsigned long long *)ws.host_clock;
    float wave_ms[RP_MAX_WAVES] = {0.0f}, ms = 0.0f;
    if (!rc) {
        for (int w = 0; w < n_waves; ++w) cudaEventElapsedTime(&wave_ms[w], ev[w], ev[w + 1]);
        cudaEventElapsedTime(&ms, ev[0], ev[n_waves]);
        drain.queued = false;  // the read-back synchronised the stream
    }
    if (rc) return rc;

    unsigned flags = hc->flags;
    if (!hits) flags &= ~(unsigned)FLAG_HIT_OVERFLOW;
    if (stats) {
        stats->rays = (int64_t)hc->out_count;
        stats->hits = (int64_t)hc->n_hits;
        stats->secondaries = (int64_t)hc->n_secondary;
        stats->steps_accepted = (int64_t)hc->steps_acc;
        stats->steps_rejected = (int64_t)hc->steps_rej;
        stats->steps_root = (int64_t)hc->steps_root;
        stats->queue_needed = (int64_t)hc->q_tail;
        stats->waves = n_waves;
        stats->flags = (int32_t)flags;
        stats->queue_capacity = (int64_t)q_cap;
        stats->threads = threads;
        stats->stack_depth = depth;
        stats->kernel_ms = ms;
        for (int w = 0; w < RP_MAX_WAVES; ++w) stats->wave_ms[w] = w < n_waves ? wave_ms[w] : 0.0;
        // tail of the first launch: warp end times after the earliest warp start
        const size_t nw = n_clk / 2;
        if (nw) {
            unsigned long long t0 = ~0ull;
            std::vector<double> ends(nw);
            for (size_t w = 0; w < nw; ++w) t0 = std::min(t0, wclk[2 * w]);
            for (size_t w = 0; w < nw; ++w) ends[w] = (double)(wclk[2 * w + 1] - t0) * 1e-6;
            const auto mm = std::minmax_element(ends.begin(), ends.end());
            stats->warp_end_ms[0] = *mm.first;
            stats->warp_end_ms[2] = *mm.second;
            std::nth_element(ends.begin(), ends.begin() + nw / 2, ends.end());
            stats->warp_end_ms[1] = ends[nw / 2];
        }
    }
    if (flags & (FLAG_OUT_OVERFLOW | FLAG_QUEUE_OVERFLOW | FLAG_HIT_OVERFLOW)) {
        set_error("rp_trace: overflow (rays %llu / capacity %lld, hits %llu / capacity %lld)",
                  hc->out_count, (long long)out->capacity, hc->n_hits,
                  (long long)(hits ? hits->capacity : 0));
        return RP_ERR_OVERFLOW;
    }
    return RP_OK;
}

}  // namespace rph
