// pathfind.cu -- batched source-receiver path finding (rp_find_paths).
//
// Sec. 2 of the paper checks the tracer against analytic solutions by finding the launch
// angles that connect a source with an observation point.  For a batch of pairs
// (z_s, z_r, D) this runs, entirely on the GPU:
//   1. k_prefix   exclusive prefix sum of the per-pair scan sizes (uneven: 32..512 angles)
//   2. k_scan     one persistent launch over all (pair, angle) rays: each ray leaves
//                 (0, 0, z_s) in the x-z plane and stops on the plane x = D; its vertical miss
//                 z - z_r is stored (+inf if the path budget ran out first: the ray is far
//                 below; NaN for any other end)
//   3. k_brackets adjacent angles of one pair whose misses change sign become brackets
//   4. k_bisect   one persistent launch over all brackets: each lane bisects its bracket in
//                 FP64 on the launch angle, one full trace per step, until |miss| < hit_tol
//   5. k_finalize per pair: candidate solutions sorted by travel time into the output slots
// Rays use the same lane state machine as rp_trace (trace_core.cuh) with a per-ray stop plane
// and path budget 2 (D + z_s + z_r) + 100 m; no secondaries are cast.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>

#include "rp_internal.h"

namespace cg = cooperative_groups;
using namespace rpk;

namespace rph {

namespace {

constexpr int kMaxCand = 16;  // candidate solutions kept per pair before sorting

struct PairIn {
    const double *zs, *zr, *dist;
    const int32_t *n_angles;
    long long n_pairs;
    double hit_tol;
    int32_t max_iter, max_sol;
};

struct Bracket {
    double tha, thb, ma;
    int32_t pair;
    int32_t it, active;  // speculative rounds: bisection step of the next midpoint; still open
    int32_t pad;
};

struct Cand {
    double launch, receive, time, path, amp, miss;
    double dth;  // refinement only: launch-angle uncertainty tol / |d miss / d launch|
    int32_t type, n_iter;
};

struct PfCtrl {
    unsigned long long claim_scan, claim_bisect, n_brackets, rays;
    unsigned long long steps_acc, steps_rej, steps_root;
    unsigned long long open;  // speculative rounds: brackets still open
    unsigned int flags, pad;
};

__device__ __forceinline__ long long pf_claim(unsigned long long *counter)
{
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    return (long long)(base + g.thread_rank());
}

__device__ __forceinline__ int scan_items(const PairIn &pi, long long i)
{
    if (pi.dist[i] < pi.hit_tol) return 1;
    const int n = pi.n_angles[i];
    return n < 2 ? 2 : n;
}

// Exclusive prefix sum of the scan sizes, one block of 1024 threads: each thread sums a
// contiguous chunk, the 1024 partial sums are scanned in shared memory.
__global__ void __launch_bounds__(1024) k_prefix(const PairIn pi, long long *prefix)
{
    __shared__ long long part[1024];
    const long long n = pi.n_pairs;
    const long long chunk = (n + 1023) / 1024;
    const long long lo = threadIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    long long s = 0;
    for (long long i = lo; i < hi; ++i) s += scan_items(pi, i);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (long long i = lo; i < hi; ++i) {
        prefix[i] = run;
        run += scan_items(pi, i);
    }
    if (threadIdx.x == 1023) prefix[n] = part[1023];
}

// pair of a global scan item (prefix is exclusive, n_pairs + 1 entries)
__device__ __forceinline__ long long pair_of(const long long *prefix, long long n_pairs, long long k)
{
    long long lo = 0, hi = n_pairs;  // invariant: prefix[lo] <= k < prefix[hi]
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (prefix[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Sets a lane up for the ray of pair i launched at angle th (from +z, in the x-z plane).
template <class P>
__device__ __forceinline__ void launch_ray(Lane<P> &L, const MediumLayered &med,
                                           const StepParams<P> &sp, const PairIn &pi, double h0,
                                           long long i, double th, bool vertical, long long id)
{
    const double zs = pi.zs[i], zr = pi.zr[i], D = pi.dist[i];
    const double t[3] = {sin(th), 0.0, cos(th)};
    const double q = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    P::set(L.r, 0, 0.0);
    P::set(L.r, 1, 0.0);
    P::set(L.r, 2, zs);
#pragma unroll
    for (int a = 0; a < 3; ++a) P::set(L.t, a, t[a] / q);
    L.A = 1.0;
    L.A0 = 1.0;
    P::sset(L.T, 0.0);
    P::sset(L.s, 0.0);
    L.h = P::from_d(h0);
    L.id = id;
    L.parent = -1;
    L.gen = 0;
    L.seq = 0;
    L.layer = layer_of(med, zs);
    L.mode = MODE_NORMAL;
    L.ev = EV_NONE;
    L.side = 0;
    L.it = 0;
    L.n_acc = L.n_rej = L.n_root = L.n_refl = L.n_turn = L.root_fail = 0;
    L.status = RP_ST_ALIVE;
    L.pend = 0;
    L.tail = 0;
    load_layer<P>(L.lc, med, L.layer);
    L.stop_axis = vertical ? 2 : 0;
    L.stop = plane_of(vertical ? zr : D);
    L.mp = plane_of(2.0 * (D + zs + zr) + 100.0);
    init_stop(L, sp);
    set_trial(L, sp);
}

// vertical miss at the stop plane: z - z_r; +inf when the path budget ran out first (the ray
// is far below), NaN for any other end
template <class P>
__device__ __forceinline__ double miss_of(const Lane<P> &L, double zr)
{
    if (L.status == RP_ST_REACHED_STOP) return P::get(L.r, 2) - zr;
    if (L.status == RP_ST_MAX_PATH) return __longlong_as_double(0x7ff0000000000000ll);
    return __longlong_as_double(0x7ff8000000000000ll);
}

template <class P>
__device__ __forceinline__ void add_candidate(const Lane<P> &L, long long i, double th,
                                              int it, double miss, int *cand_n, Cand *cand,
                                              PfCtrl *ctrl)
{
    const int c = atomicAdd(&cand_n[i], 1);
    if (c >= kMaxCand) {
        atomicOr(&ctrl->flags, 4u);
        return;
    }
    Cand &o = cand[i * kMaxCand + c];
    o.type = L.n_refl > 0 ? RP_SOL_REFLECTED : (L.n_turn > 0 ? RP_SOL_REFRACTED : RP_SOL_DIRECT);
    o.n_iter = it;
    o.launch = th;
    o.receive = acos(fmax(-1.0, fmin(1.0, P::get(L.t, 2))));
    o.time = P::sget(L.T);
    o.path = P::sget(L.s);
    o.amp = L.A;
    o.miss = miss;
    o.dth = 0.0;
}

struct ScanArgs {
    PairIn pi;
    const long long *prefix;
    double *miss;
    int *cand_n;
    Cand *cand;
    PfCtrl *ctrl;
    double h0;
};

// Warp-synchronous driver shared by the scan and the bisection: `next` gives a lane its next
// ray (false: no more work), `done` consumes a finished ray; between them every lane that
// still traces takes one Cash-Karp step per iteration; splits and finished rays are serviced
// in batches as in k_trace_wave.
template <class P, class Next, class Done>
__device__ __forceinline__ void drive(const MediumLayered &med, const StepParams<P> &sp,
                                      const Sinks &sk, PfCtrl *ctrl, Next next, Done done_fn)
{
    Lane<P> L;
    L.stk = 0;
    unsigned int acc = 0, rej = 0, root = 0, rays = 0;
    // fetch: the lane wants its next ray (the first one too comes from a service phase, so
    // that `next` is inlined once)
    bool active = false, done = false, fetch = true;
    unsigned int idle = 0;  // waiting lane-iterations since the last service phase
    while (__any_sync(0xffffffffu, active || done || fetch)) {
        __syncwarp();
        if (active && L.pend == 0 && advance<P, MediumLayered>(med, L, sp, sk)) {
            active = false;
            done = true;
        }
        const bool waits = done || fetch || (active && L.pend != 0);
        const unsigned int wait = __ballot_sync(0xffffffffu, waits);
        const unsigned int step_mask = __ballot_sync(0xffffffffu, active && L.pend == 0);
        // a ray bouncing in a duct is served at once, as in k_trace_wave
        const bool hot = __any_sync(0xffffffffu, active && L.pend != 0 && L.n_refl >= kHotSplits);
        idle += (unsigned int)__popc(wait);
        if (wait != 0u && (idle >= sp.service_idle || step_mask == 0u || hot)) {
            idle = 0;
            if (active && L.pend != 0 && finish_split<P>(med, L, sp, sk)) {
                active = false;
                done = true;
            }
            if (done || fetch) {
                if (done) {
                    acc += (unsigned int)L.n_acc;
                    rej += (unsigned int)L.n_rej;
                    root += (unsigned int)L.n_root;
                    ++rays;
                    done_fn(L);
                }
                done = fetch = false;
                active = next(L);
            }
        }
    }
    __syncwarp();
    acc = __reduce_add_sync(0xffffffffu, acc);
    rej = __reduce_add_sync(0xffffffffu, rej);
    root = __reduce_add_sync(0xffffffffu, root);
    rays = __reduce_add_sync(0xffffffffu, rays);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctrl->steps_acc, (unsigned long long)acc);
        atomicAdd(&ctrl->steps_rej, (unsigned long long)rej);
        atomicAdd(&ctrl->steps_root, (unsigned long long)root);
        atomicAdd(&ctrl->rays, (unsigned long long)rays);
    }
}

template <class P>
__global__ void __launch_bounds__(128, P::kMinBlocks)
    k_scan(const MediumLayered med, const StepParams<P> sp, const Sinks sk, const ScanArgs a)
{
    const long long total = a.prefix[a.pi.n_pairs];
    long long cur = -1, cur_pair = 0;
    int cur_j = 0;
    bool cur_vert = false;
    auto next = [&](Lane<P> &L) -> bool {
        cur = pf_claim(&a.ctrl->claim_scan);
        if (cur >= total) return false;
        cur_pair = pair_of(a.prefix, a.pi.n_pairs, cur);
        cur_j = (int)(cur - a.prefix[cur_pair]);
        cur_vert = a.pi.dist[cur_pair] < a.pi.hit_tol;
        const double pi_ = 3.14159265358979323846;
        double th;
        if (cur_vert) {
            th = a.pi.zr[cur_pair] >= a.pi.zs[cur_pair] ? 0.0 : pi_;
        } else {
            const int na = scan_items(a.pi, cur_pair);
            th = pi_ * (double)cur_j / (double)(na - 1);
        }
        launch_ray<P>(L, med, sp, a.pi, a.h0, cur_pair, th, cur_vert, cur);
        return true;
    };
    auto done = [&](Lane<P> &L) {
        const double m = miss_of<P>(L, a.pi.zr[cur_pair]);
        a.miss[cur] = m;
        if (cur_vert && L.status == RP_ST_REACHED_STOP) {
            const double th = a.pi.zr[cur_pair] >= a.pi.zs[cur_pair] ? 0.0 : 3.14159265358979323846;
            add_candidate<P>(L, cur_pair, th, 0, 0.0, a.cand_n, a.cand, a.ctrl);
        }
    };
    drive<P>(med, sp, sk, a.ctrl, next, done);
}

struct BracketArgs {
    PairIn pi;
    const long long *prefix;
    const double *miss;
    Bracket *br;
    unsigned long long br_cap;
    PfCtrl *ctrl;
};

// adjacent scan angles of one pair with misses of opposite sign (NaN never brackets)
__global__ void k_brackets(const BracketArgs a)
{
    const long long total = a.prefix[a.pi.n_pairs];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = pair_of(a.prefix, a.pi.n_pairs, k);
        if (a.pi.dist[i] < a.pi.hit_tol) continue;
        const int na = scan_items(a.pi, i);
        const int j = (int)(k - a.prefix[i]);
        if (j + 1 >= na) continue;
        const double ma = a.miss[k], mb = a.miss[k + 1];
        if (!((ma > 0.0 && mb < 0.0) || (ma < 0.0 && mb > 0.0))) continue;
        const unsigned long long b = atomicAdd(&a.ctrl->n_brackets, 1ull);
        if (b >= a.br_cap) {
            atomicOr(&a.ctrl->flags, 8u);
            continue;
        }
        const double pi_ = 3.14159265358979323846;
        Bracket &o = a.br[b];
        o.tha = pi_ * (double)j / (double)(na - 1);
        o.thb = pi_ * (double)(j + 1) / (double)(na - 1);
        o.ma = ma;
        o.pair = (int)i;
        o.it = 1;
        o.active = 1;
        o.pad = 0;
    }
}

struct BisectArgs {
    PairIn pi;
    const Bracket *br;
    unsigned long long br_cap;
    int *cand_n;
    Cand *cand;
    PfCtrl *ctrl;
    double h0;
};

// FP64 bisection on the launch angle, one bracket per lane at a time
template <class P>
__global__ void __launch_bounds__(128, P::kMinBlocks)
    k_bisect(const MediumLayered med, const StepParams<P> sp, const Sinks sk, const BisectArgs a)
{
    const unsigned long long nb0 = a.ctrl->n_brackets;
    const long long nb = (long long)(nb0 < a.br_cap ? nb0 : a.br_cap);
    double tha = 0.0, thb = 0.0, ma = 0.0, thm = 0.0;
    int it = 0, pair = 0;
    // starts the next bisection trace of the current bracket; false if the bracket is done
    auto step_bracket = [&](Lane<P> &L) -> bool {
        if (it > a.pi.max_iter) return false;
        thm = 0.5 * (tha + thb);
        if (!(thm > tha && thm < thb)) return false;  // bracket exhausted
        launch_ray<P>(L, med, sp, a.pi, a.h0, pair, thm, false, -1);
        return true;
    };
    auto next = [&](Lane<P> &L) -> bool {
        for (;;) {
            const long long b = pf_claim(&a.ctrl->claim_bisect);
            if (b >= nb) return false;
            const Bracket &B = a.br[b];
            tha = B.tha;
            thb = B.thb;
            ma = B.ma;
            pair = B.pair;
            it = 1;
            if (step_bracket(L)) return true;
        }
    };
    bool resume = false;  // set by done(): the current bracket continues with a new trace
    auto done = [&](Lane<P> &L) {
        const double mm = miss_of<P>(L, a.pi.zr[pair]);
        resume = false;
        if (isnan(mm)) return;
        if (fabs(mm) < a.pi.hit_tol) {
            add_candidate<P>(L, pair, thm, it, mm, a.cand_n, a.cand, a.ctrl);
            return;
        }
        if ((mm > 0.0) == (ma > 0.0)) {
            tha = thm;
            ma = mm;
        } else {
            thb = thm;
        }
        ++it;
        resume = true;
    };
    auto next_or_resume = [&](Lane<P> &L) -> bool {
        if (resume) {
            resume = false;
            if (step_bracket(L)) return true;
        }
        return next(L);
    };
    drive<P>(med, sp, sk, a.ctrl, next_or_resume, done);
}

// Speculative bisection for few brackets.  One round evaluates, for every open bracket, the
// G = 2^J - 1 midpoints of J consecutive bisection steps at once -- every point the sequential
// bisection could visit next, as the nodes of a binary tree in heap order, each computed by the
// same nested midpoints 0.5 (lo + hi) that the sequential steps compute -- one trace per lane;
// k_bisect_resolve then walks the tree along the signs exactly as J sequential steps would and
// keeps the same stopping rules, so the result equals k_bisect's, bit for bit, in J times fewer
// rounds of trace latency and about G / J times the traces.
struct NodeRec {
    double thm, miss, receive, time, path, amp;
    int32_t type, flag;  // flag: 0 traced, 1 not taken (step cap or exhausted bracket)
};

struct RoundArgs {
    PairIn pi;
    Bracket *br;
    long long nb;
    int32_t J, G;
    NodeRec *rec;
    PfCtrl *ctrl;
    double h0;
};

// the heap node h (1-based) of a bracket's tree: its angle, depth, and whether it lies strictly
// inside its interval
__device__ __forceinline__ void tree_node(const Bracket &B, int h, double &thm, int &depth,
                                          bool &inside)
{
    double lo = B.tha, hi = B.thb;
    depth = 31 - __clz(h);
    for (int d = depth - 1; d >= 0; --d) {
        const double mid = 0.5 * (lo + hi);
        if ((h >> d) & 1)
            lo = mid;
        else
            hi = mid;
    }
    thm = 0.5 * (lo + hi);
    inside = thm > lo && thm < hi;
}

template <class P>
__global__ void __launch_bounds__(128, P::kMinBlocks)
    k_bisect_round(const MediumLayered med, const StepParams<P> sp, const Sinks sk, const RoundArgs a)
{
    const long long items = a.nb * a.G;
    long long cur = 0;
    auto next = [&](Lane<P> &L) -> bool {
        for (;;) {
            cur = pf_claim(&a.ctrl->claim_bisect);
            if (cur >= items) return false;
            const long long b = cur / a.G;
            const Bracket &B = a.br[b];
            if (!B.active) continue;
            const int h = (int)(cur % a.G) + 1;
            double thm;
            int depth;
            bool inside;
            tree_node(B, h, thm, depth, inside);
            NodeRec &R = a.rec[cur];
            R.thm = thm;
            if (B.it + depth > a.pi.max_iter || !inside) {
                R.flag = 1;
                continue;
            }
            R.flag = 0;
            launch_ray<P>(L, med, sp, a.pi, a.h0, B.pair, thm, false, -1);
            return true;
        }
    };
    auto done = [&](Lane<P> &L) {
        const long long b = cur / a.G;
        NodeRec &R = a.rec[cur];
        R.miss = miss_of<P>(L, a.pi.zr[a.br[b].pair]);
        R.type = L.n_refl > 0 ? RP_SOL_REFLECTED : (L.n_turn > 0 ? RP_SOL_REFRACTED : RP_SOL_DIRECT);
        R.receive = acos(fmax(-1.0, fmin(1.0, P::get(L.t, 2))));
        R.time = P::sget(L.T);
        R.path = P::sget(L.s);
        R.amp = L.A;
    };
    drive<P>(med, sp, sk, a.ctrl, next, done);
}

// Walks each open bracket's tree as the sequential bisection would: stop on a NaN miss, on a
// hit (|miss| < hit_tol: a candidate), at the step cap or when the interval is exhausted;
// otherwise keep the half whose ends still differ in sign.  Counts the brackets still open.
__global__ void k_bisect_resolve(const RoundArgs a, int *cand_n, Cand *cand,
                                 unsigned long long *open)
{
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < a.nb;
         b += (long long)gridDim.x * blockDim.x) {
        Bracket &B = a.br[b];
        if (!B.active) continue;
        double lo = B.tha, hi = B.thb;
        int h = 1;
        bool open_ = true;
        for (int d = 0; d < a.J; ++d) {
            const NodeRec &R = a.rec[b * a.G + (h - 1)];
            if (R.flag || isnan(R.miss)) {
                open_ = false;
                break;
            }
            if (fabs(R.miss) < a.pi.hit_tol) {
                const int c = atomicAdd(&cand_n[B.pair], 1);
                if (c >= kMaxCand) {
                    atomicOr(&a.ctrl->flags, 4u);
                } else {
                    Cand &o = cand[(long long)B.pair * kMaxCand + c];
                    o.type = R.type;
                    o.n_iter = B.it + d;
                    o.launch = R.thm;
                    o.receive = R.receive;
                    o.time = R.time;
                    o.path = R.path;
                    o.amp = R.amp;
                    o.miss = R.miss;
                    o.dth = 0.0;
                }
                open_ = false;
                break;
            }
            if ((R.miss > 0.0) == (B.ma > 0.0)) {
                lo = R.thm;
                h = 2 * h + 1;
            } else {
                hi = R.thm;
                h = 2 * h;
            }
        }
        if (open_) {
            B.tha = lo;
            B.thb = hi;
            B.it += a.J;
            atomicAdd(open, 1ull);
        } else {
            B.active = 0;
        }
    }
}

// per pair: candidates sorted by travel time into the max_sol output slots
__global__ void k_finalize(const PairIn pi, const int *cand_n, const Cand *cand,
                           rp_solutions sol)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < pi.n_pairs;
         i += (long long)gridDim.x * blockDim.x) {
        int nc = cand_n[i] < kMaxCand ? cand_n[i] : kMaxCand;
        int order[kMaxCand];
        for (int c = 0; c < nc; ++c) order[c] = c;
        for (int c = 1; c < nc; ++c) {  // insertion sort by time, ties by launch angle
            const int key = order[c];
            const Cand &K = cand[i * kMaxCand + key];
            int d = c - 1;
            while (d >= 0) {
                const Cand &X = cand[i * kMaxCand + order[d]];
                if (X.time > K.time || (X.time == K.time && X.launch > K.launch)) {
                    order[d + 1] = order[d];
                    --d;
                } else {
                    break;
                }
            }
            order[d + 1] = key;
        }
        const int keep = nc < pi.max_sol ? nc : pi.max_sol;
        sol.count[i] = keep;
        for (int c = 0; c < pi.max_sol; ++c) {
            const long long o = i * pi.max_sol + c;
            if (c < keep) {
                const Cand &X = cand[i * kMaxCand + order[c]];
                if (sol.type) sol.type[o] = X.type;
                if (sol.n_iter) sol.n_iter[o] = X.n_iter;
                if (sol.launch) sol.launch[o] = X.launch;
                if (sol.receive) sol.receive[o] = X.receive;
                if (sol.time) sol.time[o] = X.time;
                if (sol.path) sol.path[o] = X.path;
                if (sol.amp) sol.amp[o] = X.amp;
                if (sol.miss) sol.miss[o] = X.miss;
            } else {
                if (sol.type) sol.type[o] = 0;
                if (sol.n_iter) sol.n_iter[o] = 0;
                if (sol.launch) sol.launch[o] = 0.0;
                if (sol.receive) sol.receive[o] = 0.0;
                if (sol.time) sol.time[o] = 0.0;
                if (sol.path) sol.path[o] = 0.0;
                if (sol.amp) sol.amp[o] = 0.0;
                if (sol.miss) sol.miss[o] = 0.0;
            }
        }
    }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

int occ_of(const void *fn)
{
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 128, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    return occ > 0 ? occ : 1;
}

template <class P>
int run_pf(rp_medium_t m, const PairIn &pi, const rp_trace_params *tp, rp_solutions *sol,
           rp_stats *stats, cudaStream_t st, int dev)
{
    StepParams<P> sp = step_params<P>(tp, 0, 1.0f);
    sp.use_stop = 1;
    sp.max_generation = 0;
    const int occ_s = occ_of((const void *)k_scan<P>);
    const int occ_b = occ_of((const void *)k_bisect<P>);
    const int occ_r = occ_of((const void *)k_bisect_round<P>);
    if (occ_s < 0) return occ_s;
    if (occ_b < 0) return occ_b;
    if (occ_r < 0) return occ_r;
    const int sms = sm_count(dev);
    const long long np = pi.n_pairs;
    const long long lanes = (long long)sms * occ_r * 128;
    const size_t rec_cap = (size_t)(lanes + lanes / 4) + 4096;  // tree nodes of one round
    // workspace: path-finding control, tracer control block (for the split code's flags),
    // prefix sums, candidates and their counts, brackets, speculative tree nodes, then one miss
    // per scan ray
    const size_t off_pf = 0;
    const size_t off_tc = al(sizeof(PfCtrl));
    const size_t off_pre = off_tc + al(sizeof(Ctrl));
    const size_t off_cn = off_pre + al(sizeof(long long) * (size_t)(np + 1));
    const size_t off_c = off_cn + al(sizeof(int) * (size_t)np);
    const size_t br_cap = (size_t)np * 16 + 1024;
    const size_t off_br = off_c + al(sizeof(Cand) * (size_t)np * kMaxCand);
    const size_t off_rec = off_br + al(sizeof(Bracket) * br_cap);
    const size_t off_miss = off_rec + al(sizeof(NodeRec) * rec_cap);

    Workspace &ws = workspace(dev);
    std::lock_guard<std::mutex> lock(ws.mu);
    int rc = ensure_workspace(ws, off_miss + (8u << 20));
    if (rc) return rc;
    long long total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        char *base = (char *)ws.ptr;
        RP_CUDA_TRY(cudaMemsetAsync(base, 0, off_pre, st));  // both control blocks
        k_prefix<<<1, 1024, 0, st>>>(pi, (long long *)(base + off_pre));
        RP_CUDA_TRY(cudaGetLastError());
        RP_CUDA_TRY(cudaMemcpyAsync(&total, (long long *)(base + off_pre) + np, sizeof(long long),
                                    cudaMemcpyDeviceToHost, st));
        RP_CUDA_TRY(cudaStreamSynchronize(st));
        const size_t need = off_miss + al(sizeof(double) * (size_t)std::max(total, 1LL));
        if (need <= ws.size) break;
        if ((rc = ensure_workspace(ws, need))) return rc;  // grown: contents are gone, redo
    }
    char *base = (char *)ws.ptr;
    PfCtrl *ctrl = (PfCtrl *)(base + off_pf);
    const long long *prefix = (const long long *)(base + off_pre);
    int *cand_n = (int *)(base + off_cn);
    Cand *cand = (Cand *)(base + off_c);
    Bracket *br = (Bracket *)(base + off_br);
    NodeRec *rec = (NodeRec *)(base + off_rec);
    double *miss = (double *)(base + off_miss);
    RP_CUDA_TRY(cudaMemsetAsync(cand_n, 0, sizeof(int) * (size_t)std::max(np, 1LL), st));

    Sinks sk;
    memset(&sk, 0, sizeof sk);
    sk.ctrl = (Ctrl *)(base + off_tc);  // flags only: path-finding rays cast no secondaries
    sk.stack_depth = 0;

    cudaEvent_t ev[3];
    for (int k = 0; k < 3; ++k) RP_CUDA_TRY(cudaEventCreate(&ev[k]));
    RP_CUDA_TRY(cudaEventRecord(ev[0], st));
    ScanArgs sa;
    sa.pi = pi;
    sa.prefix = prefix;
    sa.miss = miss;
    sa.cand_n = cand_n;
    sa.cand = cand;
    sa.ctrl = ctrl;
    sa.h0 = tp->h0;
    k_scan<P><<<sms * occ_s, 128, 0, st>>>(m->layered, sp, sk, sa);
    BracketArgs ba;
    ba.pi = pi;
    ba.prefix = prefix;
    ba.miss = miss;
    ba.br = br;
    ba.br_cap = br_cap;
    ba.ctrl = ctrl;
    k_brackets<<<sms * 8, 256, 0, st>>>(ba);
    RP_CUDA_TRY(cudaEventRecord(ev[1], st));
    // Few brackets for the lanes: speculative rounds of J bisection steps (J as large as the
    // lanes allow, at most 5); otherwise one lane per bracket, bisecting on its own.
    unsigned long long nb_raw = 0;
    RP_CUDA_TRY(cudaMemcpyAsync(&nb_raw, &ctrl->n_brackets, sizeof nb_raw, cudaMemcpyDeviceToHost,
                                st));
    RP_CUDA_TRY(cudaStreamSynchronize(st));
    const long long nb = (long long)std::min<unsigned long long>(nb_raw, br_cap);
    int J = 1;
    while (J < 5 && nb > 0 && nb * ((1LL << (J + 1)) - 1) <= (long long)rec_cap &&
           nb * ((1LL << (J + 1)) - 1) <= lanes + lanes / 4)
        ++J;
    int rounds = 0;
    if (J == 1) {
        BisectArgs bb;
        bb.pi = pi;
        bb.br = br;
        bb.br_cap = br_cap;
        bb.cand_n = cand_n;
        bb.cand = cand;
        bb.ctrl = ctrl;
        bb.h0 = tp->h0;
        k_bisect<P><<<sms * occ_b, 128, 0, st>>>(m->layered, sp, sk, bb);
    } else {
        RoundArgs ra;
        ra.pi = pi;
        ra.br = br;
        ra.nb = nb;
        ra.J = J;
        ra.G = (1 << J) - 1;
        ra.rec = rec;
        ra.ctrl = ctrl;
        ra.h0 = tp->h0;
        const int max_rounds = pi.max_iter / J + 2;
        const int rblocks = std::max(1, (int)std::min<long long>((nb + 255) / 256, (long long)sms * 8));
        for (; rounds < max_rounds; ++rounds) {
            RP_CUDA_TRY(cudaMemsetAsync(&ctrl->claim_bisect, 0, sizeof(unsigned long long), st));
            RP_CUDA_TRY(cudaMemsetAsync(&ctrl->open, 0, sizeof(unsigned long long), st));
            k_bisect_round<P><<<sms * occ_r, 128, 0, st>>>(m->layered, sp, sk, ra);
            k_bisect_resolve<<<rblocks, 256, 0, st>>>(ra, cand_n, cand, &ctrl->open);
            RP_CUDA_TRY(cudaGetLastError());
            unsigned long long open = 0;
            RP_CUDA_TRY(cudaMemcpyAsync(&open, &ctrl->open, sizeof open, cudaMemcpyDeviceToHost, st));
            RP_CUDA_TRY(cudaStreamSynchronize(st));
            if (open == 0) {
                ++rounds;
                break;
            }
        }
    }
    k_finalize<<<std::max(1, (int)std::min<long long>((np + 255) / 256, (long long)sms * 8)), 256,
                 0, st>>>(pi, cand_n, cand, *sol);
    RP_CUDA_TRY(cudaEventRecord(ev[2], st));
    RP_CUDA_TRY(cudaGetLastError());
    PfCtrl hc;
    unsigned int tflags = 0;
    RP_CUDA_TRY(cudaMemcpyAsync(&hc, ctrl, sizeof hc, cudaMemcpyDeviceToHost, st));
    RP_CUDA_TRY(cudaMemcpyAsync(&tflags, &sk.ctrl->flags, sizeof tflags, cudaMemcpyDeviceToHost, st));
    RP_CUDA_TRY(cudaStreamSynchronize(st));
    float ms_scan = 0.0f, ms_all = 0.0f;
    cudaEventElapsedTime(&ms_scan, ev[0], ev[1]);
    cudaEventElapsedTime(&ms_all, ev[0], ev[2]);
    for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
    if (stats) {
        stats->rays = (int64_t)hc.rays;
        stats->steps_accepted = (int64_t)hc.steps_acc;
        stats->steps_rejected = (int64_t)hc.steps_rej;
        stats->steps_root = (int64_t)hc.steps_root;
        stats->queue_needed = (int64_t)hc.n_brackets;
        stats->waves = 2 + rounds;
        stats->flags = (int32_t)(hc.flags | tflags);
        stats->kernel_ms = ms_all;
        stats->wave_ms[0] = ms_scan;
        stats->wave_ms[1] = ms_all - ms_scan;
    }
    if (hc.flags & 12u) {
        set_error("rp_find_paths: more than %d candidate solutions of a pair or more than %zu "
                  "brackets; the kept solutions may not be the earliest",
                  kMaxCand, br_cap);
        return RP_ERR_OVERFLOW;
    }
    return RP_OK;
}

// ---------------------------------------------------------------------------------------
// Surrogate pipeline: geometry encoding, inference planning, secant refinement with the
// tracer, and fallback to the path finder
// ---------------------------------------------------------------------------------------

// network input of a pair: each of z_s, z_r, D mapped linearly from its range onto [-1, 1]
__device__ __forceinline__ void encode_x(double zs, double zr, double D, float *x)
{
    x[0] = (float)(2.0 * zs / RP_SUR_ZS_MAX - 1.0);
    x[1] = (float)(2.0 * zr / RP_SUR_ZR_MAX - 1.0);
    x[2] = (float)(2.0 * D / RP_SUR_D_MAX - 1.0);
}

__global__ void k_encode(long long n, const double *zs, const double *zr, const double *D,
                         const rp_solutions sol, int max_sol, float *x, float *y, float *t)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        encode_x(zs[i], zr[i], D[i], x + 3 * i);
        if (!y) continue;
        const int cnt = sol.count[i];
        const double L = sqrt(D[i] * D[i] + (zs[i] - zr[i]) * (zs[i] - zr[i]));
        const double pi_ = 3.14159265358979323846;
        for (int k = 0; k < 2; ++k) {
            const long long o = i * max_sol + k;
            const bool ex = k < cnt;
            y[2 * i + k] = cnt > 2 ? 0.5f : (ex ? 1.0f : 0.0f);
            float *tk = t + 10 * i + 5 * k;
            if (!ex) {
                for (int j = 0; j < 5; ++j) tk[j] = 0.0f;
                continue;
            }
            tk[0] = (float)(2.0 * sol.launch[o] / pi_ - 1.0);
            tk[1] = (float)(2.0 * sol.receive[o] / pi_ - 1.0);
            tk[2] = (float)((kC0 * sol.time[o] / RP_SUR_N_REF - L) / RP_SUR_LEN_SCALE);
            tk[3] = (float)((sol.path[o] - L) / RP_SUR_LEN_SCALE);
            tk[4] = (float)sol.amp[o];
        }
    }
}

struct RTask {
    long long q;
    int32_t mask, pad;  // bit k: slot k is to be searched
    double th0[2];      // the network's launch angles of the two slots
};

struct SurCtrl {
    unsigned long long n_tasks, claim, n_fallback, failed;
    unsigned long long fail_end, fail_iters, fail_step, duplicates, deflated;
};

// slot states in `cok`: absent (trusted), refining, refined
enum { SLOT_ABSENT = 0, SLOT_PENDING = 2, SLOT_OK = 1 };

// Per query: a slot whose existence probability is <= 1 - conf is trusted to be absent; the
// other slots of the query form one refinement task.  Vertical pairs, and pairs whose slot 0
// is absent but slot 1 is not, go to the path finder.
__global__ void k_plan(long long n, const float *out, double conf, const PairIn pi, RTask *tasks,
                       SurCtrl *sc, int *qflag, int *cok)
{
    const double pi_ = 3.14159265358979323846;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        bool ex[2];
        for (int k = 0; k < 2; ++k) {
            const double p = 1.0 / (1.0 + exp(-(double)out[12 * i + 6 * k]));
            ex[k] = p > 1.0 - conf;
        }
        const int flag = (pi.dist[i] < pi.hit_tol || (ex[1] && !ex[0])) ? 1 : 0;
        qflag[i] = flag;
        for (int k = 0; k < 2; ++k) cok[2 * i + k] = (ex[k] && !flag) ? SLOT_PENDING : SLOT_ABSENT;
        if (flag || !ex[0]) continue;
        const unsigned long long t = atomicAdd(&sc->n_tasks, 1ull);
        RTask &T = tasks[t];
        T.q = i;
        T.mask = (ex[0] ? 1 : 0) | (ex[1] ? 2 : 0);
        T.pad = 0;
        for (int k = 0; k < 2; ++k) {
            const double th = 0.5 * pi_ * ((double)out[12 * i + 6 * k + 1] + 1.0);
            T.th0[k] = fmin(fmax(th, 1e-6), pi_ - 1e-6);
        }
    }
}

struct RefArgs {
    PairIn pi;
    const RTask *tasks;
    SurCtrl *sc;
    Cand *cand;
    int *cok, *qflag;
    PfCtrl *ctrl;
    double h0, tol, step0, max_step;
    int32_t iters, deflate;
};

// Root searches on the launch angle, one lane per query, slot 0 first: from the network's
// launch angle, one full trace per step, secant steps (the second point at launch + step0,
// steps clamped to max_step) until two misses of opposite sign bracket the root, then Illinois
// false position inside the bracket, until |miss| < tol.  Slot 1's search runs on the deflated
// miss, miss / (launch - r0), where r0 is the root slot 0 found, so it cannot converge to that
// ray again.  A ray that exhausts its path budget (far below the receiver) sends the search
// halfway back to the previous angle.  Any other end short of the receiver plane, a step
// leaving (0, pi), or `iters` traces without convergence send the query to the path finder.
template <class P>
__global__ void __launch_bounds__(128, P::kMinBlocks)
    k_refine(const MediumLayered med, const StepParams<P> sp, const Sinks sk, const RefArgs a)
{
    const long long nt = (long long)a.sc->n_tasks;
    const double pi_ = 3.14159265358979323846;
    long long q = 0;
    int slot = 0, mask = 0, it = 0, side = 0;
    bool br = false, have_prev = false, defl = false, resume = false, next_slot = false;
    double th_prev = 0.0, m_prev = 0.0, raw_prev = 0.0, th_cur = 0.0;
    double ta = 0.0, ma = 0.0, tb = 0.0, mb = 0.0, th_d = 0.0, th1 = 0.0;
    auto fail = [&](unsigned long long *why) {
        a.qflag[q] = 1;
        atomicAdd(&a.sc->failed, 1ull);
        atomicAdd(why, 1ull);
        next_slot = false;
    };
    auto start = [&](Lane<P> &L, int k, double th, bool deflated, double r) {
        slot = k;
        th_cur = th;
        defl = deflated;
        th_d = r;
        it = 0;
        side = 0;
        br = false;
        have_prev = false;
        launch_ray<P>(L, med, sp, a.pi, a.h0, q, th_cur, false, -1);
    };
    auto next = [&](Lane<P> &L) -> bool {
        if (resume) {
            resume = false;
            launch_ray<P>(L, med, sp, a.pi, a.h0, q, th_cur, false, -1);
            return true;
        }
        if (next_slot) {  // slot 1 after slot 0 converged
            next_slot = false;
            const double r0 = a.cand[2 * q].launch;
            double th = th1;
            if (a.deflate && fabs(th - r0) < 1e-3) th = r0 + copysign(1e-3, th - r0);
            if (a.deflate) atomicAdd(&a.sc->deflated, 1ull);
            start(L, 1, fmin(fmax(th, 1e-6), pi_ - 1e-6), a.deflate != 0, r0);
            return true;
        }
        const long long t = pf_claim(&a.sc->claim);
        if (t >= nt) return false;
        const RTask &T = a.tasks[t];
        q = T.q;
        mask = T.mask;
        th1 = T.th0[1];
        start(L, 0, T.th0[0], false, 0.0);
        return true;
    };
    auto done = [&](Lane<P> &L) {
        const double m = miss_of<P>(L, a.pi.zr[q]);
        if (isnan(m) || (isinf(m) && !have_prev)) {
            fail(&a.sc->fail_end);
            return;
        }
        if (fabs(m) < a.tol) {
            Cand &o = a.cand[2 * q + slot];
            o.type = L.n_refl > 0 ? RP_SOL_REFLECTED
                                  : (L.n_turn > 0 ? RP_SOL_REFRACTED : RP_SOL_DIRECT);
            o.n_iter = it + 1;
            o.launch = th_cur;
            o.receive = acos(fmax(-1.0, fmin(1.0, P::get(L.t, 2))));
            o.time = P::sget(L.T);
            o.path = P::sget(L.s);
            o.amp = L.A;
            o.miss = m;
            o.dth = have_prev ? a.tol * fabs((th_cur - th_prev) / (m - raw_prev)) : 0.0;
            a.cok[2 * q + slot] = SLOT_OK;
            next_slot = slot == 0 && (mask & 2);
            return;
        }
        ++it;
        if (it >= a.iters) {
            fail(&a.sc->fail_iters);
            return;
        }
        double th_new;
        if (isinf(m)) {  // far below: back toward the last angle that reached the receiver plane
            th_new = 0.5 * (th_cur + th_prev);
        } else {
            double g = m;
            if (defl) {
                const double d = th_cur - th_d;
                if (fabs(d) < 1e-12) {
                    fail(&a.sc->fail_step);
                    return;
                }
                g = m / d;
            }
            if (br) {  // th_cur lies inside the bracket: keep the end of opposite sign
                if ((g > 0.0) == (ma > 0.0)) {
                    ta = th_cur;
                    ma = g;
                    if (side == -1) mb *= 0.5;
                    side = -1;
                } else {
                    tb = th_cur;
                    mb = g;
                    if (side == 1) ma *= 0.5;
                    side = 1;
                }
                th_new = (ta * mb - tb * ma) / (mb - ma);
            } else if (!have_prev) {
                th_new = th_cur + a.step0;
            } else if ((g > 0.0) != (m_prev > 0.0)) {
                br = true;
                ta = th_prev;
                ma = m_prev;
                tb = th_cur;
                mb = g;
                side = 0;
                th_new = (ta * mb - tb * ma) / (mb - ma);
            } else {
                th_new = th_cur - g * (th_cur - th_prev) / (g - m_prev);
                if (isfinite(th_new) && fabs(th_new - th_cur) > a.max_step)
                    th_new = th_cur + copysign(a.max_step, th_new - th_cur);
            }
            th_prev = th_cur;
            m_prev = g;  // the searched function: the miss, or the deflated miss
            raw_prev = m;
            have_prev = true;
        }
        if (!(th_new > 0.0 && th_new < pi_)) {
            fail(&a.sc->fail_step);
            return;
        }
        th_cur = th_new;
        resume = true;
    };
    drive<P>(med, sp, sk, a.ctrl, next, done);
}

// two refined slots of a pair land on the same ray: same type, launch angles within twice the
// sum of their uncertainties (at least 1e-5 rad)
__device__ __forceinline__ bool same_ray(const Cand &A, const Cand &B)
{
    return A.type == B.type && fabs(A.launch - B.launch) <= fmax(1e-5, 2.0 * (A.dth + B.dth));
}

// Queries served by the network: their refined slots sorted by travel time into the outputs;
// a failed slot, or two slots on the same ray, send the query to the fallback list.
__global__ void k_collect(long long n, int max_sol, const int *cok, const Cand *cand,
                          const int *qflag, rp_solutions sol, long long *fb, SurCtrl *sc)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        bool to_fb = qflag[i] != 0;
        int cnt = 0;
        int idx[2] = {0, 0};
        if (!to_fb) {
            for (int k = 0; k < 2; ++k) {
                if (cok[2 * i + k] == SLOT_PENDING) to_fb = true;
                if (cok[2 * i + k] == SLOT_OK) idx[cnt++] = k;
            }
            if (!to_fb && cnt == 2 && same_ray(cand[2 * i], cand[2 * i + 1])) {
                to_fb = true;
                atomicAdd(&sc->duplicates, 1ull);
            }
        }
        if (to_fb) {
            const unsigned long long f = atomicAdd(&sc->n_fallback, 1ull);
            fb[f] = i;
            continue;
        }
        if (cnt == 2 && cand[2 * i + idx[1]].time < cand[2 * i + idx[0]].time) {
            const int tmp = idx[0];
            idx[0] = idx[1];
            idx[1] = tmp;
        }
        const int keep = cnt < max_sol ? cnt : max_sol;
        sol.count[i] = keep;
        for (int c = 0; c < max_sol; ++c) {
            const long long o = i * max_sol + c;
            const bool has = c < keep;
            const Cand &X = cand[2 * i + (has ? idx[c] : 0)];
            if (sol.type) sol.type[o] = has ? X.type : 0;
            if (sol.n_iter) sol.n_iter[o] = has ? X.n_iter : 0;
            if (sol.launch) sol.launch[o] = has ? X.launch : 0.0;
            if (sol.receive) sol.receive[o] = has ? X.receive : 0.0;
            if (sol.time) sol.time[o] = has ? X.time : 0.0;
            if (sol.path) sol.path[o] = has ? X.path : 0.0;
            if (sol.amp) sol.amp[o] = has ? X.amp : 0.0;
            if (sol.miss) sol.miss[o] = has ? X.miss : 0.0;
        }
    }
}

__global__ void k_gather(const long long *fb, long long nf, const PairIn pi, double *zs, double *zr,
                         double *D, int32_t *na)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nf;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = fb[j];
        zs[j] = pi.zs[i];
        zr[j] = pi.zr[i];
        D[j] = pi.dist[i];
        na[j] = pi.n_angles[i];
    }
}

__global__ void k_scatter(const long long *fb, long long nf, int max_sol, const rp_solutions src,
                          rp_solutions dst)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nf;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = fb[j];
        dst.count[i] = src.count[j];
        for (int c = 0; c < max_sol; ++c) {
            const long long o = i * max_sol + c, p = j * max_sol + c;
            if (dst.type) dst.type[o] = src.type[p];
            if (dst.n_iter) dst.n_iter[o] = src.n_iter[p];
            if (dst.launch) dst.launch[o] = src.launch[p];
            if (dst.receive) dst.receive[o] = src.receive[p];
            if (dst.time) dst.time[o] = src.time[p];
            if (dst.path) dst.path[o] = src.path[p];
            if (dst.amp) dst.amp[o] = src.amp[p];
            if (dst.miss) dst.miss[o] = src.miss[p];
        }
    }
}

// device buffers of the pipeline, grown on demand, owned by the surrogate handle
struct SurPipe {
    long long cap = 0;
    float *x = nullptr, *out = nullptr;
    RTask *tasks = nullptr;
    Cand *cand = nullptr;
    int *cok = nullptr, *qflag = nullptr;
    long long *fb = nullptr;
    double *zs = nullptr, *zr = nullptr, *D = nullptr;
    int32_t *na = nullptr;
    rp_solutions tmp;
    int32_t *tmp_i[3] = {nullptr, nullptr, nullptr};
    double *tmp_d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    SurCtrl *sc = nullptr;
    PfCtrl *pc = nullptr;
    Ctrl *tc = nullptr;
};

void pipe_free(SurPipe *p)
{
    if (!p) return;
    cudaFree(p->x);
    cudaFree(p->out);
    cudaFree(p->tasks);
    cudaFree(p->cand);
    cudaFree(p->cok);
    cudaFree(p->qflag);
    cudaFree(p->fb);
    cudaFree(p->zs);
    cudaFree(p->zr);
    cudaFree(p->D);
    cudaFree(p->na);
    for (int k = 0; k < 3; ++k) cudaFree(p->tmp_i[k]);
    for (int k = 0; k < 6; ++k) cudaFree(p->tmp_d[k]);
    cudaFree(p->sc);
    cudaFree(p->pc);
    cudaFree(p->tc);
    delete p;
}

int pipe_ensure(rp_surrogate_s *s, long long n, int max_sol)
{
    SurPipe *p = (SurPipe *)s->pipe;
    if (p && p->cap >= n) return RP_OK;
    RP_CUDA_TRY(cudaDeviceSynchronize());
    pipe_free(p);
    s->pipe = nullptr;
    p = new SurPipe();
    s->pipe = p;
    const long long c = n + n / 4 + 16;
    p->cap = c;
    RP_CUDA_TRY(cudaMalloc(&p->x, sizeof(float) * 3 * c));
    RP_CUDA_TRY(cudaMalloc(&p->out, sizeof(float) * 12 * c));
    RP_CUDA_TRY(cudaMalloc(&p->tasks, sizeof(RTask) * c));
    RP_CUDA_TRY(cudaMalloc(&p->cand, sizeof(Cand) * 2 * c));
    RP_CUDA_TRY(cudaMalloc(&p->cok, sizeof(int) * 2 * c));
    RP_CUDA_TRY(cudaMalloc(&p->qflag, sizeof(int) * c));
    RP_CUDA_TRY(cudaMalloc(&p->fb, sizeof(long long) * c));
    RP_CUDA_TRY(cudaMalloc(&p->zs, sizeof(double) * c));
    RP_CUDA_TRY(cudaMalloc(&p->zr, sizeof(double) * c));
    RP_CUDA_TRY(cudaMalloc(&p->D, sizeof(double) * c));
    RP_CUDA_TRY(cudaMalloc(&p->na, sizeof(int32_t) * c));
    RP_CUDA_TRY(cudaMalloc(&p->tmp_i[0], sizeof(int32_t) * c));
    RP_CUDA_TRY(cudaMalloc(&p->tmp_i[1], sizeof(int32_t) * c * 8));
    RP_CUDA_TRY(cudaMalloc(&p->tmp_i[2], sizeof(int32_t) * c * 8));
    for (int k = 0; k < 6; ++k) RP_CUDA_TRY(cudaMalloc(&p->tmp_d[k], sizeof(double) * c * 8));
    RP_CUDA_TRY(cudaMalloc(&p->sc, sizeof(SurCtrl)));
    RP_CUDA_TRY(cudaMalloc(&p->pc, sizeof(PfCtrl)));
    RP_CUDA_TRY(cudaMalloc(&p->tc, sizeof(Ctrl)));
    p->tmp.count = p->tmp_i[0];
    p->tmp.type = p->tmp_i[1];
    p->tmp.n_iter = p->tmp_i[2];
    p->tmp.launch = p->tmp_d[0];
    p->tmp.receive = p->tmp_d[1];
    p->tmp.time = p->tmp_d[2];
    p->tmp.path = p->tmp_d[3];
    p->tmp.amp = p->tmp_d[4];
    p->tmp.miss = p->tmp_d[5];
    (void)max_sol;
    return RP_OK;
}

template <class P>
int run_surrogate(rp_surrogate_s *s, rp_medium_t m, const PairIn &pi, const rp_trace_params *tp,
                  const rp_surrogate_params *sp_in, rp_solutions *sol, rp_surrogate_stats *stats,
                  cudaStream_t st, int dev)
{
    const long long n = pi.n_pairs;
    int rc = pipe_ensure(s, n, pi.max_sol);
    if (rc) return rc;
    SurPipe *p = (SurPipe *)s->pipe;
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; ++k) RP_CUDA_TRY(cudaEventCreate(&ev[k]));
    const int sms = sm_count(dev);
    const int gblocks = std::max(1, (int)std::min<long long>((n + 255) / 256, (long long)sms * 8));
    RP_CUDA_TRY(cudaEventRecord(ev[0], st));
    RP_CUDA_TRY(cudaMemsetAsync(p->sc, 0, sizeof(SurCtrl), st));
    RP_CUDA_TRY(cudaMemsetAsync(p->pc, 0, sizeof(PfCtrl), st));
    RP_CUDA_TRY(cudaMemsetAsync(p->tc, 0, sizeof(Ctrl), st));
    rp_solutions none;
    memset(&none, 0, sizeof none);
    k_encode<<<gblocks, 256, 0, st>>>(n, pi.zs, pi.zr, pi.dist, none, 0, p->x, nullptr, nullptr);
    RP_CUDA_TRY(cudaGetLastError());
    if ((rc = forward_fused(s, n, p->x, p->out, st))) return rc;
    RP_CUDA_TRY(cudaEventRecord(ev[1], st));
    k_plan<<<gblocks, 256, 0, st>>>(n, p->out, sp_in->conf, pi, p->tasks, p->sc, p->qflag, p->cok);
    RP_CUDA_TRY(cudaGetLastError());
    StepParams<P> sp = step_params<P>(tp, 0, 1.0f);
    sp.use_stop = 1;
    sp.max_generation = 0;
    Sinks sk;
    memset(&sk, 0, sizeof sk);
    sk.ctrl = p->tc;
    RefArgs ra;
    ra.pi = pi;
    ra.tasks = p->tasks;
    ra.sc = p->sc;
    ra.cand = p->cand;
    ra.cok = p->cok;
    ra.qflag = p->qflag;
    ra.ctrl = p->pc;
    ra.h0 = tp->h0;
    ra.tol = sp_in->refine_tol;
    ra.step0 = sp_in->refine_step;
    ra.max_step = sp_in->max_step;
    ra.iters = sp_in->refine_iters;
    ra.deflate = sp_in->deflate;
    const int occ = occ_of((const void *)k_refine<P>);
    if (occ < 0) return occ;
    k_refine<P><<<sms * occ, 128, 0, st>>>(m->layered, sp, sk, ra);
    RP_CUDA_TRY(cudaGetLastError());
    k_collect<<<gblocks, 256, 0, st>>>(n, pi.max_sol, p->cok, p->cand, p->qflag, *sol, p->fb,
                                       p->sc);
    RP_CUDA_TRY(cudaGetLastError());
    RP_CUDA_TRY(cudaEventRecord(ev[2], st));
    SurCtrl hs;
    PfCtrl hp;
    RP_CUDA_TRY(cudaMemcpyAsync(&hs, p->sc, sizeof hs, cudaMemcpyDeviceToHost, st));
    RP_CUDA_TRY(cudaMemcpyAsync(&hp, p->pc, sizeof hp, cudaMemcpyDeviceToHost, st));
    if ((rc = fused_status(s, st))) return rc;  // synchronises the stream
    const long long nf = (long long)hs.n_fallback;
    rp_stats fs;
    memset(&fs, 0, sizeof fs);
    if (nf > 0) {
        k_gather<<<std::max(1, (int)std::min<long long>((nf + 255) / 256, (long long)sms * 8)), 256,
                   0, st>>>(p->fb, nf, pi, p->zs, p->zr, p->D, p->na);
        RP_CUDA_TRY(cudaGetLastError());
        PairIn sub = pi;
        sub.zs = p->zs;
        sub.zr = p->zr;
        sub.dist = p->D;
        sub.n_angles = p->na;
        sub.n_pairs = nf;
        rc = run_pf<P>(m, sub, tp, &p->tmp, &fs, st, dev);
        if (rc && rc != RP_ERR_OVERFLOW) return rc;
        k_scatter<<<std::max(1, (int)std::min<long long>((nf + 255) / 256, (long long)sms * 8)), 256,
                    0, st>>>(p->fb, nf, pi.max_sol, p->tmp, *sol);
        RP_CUDA_TRY(cudaGetLastError());
    }
    RP_CUDA_TRY(cudaEventRecord(ev[3], st));
    RP_CUDA_TRY(cudaEventSynchronize(ev[3]));
    float t_fwd = 0, t_ref = 0, t_all = 0;
    cudaEventElapsedTime(&t_fwd, ev[0], ev[1]);
    cudaEventElapsedTime(&t_ref, ev[1], ev[2]);
    cudaEventElapsedTime(&t_all, ev[0], ev[3]);
    for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
    if (stats) {
        stats->queries = n;
        stats->fallback = nf;
        stats->tasks = (int64_t)hs.n_tasks;
        stats->tasks_failed = (int64_t)hs.failed;
        stats->fail_end = (int64_t)hs.fail_end;
        stats->fail_iters = (int64_t)hs.fail_iters;
        stats->fail_step = (int64_t)hs.fail_step;
        stats->duplicates = (int64_t)hs.duplicates;
        stats->deflated = (int64_t)hs.deflated;
        stats->refine_rays = (int64_t)hp.rays;
        stats->refine_steps = (int64_t)hp.steps_acc;
        stats->fallback_rays = fs.rays;
        stats->fallback_steps = fs.steps_accepted;
        stats->ms_forward = t_fwd;
        stats->ms_refine = t_ref;
        stats->ms_total = t_all;
        stats->ms_fallback = t_all - t_fwd - t_ref;
        stats->ms_fallback_scan = fs.wave_ms[0];
    }
    return rc;
}

}  // namespace

void free_pipe(rp_surrogate_s *s)
{
    if (s && s->pipe) {
        pipe_free((SurPipe *)s->pipe);
        s->pipe = nullptr;
    }
}

int run_surrogate_paths(rp_surrogate_s *s, rp_medium_t m, int64_t n, const double *zs,
                        const double *zr, const double *dist, const int32_t *n_angles,
                        const rp_path_params *p, const rp_surrogate_params *sp,
                        rp_solutions *sol, rp_surrogate_stats *stats, cudaStream_t st)
{
    if (!s || !m || !p || !sp || !sol || n < 0 || medium_variant(m) != VARIANT_LAYERED) {
        set_error("rp_surrogate_find_paths: bad arguments (a layered medium with horizontal "
                  "boundaries and no spheres required)");
        return RP_ERR_INVALID_ARG;
    }
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) return RP_OK;
    if (!zs || !zr || !dist || !n_angles || !sol->count || p->max_sol < 2 || p->max_sol > 8 ||
        !(sp->conf > 0.5 && sp->conf < 1.0) || !(sp->refine_tol > 0.0) || sp->refine_iters < 1 ||
        !(sp->refine_step > 0.0) || !(sp->max_step > 0.0) || !(p->hit_tol > 0.0) ||
        (sp->deflate != 0 && sp->deflate != 1)) {
        set_error("rp_surrogate_find_paths: bad arrays or parameters (max_sol 2..8, 0.5 < conf < 1)");
        return RP_ERR_INVALID_ARG;
    }
    int rc = validate_params(&p->trace, true);
    if (rc) return rc;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device || dev != s->device) {
        set_error("rp_surrogate_find_paths: medium (device %d), network (device %d) and current "
                  "device %d differ", m->device, s->device, dev);
        return RP_ERR_INVALID_ARG;
    }
    PairIn pi;
    pi.zs = zs;
    pi.zr = zr;
    pi.dist = dist;
    pi.n_angles = n_angles;
    pi.n_pairs = n;
    pi.hit_tol = p->hit_tol;
    pi.max_iter = p->max_iter;
    pi.max_sol = p->max_sol;
    if (p->trace.precision == RP_FP64)
        return run_surrogate<PrecF64>(s, m, pi, &p->trace, sp, sol, stats, st, dev);
    return run_surrogate<PrecF32>(s, m, pi, &p->trace, sp, sol, stats, st, dev);
}

int run_surrogate_encode(int64_t n, const double *zs, const double *zr, const double *dist,
                         const rp_solutions *sol, int max_sol, float *x, float *y, float *t,
                         cudaStream_t st)
{
    if (n < 0 || (n > 0 && (!zs || !zr || !dist || !x)) || (y && (!t || !sol || !sol->count)) ||
        (y && max_sol < 2)) {
        set_error("rp_surrogate_encode: bad arguments");
        return RP_ERR_INVALID_ARG;
    }
    if (n == 0) return RP_OK;
    rp_solutions none;
    memset(&none, 0, sizeof none);
    k_encode<<<std::max(1, (int)std::min<long long>((n + 255) / 256, 4096)), 256, 0, st>>>(
        n, zs, zr, dist, y ? *sol : none, max_sol, x, y, t);
    RP_CUDA_TRY(cudaGetLastError());
    RP_CUDA_TRY(cudaStreamSynchronize(st));
    return RP_OK;
}

int run_find_paths(rp_medium_t m, int64_t n_pairs, const double *zs, const double *zr,
                   const double *dist, const int32_t *n_angles, const rp_path_params *p,
                   rp_solutions *sol, rp_stats *stats, cudaStream_t st)
{
    if (!m || !p || !sol || n_pairs < 0) {
        set_error("rp_find_paths: null medium, params or solutions, or n_pairs < 0");
        return RP_ERR_INVALID_ARG;
    }
    if (medium_variant(m) != VARIANT_LAYERED) {
        set_error("rp_find_paths: path finding needs a layered medium with horizontal "
                  "boundaries and no spheres");
        return RP_ERR_INVALID_ARG;
    }
    if (n_pairs == 0) return RP_OK;
    if (!zs || !zr || !dist || !n_angles || !sol->count) {
        set_error("rp_find_paths: null pair or count array");
        return RP_ERR_INVALID_ARG;
    }
    if (!(p->hit_tol > 0.0) || p->max_iter < 1 || p->max_iter > 200 || p->max_sol < 1 ||
        p->max_sol > 8) {
        set_error("rp_find_paths: need hit_tol > 0, 1 <= max_iter <= 200, 1 <= max_sol <= 8");
        return RP_ERR_INVALID_ARG;
    }
    int rc = validate_params(&p->trace, true);
    if (rc) return rc;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device) {
        set_error("rp_find_paths: medium lives on device %d, current device is %d", m->device, dev);
        return RP_ERR_INVALID_ARG;
    }
    PairIn pi;
    pi.zs = zs;
    pi.zr = zr;
    pi.dist = dist;
    pi.n_angles = n_angles;
    pi.n_pairs = n_pairs;
    pi.hit_tol = p->hit_tol;
    pi.max_iter = p->max_iter;
    pi.max_sol = p->max_sol;
    if (p->trace.precision == RP_FP64)
        return run_pf<PrecF64>(m, pi, &p->trace, sol, stats, st, dev);
    return run_pf<PrecF32>(m, pi, &p->trace, sol, stats, st, dev);
}

}  // namespace rph
