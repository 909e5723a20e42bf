// mlp_train_fused.cu -- one training step of the surrogate network in two fused tensor-core
// kernels per batch: the whole forward pass with the loss and the last layer's backward pass,
// then the backward-data chain through the three hidden layers.
//
// Both kernels run clusters of two CTAs (512 threads each); a cluster takes one tile of 128
// rows at a time and CTA h of the pair (its rank in the cluster) computes output columns
// 128 h .. 128 h + 127 of every 256-wide layer: 16 tcgen05.mma of M 128, N 128, K 16 from the
// whole 128 x 256 BF16 A tile and its half of the layer's B image (bulk-copied, 64 KB) into a
// 128-column TMEM accumulator, then an epilogue by sixteen warps.  The epilogue writes its half
// of the layer's output, in BF16, into its own next A tile, and one thread copies that half
// (32 KB, contiguous) into the peer's (a shared-to-shared bulk copy that completes on an
// mbarrier of the peer), so that each CTA holds the whole next A tile without a cluster-wide
// barrier.  The A tile is double-buffered (the MMAs read one buffer while the epilogue fills
// the other) with one exchange barrier per buffer; a CTA sends a layer's half only after its
// MMAs used the peer's half of the layer before, which the peer sent after its own MMAs had
// read the buffer the new half goes to, so no copy lands in a buffer still being read.
//
// k_train_fwd: layer 0 (3 -> 256) as one MMA of K = 16 (x zero-padded, from a 16-column A
//   operand the CTA writes), then the three 256 -> 256 layers.  An epilogue evaluates GELU and
//   its derivative from one Phi and one density, and also stores what the later kernels
//   read: gelu'(z) of the pre-activations z0..z2 in BF16 (tiled: a tile's 8 columns k..k+7 of
//   its 128 rows are 2 KB contiguous, so a warp's stores of one 8-column group are 512 B
//   contiguous and a CTA's 128 columns are one 32 KB block) and the activations H1..H4 as BF16 operand images
//   (tc_common.cuh), and x as a 16-column image.  The last layer (256 -> 12) is 16 MMAs of
//   N = 16 (outputs zero-padded) from the whole H4 tile, done alike by both CTAs; the loss and
//   its gradient g4 follow per row (g4 stored as a 16-column image, its column sums added to
//   db4), and the last layer's backward data pass g3 = (g4 W4^T) gelu'(z3) is one MMA of K = 16
//   from g4 for the CTA's 128 columns, with gelu'(z3) written into tensor memory over z3 by the
//   fourth epilogue; g3 is stored as a BF16 image and its column sums are added to the bias
//   gradient db3.
// k_train_bwd: per tile, the g3 image by bulk copy as the A tile (prefetched while the previous
//   tile's last epilogue runs), then for the hidden layers
//   3, 2, 1 the backward images B[n][k] = W[n][k], gelu'(z) of the CTA's columns by bulk copy
//   while the MMAs run, and an epilogue
//   g_{l-1} = (g_l W_l^T) gelu'(z_{l-1}) that stores g_{l-1} as a BF16 image, adds its column
//   sums to db_{l-1} and, but for the last, feeds it to both CTAs' next A tile.
// Arithmetic is that of the per-layer path: BF16 operands (weights, activations and
// gradients rounded to BF16 where they enter a product, gelu'(z) rounded to BF16 between the
// passes), FP32 products and sums, FP32 bias, GELU and GELU'; bias gradients are sums of the
// FP32 g before its rounding.  A batch's last, partial
// tile is computed whole: its rows past n have zero output gradients, so they add nothing to
// any gradient.
// Synchronisation and failure: every mbarrier wait is bounded (the surrogate's wait limit).
// A CTA whose wait gives up sets the error flag and skips all further work (sending no more
// halves).  Before it exits each CTA waits (with the default bound) for the copies and MMAs it
// issued, tells its peer how many halves it sent, waits for the peer's halves it has not
// consumed, and passes a last cluster barrier, so that no CTA leaves while a copy into its
// shared memory is in flight; the two CTAs pass the same three cluster barriers (one at the
// start, two at the end) whatever happens.
#include <cuda_bf16.h>

#include <algorithm>

#include "rp_internal.h"
#include "tc_common.cuh"

namespace rph {

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kThreads = 512;  // 16 warps: lane quarter (warp % 4) x column group (warp / 4)
constexpr int kHalf = 128;     // output columns of a CTA
constexpr int kGroups = kThreads / 128;     // column groups of a row
constexpr int kGroupCols = kHalf / kGroups; // 32: one TMEM load per warp
constexpr uint32_t kHalfImage = kImage;     // bytes of a half B image (N 128 x K 256, BF16)
// shared memory map (bytes): A tiles 0 and 1, the half B image, barriers, then per kernel
constexpr uint32_t SM_A0 = 0;
constexpr uint32_t SM_A1 = 65536;
constexpr uint32_t SM_B = 131072;
// barriers: B image, MMAs, A tile / W0 image, the peer's halves of A tiles 0 and 1, gelu'(z)
constexpr uint32_t SM_BAR = SM_B + kHalfImage;
constexpr uint32_t SM_SLOT = SM_BAR + 48;  // TMEM address, abort word; the peer's sent count, failure
constexpr uint32_t SM_OWN = SM_BAR + 1024;
// forward: the FP32 constants, the CTA's half of the W0 image (4 KB) and the x operand (128
// rows x 16, 4 KB)
constexpr uint32_t SM_F = SM_OWN;
constexpr uint32_t SM_W0 = (SM_F + kPackF * 4 + 1023) / 1024 * 1024;
constexpr uint32_t SM_XA = SM_W0 + 4096;
constexpr uint32_t SM_TOTAL_FWD = SM_XA + 4096;
// backward: gelu'(z) of the tile's rows and the CTA's 128 columns (BF16, 16 groups of 2 KB)
constexpr uint32_t SM_DZ = SM_OWN;
constexpr uint32_t SM_TOTAL_BWD = SM_DZ + 32768;
static_assert(SM_TOTAL_FWD <= 227 * 1024 && SM_TOTAL_BWD <= 227 * 1024,
              "shared memory map exceeds a CTA's limit");
static_assert(SM_F % 16 == 0 && SM_DZ % 16 == 0 && SM_BAR % 8 == 0, "alignment");
static_assert(PF_B0 % 4 == 0 && PF_B1 % 4 == 0, "bias blocks load as float4");

// instruction descriptors: D FP32, A and B BF16, both K-major, M = 128; N = 128 (a CTA's
// columns of a layer) and N = 16 (the last layer, 12 outputs zero-padded)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);
constexpr uint32_t kIdescN16 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) |
                               ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// the shared::cluster address of the same location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// All threads of both CTAs (at the start and the end of a kernel only): memory accesses of
// either CTA before it happen before those after it.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
    fence_before();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
    fence_after();
}

// the CTA's half (output columns 128 h ..) of a 256 x 256 B image: 64 KB contiguous in the
// half-major image (bimg_off), laid out like the A tile (K groups 2 KB apart)
__device__ __forceinline__ void load_half_image(uint32_t b_base, const unsigned char *img, int h,
                                                uint32_t bar)
{
    mbar_expect(bar, kHalfImage);
    bulk_g2s(b_base, img + h * 65536, 32768u, bar);
    bulk_g2s(b_base + 32768u, img + h * 65536 + 32768, 32768u, bar);
}

// K steps s0 .. s0 + 7 (16 K each) of one layer (A tile x half B image) into the accumulator;
// the first of them starts the accumulation if `fresh`
__device__ __forceinline__ void issue_ksteps(uint32_t tmem, uint32_t a_base, uint32_t b_base,
                                             int s0, bool fresh)
{
    // a K step is 4 KB further on in both operands: 256 in the descriptors' address field
    // (address / 16, 14 bits, which shared addresses below 256 KB never carry out of)
    const uint64_t ad0 = sdesc(a_base + s0 * 4096u, 2048u, 128u);
    const uint64_t bd0 = sdesc(b_base + s0 * 4096u, 2048u, 128u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint64_t ad = ad0 + (uint64_t)(i * 256);
        const uint64_t bd = bd0 + (uint64_t)(i * 256);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"((uint32_t)(!fresh || i > 0))
            : "memory");
    }
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}
// byte offset of the 8 BF16 values of columns k0..k0+7 (k0 % 8 == 0) of row `row` of tile
// `tile` in a tiled gelu'(z) buffer: 2 KB per 8-column group, the groups in column order
__device__ __forceinline__ long long zb_off(long long tile, int row, int k0)
{
    return tile * 65536LL + (long long)(k0 >> 3) * 2048 + row * 16;
}

// One CTA's state of the bounded waits: whether a copy (or MMAs) is in flight and the phase
// its completion has; and of the exchange with the peer (thread 0 only): copy c of the
// sequence of halves sent each way goes to A tile (c + off) % 2 and completes phase c / 2 of
// barrier 3 + (c + off) % 2 of the receiver.
struct Pending {
    bool ld = false, mma = false, a = false, dz = false;
    uint32_t ph_ld = 0, ph_mma = 0, ph_a = 0, ph_dz = 0;
    long long sent = 0, recv = 0;
    int off = 0;
};

// Shared setup of both kernels: barriers (each exchange barrier armed for its first copy),
// abort word, `cols` columns of tensor memory, then a cluster barrier (the peer's shared memory
// is in use only after it).
__device__ __forceinline__ uint32_t setup_cta(unsigned char *sm, int tid, int warp, uint32_t cols)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + SM_SLOT);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    if (tid == 0) {
        for (int b = 0; b < 6; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect(su32(&bar[3]), kImage / 2);
        mbar_expect(su32(&bar[4]), kImage / 2);
        *abort_cta = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *slot;
    cluster_sync();
    return tmem;
}

// Thread 0, after every thread wrote its part of this CTA's half (columns 128 h ..) of A tile
// `buf` and passed a proxy fence and a CTA barrier: the half (32 KB, contiguous) to the same
// place in the peer, completing on the peer's exchange barrier of that tile.
__device__ __forceinline__ void send_half(Pending &pd, uint32_t local, uint32_t remote,
                                          uint32_t remote_bar0, int buf, int h)
{
    const uint32_t o = (uint32_t)buf * 65536u + (uint32_t)h * 32768u;
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            remote + o),
        "r"(local + o), "r"(32768u), "r"(remote_bar0 + (uint32_t)buf * 8u)
        : "memory");
    ++pd.sent;
}

// Thread 0: wait for the peer's next half (bounded); then arm its barrier for the copy after
// next.  The peer sends a copy only after it used the one this CTA sent before (each layer's
// MMAs need both halves of their input), so the copy after next finds the barrier armed for
// it, and a tile's buffer is never overwritten while this CTA's MMAs may still read it.
__device__ __forceinline__ bool recv_half(Pending &pd, unsigned char *sm, long long wait)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    const long long c = pd.recv;
    const uint32_t xb = su32(&bar[3 + ((c + pd.off) & 1)]);
    if (!mbar_wait(xb, (uint32_t)((c >> 1) & 1), wait)) return false;
    ++pd.recv;
    mbar_expect(xb, kImage / 2);
    return true;
}

// the last layer's two images into the B region: the forward image (8 KB) at b_base and the
// CTA's half of the backward image (two K groups of 2 KB, 2 KB apart) at b_base + 8 KB
__device__ __forceinline__ void load_w4(uint32_t b_base, const unsigned char *pack, int h,
                                        uint32_t bar)
{
    mbar_expect(bar, 8192u + 4096u);
    bulk_g2s(b_base, pack + kPackW4F, 8192u, bar);
    for (int kg = 0; kg < 2; ++kg)
        bulk_g2s(b_base + 8192u + kg * 2048u, pack + kPackW4B + kg * 4096 + h * 2048, 2048u, bar);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// What thread 0 copies into the B region once a layer's MMAs are done.
enum { NEXT_NONE = 0, NEXT_HALF = 1, NEXT_W4 = 2 };

// Thread 0: wait for the B image, issue the layer's MMAs from A tile `a_base` (first the K steps
// over this CTA's own half of the input, then, once the peer's half has arrived if `exchange`,
// the others), wait for them and start the next copy into the B region (a half image of `img`,
// the last layer's images from the pack `img`, or none); false once a wait gives up (MMAs
// issued are committed first, so that the drain can wait for them).
__device__ __forceinline__ bool run_layer(Pending &pd, unsigned char *sm, uint32_t tmem,
                                          uint32_t a_base, uint32_t b_base, uint32_t bar_ld,
                                          uint32_t bar_mma, int next, const unsigned char *img,
                                          int h, bool exchange, long long wait)
{
    if (!mbar_wait(bar_ld, pd.ph_ld, wait)) return false;
    pd.ld = false;
    pd.ph_ld ^= 1u;
    issue_ksteps(tmem, a_base, b_base, 8 * h, true);
    pd.mma = true;
    if (exchange && !recv_half(pd, sm, wait)) {
        mma_commit(bar_mma);
        return false;
    }
    issue_ksteps(tmem, a_base, b_base, 8 * (h ^ 1), false);
    mma_commit(bar_mma);
    if (!mbar_wait(bar_mma, pd.ph_mma, wait)) return false;
    pd.mma = false;
    pd.ph_mma ^= 1u;
    if (next == NEXT_HALF) load_half_image(b_base, img, h, bar_ld);
    if (next == NEXT_W4) load_w4(b_base, img, h, bar_ld);
    pd.ld = next != NEXT_NONE;
    return true;
}

// Shared teardown: on failure record it and drain the issued work (default bound); then tell
// the peer how many halves this CTA sent it and whether it failed, and pass a cluster barrier.
// Without a failure in the cluster each CTA has waited for every half the peer sent (each
// layer's MMAs wait for the peer's half of their input), so no copy is in flight any more.
// After a failure each CTA waits (default bound) for the halves the peer sent that it has not
// waited for, and passes a second cluster barrier, so that no CTA leaves while a copy into or
// out of its shared memory is in flight; both CTAs take the same branch, as both know both
// failure flags.  Then tensor memory is freed.
__device__ __forceinline__ void teardown_cta(unsigned char *sm, int tid, int warp, uint32_t tmem,
                                             uint32_t cols, bool failed, Pending &pd, int *flag,
                                             uint32_t remote)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    if (tid == 0) {
        if (failed) atomicExch(flag, 1);
        if (pd.ld) mbar_wait(su32(&bar[0]), pd.ph_ld);
        if (pd.mma) mbar_wait(su32(&bar[1]), pd.ph_mma);
        if (pd.a) mbar_wait(su32(&bar[2]), pd.ph_a);
        if (pd.dz) mbar_wait(su32(&bar[5]), pd.ph_dz);
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote + SM_SLOT + 8),
                     "r"((uint32_t)pd.sent)
                     : "memory");
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote + SM_SLOT + 12),
                     "r"((uint32_t)failed)
                     : "memory");
    }
    __syncthreads();
    cluster_sync();
    const bool peer_failed = *reinterpret_cast<volatile uint32_t *>(sm + SM_SLOT + 12) != 0u;
    if (failed || peer_failed) {
        if (tid == 0) {
            const long long peer_sent = *reinterpret_cast<volatile uint32_t *>(sm + SM_SLOT + 8);
            while (pd.recv < peer_sent && recv_half(pd, sm, kWaitCycles)) {
            }
        }
        __syncthreads();
        cluster_sync();
    }
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols)
                     : "memory");
    }
}

// Forward pass, loss and last-layer backward of n rows (x (n, 3), targets y (n, 2), t (n, 10)).
// Writes gelu'(z0), gelu'(z1), gelu'(z2) (tiled BF16), the images of x, H1..H4, g4 and g3, adds the loss sum to
// *loss and the column sums of g4 and g3 to db4 and db3.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_train_fwd(const unsigned char *__restrict__ pack, const float *__restrict__ x,
                const float *__restrict__ y, const float *__restrict__ t, long long n,
                unsigned char *__restrict__ Z0, unsigned char *__restrict__ Z1,
                unsigned char *__restrict__ Z2, unsigned char *__restrict__ H1, unsigned char *__restrict__ H2,
                unsigned char *__restrict__ H3, unsigned char *__restrict__ H4,
                unsigned char *__restrict__ Xi, unsigned char *__restrict__ G4,
                unsigned char *__restrict__ G3, float *__restrict__ db4,
                float *__restrict__ db3, double *loss, int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    float *sF = reinterpret_cast<float *>(sm + SM_F);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]);
    const uint32_t b_base = su32(sm + SM_B);
    const int h = (int)cluster_rank(), peer = h ^ 1;
    const uint32_t local = su32(sm), remote = peer_addr(local, (uint32_t)peer);
    const uint32_t remote_xbar = peer_addr(su32(&bar[3]), (uint32_t)peer);

    const uint32_t tmem = setup_cta(sm, tid, warp, 256u);
    chain_wait_release();  // the weight images come from the previous Adam step

    Pending pd;
    const long long n_tiles = (n + kTile - 1) / kTile;
    const long long first = cluster_id(), stride = cluster_count();
    const int row0 = tid & 127, grp0 = tid >> 7;
    const int q = warp & 3, ch = warp >> 2;
    const int erow = q * 32 + lane;
    const float inv_n = 1.0f / (float)n;
    unsigned char *Zs[3] = {Z0, Z1, Z2};
    unsigned char *Hs[4] = {H1, H2, H3, H4};
    bool failed = false;
    const uint32_t bar_w0 = su32(&bar[2]);
    if (tid == 0 && first < n_tiles) {
        load_half_image(b_base, pack, h, bar_ld);
        pd.ld = true;
        // the W0 half and the FP32 constants, once (read after the first layer-0 MMA, whose
        // issue waits for this copy)
        mbar_expect(bar_w0, 4096u + kPackF * 4u);
        bulk_g2s(local + SM_W0, pack + kPackW0 + h * 4096, 4096u, bar_w0);
        bulk_g2s(local + SM_F, pack + 3 * kPackW, kPackF * 4u, bar_w0);
        pd.a = true;
    }

    for (long long tile = first; tile < n_tiles; tile += stride) {
        const long long g0 = tile * kTile;
        if (!failed) {
            if (grp0 == 0) {  // one thread per row: x in BF16 as the layer-0 A operand (K 16)
                const long long gr = g0 + row0;
                float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
                if (gr < n) {
                    x0 = x[3 * gr];
                    x1 = x[3 * gr + 1];
                    x2 = x[3 * gr + 2];
                }
                const uint4 p0 = make_uint4(pack2(x0, x1), pack2(x2, 0.0f), 0u, 0u);
                const uint4 p1 = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(sm + SM_XA + a_off(row0, 0)) = p0;
                *reinterpret_cast<uint4 *>(sm + SM_XA + a_off(row0, 8)) = p1;
                if (h == 0) {  // the x image, zero-padded to 16 columns
                    *reinterpret_cast<uint4 *>(Xi + tile * kImage16 + a_off(row0, 0)) = p0;
                    *reinterpret_cast<uint4 *>(Xi + tile * kImage16 + a_off(row0, 8)) = p1;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }

        // layer 0 (one MMA, K = 16) and the hidden layers 1..3 (16 MMAs each) into TMEM columns
        // 0..127; the epilogue of layer l writes gelu(z_l) (H_{l+1}) to A tile l % 2 of both CTAs
        for (int l = 0; l < 4; ++l) {
            if (!failed) {
                fence_before();
                __syncthreads();
                fence_after();
                if (tid == 0) {
                    bool ok;
                    if (l == 0) {
                        ok = true;
                        if (pd.a) {
                            ok = mbar_wait(bar_w0, pd.ph_a, wait);
                            if (ok) {
                                pd.a = false;
                                pd.ph_a ^= 1u;
                            }
                        }
                        if (ok) {
                            mma_bf16(tmem, sdesc(local + SM_XA, 2048u, 128u),
                                     sdesc(local + SM_W0, 2048u, 128u), kIdesc, 0u);
                            mma_commit(bar_mma);
                            pd.mma = true;
                            ok = mbar_wait(bar_mma, pd.ph_mma, wait);
                            if (ok) {
                                pd.mma = false;
                                pd.ph_mma ^= 1u;
                            }
                        }
                    } else {
                        const int next = l < 3 ? NEXT_HALF : NEXT_W4;
                        const unsigned char *img = l < 3 ? pack + l * kPackW : pack;
                        ok = run_layer(pd, sm, tmem, local + ((l - 1) & 1) * 65536u, b_base,
                                       bar_ld, bar_mma, next, img, h, true, wait);
                    }
                    if (!ok) *abort_cta = 1;
                }
                __syncthreads();
                fence_after();
                failed = *abort_cta != 0;
            }
            if (!failed) {
                const int col0 = ch * kGroupCols, gc0 = h * kHalf + col0;
                const float *bias = sF + (l == 0 ? PF_B0 : PF_B1 + (l - 1) * 256);
                unsigned char *Hl = Hs[l] + tile * kImage;
                const uint32_t abuf = (l & 1) * 65536u;
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0;
                uint32_t v[32];
                tmem_ld32(ta, v);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k0 = gc0 + e * 8;
                    float hh[8], dd[8];
                    // 16-byte aligned: the bias blocks start at multiples of 4 floats, k0 % 8 == 0
                    const float4 bl = *reinterpret_cast<const float4 *>(bias + k0);
                    const float4 bh = *reinterpret_cast<const float4 *>(bias + k0 + 4);
                    const float bv[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {  // gelu(z), gelu'(z) from one Phi, one phi
                        const float2 z = __fadd2_rn(make_float2(__uint_as_float(v[e * 8 + u]),
                                                                __uint_as_float(v[e * 8 + u + 1])),
                                                    make_float2(bv[u], bv[u + 1]));
                        float2 phi, d;
                        phi_e2(z, phi, d);
                        const float2 g = __fmul2_rn(z, phi), gp = __ffma2_rn(z, d, phi);
                        hh[u] = g.x;
                        hh[u + 1] = g.y;
                        dd[u] = gp.x;
                        dd[u + 1] = gp.y;
                        v[e * 8 + u] = __float_as_uint(gp.x);
                        v[e * 8 + u + 1] = __float_as_uint(gp.y);
                    }
                    const uint4 pk = pack8(hh);
                    *reinterpret_cast<uint4 *>(Hl + a_off(erow, k0)) = pk;
                    if (l < 3) *reinterpret_cast<uint4 *>(Zs[l] + zb_off(tile, erow, k0)) = pack8(dd);
                    *reinterpret_cast<uint4 *>(sm + abuf + a_off(erow, k0)) = pk;
                }
                if (l == 3) tmem_st32(ta, v);  // gelu'(z3) in place of z3, for the g3 pass
                // the half to the peer's A tile l % 2
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) send_half(pd, local, remote, remote_xbar, l & 1, h);
            }
        }
        // the targets of the loss phase's rows (one per thread of column group 0), loaded while
        // the last layer's MMAs run
        float yr[2], tr[10];
#pragma unroll
        for (int k = 0; k < 2; ++k) yr[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < 10; ++j) tr[j] = 0.0f;
        if (!failed && ch == 0 && g0 + erow < n) {
            const long long gr = g0 + erow;
#pragma unroll
            for (int k = 0; k < 2; ++k) yr[k] = y[gr * 2 + k];
#pragma unroll
            for (int j = 0; j < 10; ++j) tr[j] = t[gr * 10 + j];
        }
        // the last layer (256 -> 12, as N = 16) from A tile 1 (H4) into TMEM columns 128..143
        if (!failed) {
            if (tid == 0) {
                bool ok = mbar_wait(bar_ld, pd.ph_ld, wait);
                if (ok) {  // the K steps over the own half of H4 first, then the peer's
                    pd.ld = false;
                    pd.ph_ld ^= 1u;
                    for (int half = 0; half < 2 && ok; ++half) {
                        if (half == 1) ok = recv_half(pd, sm, wait);
                        if (!ok) break;
                        const int k0 = 8 * (h ^ half);
#pragma unroll
                        for (int k = k0; k < k0 + 8; ++k)
                            mma_bf16(tmem + 128u, sdesc(local + SM_A1 + k * 4096u, 2048u, 128u),
                                     sdesc(b_base + k * 512u, 256u, 128u), kIdescN16,
                                     (uint32_t)(half > 0 || k > k0));
                    }
                    mma_commit(bar_mma);
                    pd.mma = true;
                    if (ok) ok = mbar_wait(bar_mma, pd.ph_mma, wait);
                    if (ok) {
                        pd.mma = false;
                        pd.ph_mma ^= 1u;
                    }
                }
                if (!ok) *abort_cta = 1;
            }
            __syncthreads();
            fence_after();
            failed = *abort_cta != 0;
        }
        if (!failed) {
            if (ch == 0) {
                // output, loss and its gradient g4 per row (logistic loss of the existence
                // logits, half the squared error of the regression outputs of existing slots,
                // over n); both CTAs compute them alike, CTA 0 stores them.  g4 in BF16 goes to
                // A tile 1 (free now) as the next MMA's A operand (K = 16).
                const long long gr = g0 + erow;
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + 128u, v);
                float L = 0.0f;
                float gg[12];
#pragma unroll
                for (int o = 0; o < 12; ++o) gg[o] = 0.0f;
                if (gr < n) {
                    float out[12];
#pragma unroll
                    for (int o = 0; o < 12; ++o) out[o] = __uint_as_float(v[o]) + sF[PF_B4 + o];
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float z = out[6 * k], yk = yr[k];
                        L += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - yk * z;
                        gg[6 * k] = (1.0f / (1.0f + expf(-z)) - yk) * inv_n;
#pragma unroll
                        for (int j = 0; j < 5; ++j) {
                            const float d = out[6 * k + 1 + j] - tr[5 * k + j];
                            L += 0.5f * yk * d * d;
                            gg[6 * k + 1 + j] = yk * d * inv_n;
                        }
                    }
                }
                const uint4 p0 = make_uint4(pack2(gg[0], gg[1]), pack2(gg[2], gg[3]),
                                            pack2(gg[4], gg[5]), pack2(gg[6], gg[7]));
                const uint4 p1 = make_uint4(pack2(gg[8], gg[9]), pack2(gg[10], gg[11]), 0u, 0u);
                *reinterpret_cast<uint4 *>(sm + SM_A1 + a_off(erow, 0)) = p0;
                *reinterpret_cast<uint4 *>(sm + SM_A1 + a_off(erow, 8)) = p1;
                if (h == 0) {  // g4 as a 16-column image, its column sums, the loss
                    unsigned char *G4t = G4 + tile * kImage16;
                    *reinterpret_cast<uint4 *>(G4t + a_off(erow, 0)) = p0;
                    *reinterpret_cast<uint4 *>(G4t + a_off(erow, 8)) = p1;
                    float cs[16];
#pragma unroll
                    for (int o = 0; o < 16; ++o) cs[o] = o < 12 ? gg[o] : 0.0f;
                    const float sum = warp_colsum<16>(cs, lane);
                    if (lane < 12) atomicAdd(db4 + lane, sum);
                    for (int d = 16; d > 0; d >>= 1) L += __shfl_xor_sync(0xffffffffu, L, d);
                    if (lane == 0) atomicAdd(loss, (double)L);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();
            fence_after();
            // g4 W4^T for the CTA's 128 columns: one MMA (K = 16) into TMEM columns 128..255
            if (tid == 0) {
                mma_bf16(tmem + 128u, sdesc(local + SM_A1, 2048u, 128u),
                         sdesc(b_base + 8192u, 2048u, 128u), kIdesc, 0u);
                mma_commit(bar_mma);
                pd.mma = true;
                bool ok = mbar_wait(bar_mma, pd.ph_mma, wait);
                if (ok) {
                    pd.mma = false;
                    pd.ph_mma ^= 1u;
                    if (tile + stride < n_tiles) {
                        load_half_image(b_base, pack, h, bar_ld);
                        pd.ld = true;
                    }
                } else {
                    *abort_cta = 1;
                }
            }
            __syncthreads();
            fence_after();
            failed = *abort_cta != 0;
        }
        if (!failed) {
            // last layer backward: g3 = (g4 W4^T) gelu'(z3), gelu'(z3) from tensor memory (the
            // fourth epilogue left it there)
            unsigned char *G3t = G3 + tile * kImage;
#pragma unroll 1
            for (int c = 0; c < 2; ++c) {
                const int col0 = ch * kGroupCols + c * 16, gc0 = h * kHalf + col0;
                uint32_t vz[16], vd[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, vz);
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + 128u + (uint32_t)col0, vd);
                float cs[16];  // this row's g3 of the 16 columns, for the column sums
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float gg[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = e * 8 + u;
                        gg[u] = __uint_as_float(vd[j]) * __uint_as_float(vz[j]);
                        cs[j] = gg[u];
                    }
                    *reinterpret_cast<uint4 *>(G3t + a_off(erow, gc0 + e * 8)) = pack8(gg);
                }
                const float sum = warp_colsum<16>(cs, lane);
                if (lane < 16) atomicAdd(db3 + gc0 + lane, sum);
            }
            fence_before();
            __syncthreads();
        }
    }
    teardown_cta(sm, tid, warp, tmem, 256u, failed, pd, flag, remote);
}

// Backward-data chain of the hidden layers for n rows: from the g3 image and the tiled BF16
// gelu'(z0..z2), writes the images of g2, g1, g0 with g_{l-1} = (g_l W_l^T) gelu'(z_{l-1}) and
// adds their column sums to db2, db1, db0.  pack_t: the backward images of
// W1, W2, W3 (B[n][k] = W[n][k]).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_train_bwd(const unsigned char *__restrict__ pack_t, const unsigned char *__restrict__ G3,
                const unsigned char *__restrict__ Z0, const unsigned char *__restrict__ Z1,
                const unsigned char *__restrict__ Z2, long long n, unsigned char *__restrict__ G2,
                unsigned char *__restrict__ G1, unsigned char *__restrict__ G0,
                float *__restrict__ db2, float *__restrict__ db1, float *__restrict__ db0,
                int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]), bar_a = su32(&bar[2]);
    const uint32_t bar_dz = su32(&bar[5]);
    const uint32_t b_base = su32(sm + SM_B);
    const int h = (int)cluster_rank(), peer = h ^ 1;
    const uint32_t local = su32(sm), remote = peer_addr(local, (uint32_t)peer);
    const uint32_t remote_xbar = peer_addr(su32(&bar[3]), (uint32_t)peer);
    const uint32_t tmem = setup_cta(sm, tid, warp, 128u);
    chain_wait_release();  // g3 and gelu'(z) come from the forward pass

    Pending pd;
    pd.off = 1;  // the halves alternate between A tiles 1 (g2) and 0 (g1)
    const long long n_tiles = (n + kTile - 1) / kTile;
    const long long first = cluster_id(), stride = cluster_count();
    const int q = warp & 3, ch = warp >> 2;
    const int erow = q * 32 + lane;
    const unsigned char *Zin[3] = {Z2, Z1, Z0};  // gelu'(z) of the layer below layers 3, 2, 1
    unsigned char *Gout[3] = {G2, G1, G0};
    float *dbs[3] = {db2, db1, db0};
    bool failed = false;
    // the g3 image of a tile is the first A tile: copied as soon as A tile 0 is free (at the
    // start, then once the previous tile's last MMAs are done)
    auto load_g3 = [&](long long tl) {
        mbar_expect(bar_a, kImage);
        bulk_g2s(local + SM_A0, G3 + tl * kImage, kImage / 2, bar_a);
        bulk_g2s(local + SM_A0 + kImage / 2, G3 + tl * kImage + kImage / 2, kImage / 2, bar_a);
        pd.a = true;
    };
    if (tid == 0 && first < n_tiles) {  // layer 3's image first
        load_half_image(b_base, pack_t + 2 * kPackW, h, bar_ld);
        pd.ld = true;
        load_g3(first);
    }

    for (long long tile = first; tile < n_tiles; tile += stride) {
        for (int l = 0; l < 3; ++l) {  // hidden layers 3, 2, 1
            if (!failed) {
                fence_before();
                __syncthreads();
                fence_after();
                if (tid == 0) {
                    // gelu'(z) of the layer below for the CTA's 128 columns (32 KB), copied
                    // while the MMAs run; the buffer's last readers, the previous epilogue,
                    // have passed the barrier above after a proxy fence
                    mbar_expect(bar_dz, 32768u);
                    bulk_g2s(local + SM_DZ, Zin[l] + zb_off(tile, 0, h * kHalf), 32768u, bar_dz);
                    pd.dz = true;
                    bool ok;
                    if (l == 0) {
                        ok = mbar_wait(bar_a, pd.ph_a, wait);
                        if (ok) {
                            pd.a = false;
                            pd.ph_a ^= 1u;
                        }
                    } else {
                        ok = true;
                    }
                    const int next = l < 2 || tile + stride < n_tiles ? NEXT_HALF : NEXT_NONE;
                    const unsigned char *img = pack_t + (l < 2 ? 1 - l : 2) * kPackW;
                    if (!ok || !run_layer(pd, sm, tmem, local + (l & 1) * 65536u, b_base, bar_ld,
                                          bar_mma, next, img, h, l > 0, wait))
                        ok = false;
                    else if (l == 2 && tile + stride < n_tiles)
                        load_g3(tile + stride);  // A tile 0 read for the last time this tile
                    if (ok) {
                        ok = mbar_wait(bar_dz, pd.ph_dz, wait);
                        if (ok) {
                            pd.dz = false;
                            pd.ph_dz ^= 1u;
                        }
                    }
                    if (!ok) *abort_cta = 1;
                }
                __syncthreads();
                fence_after();
                failed = *abort_cta != 0;
            }
            if (!failed) {
                const int col0 = ch * kGroupCols, gc0 = h * kHalf + col0;
                unsigned char *Gl = Gout[l] + tile * kImage;
                const uint32_t abuf = ((l + 1) & 1) * 65536u;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
                float cs[32];  // this row's g of the 32 columns, for the column sums
                // this row's gelu'(z) of the 32 columns: group ch * 4 + e of the CTA's 16
                const unsigned char *dzs = sm + SM_DZ + ch * 4 * 2048 + erow * 16;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k0 = gc0 + e * 8;
                    const uint4 w = *reinterpret_cast<const uint4 *>(dzs + e * 2048);
                    const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
                    float gg[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {  // BF16 pairs: column k0 + u in half u % 2
                        const uint32_t b = wv[u >> 1];
                        const float dz = __uint_as_float((u & 1) ? (b & 0xffff0000u) : (b << 16));
                        gg[u] = __uint_as_float(v[e * 8 + u]) * dz;
                        cs[e * 8 + u] = gg[u];
                    }
                    const uint4 pk = pack8(gg);
                    *reinterpret_cast<uint4 *>(Gl + a_off(erow, k0)) = pk;
                    if (l < 2) *reinterpret_cast<uint4 *>(sm + abuf + a_off(erow, k0)) = pk;
                }
                atomicAdd(dbs[l] + gc0 + lane, warp_colsum<32>(cs, lane));
                if (l < 2) {  // the half to the peer's A tile (l + 1) % 2
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                    if (tid == 0) send_half(pd, local, remote, remote_xbar, (l + 1) & 1, h);
                }
            }
        }
        if (!failed) {  // the next tile's copies overwrite A tile 0 and gelu'(z), its MMAs
                        // the accumulator
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();
        }
    }
    teardown_cta(sm, tid, warp, tmem, 128u, failed, pd, flag, remote);
}

}  // namespace

int train_fwd(rp_surrogate_s *s, long long n, const float *x, const float *y, const float *t,
              float *db3, float *db4, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    RP_CUDA_TRY(cudaFuncSetAttribute(k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SM_TOTAL_FWD));
    const long long tiles = (n + kTile - 1) / kTile;
    const int clusters = (int)std::min<long long>(tiles, (long long)sm_count(dev) / 2);
    return launch_chained(k_train_fwd, dim3(2 * clusters), dim3(kThreads), SM_TOTAL_FWD, st,
                          (const unsigned char *)s->pack, x, y, t, n, s->Z[0], s->Z[1], s->Z[2],
                          s->H[1], s->H[2], s->H[3], s->H[4], s->ximg, s->g4img, s->gl[3], db4,
                          db3, s->loss, s->fflag, wait_cycles(s));
}

int train_bwd(rp_surrogate_s *s, long long n, float *db2, float *db1, float *db0, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    RP_CUDA_TRY(cudaFuncSetAttribute(k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SM_TOTAL_BWD));
    const long long tiles = (n + kTile - 1) / kTile;
    const int clusters = (int)std::min<long long>(tiles, (long long)sm_count(dev) / 2);
    return launch_chained(k_train_bwd, dim3(2 * clusters), dim3(kThreads), SM_TOTAL_BWD, st,
                          (const unsigned char *)s->pack_t, (const unsigned char *)s->gl[3],
                          (const unsigned char *)s->Z[0], (const unsigned char *)s->Z[1],
                          (const unsigned char *)s->Z[2],
                          n, s->gl[2], s->gl[1], s->gl[0], db2, db1, db0, s->fflag,
                          wait_cycles(s));
}

}  // namespace rph
