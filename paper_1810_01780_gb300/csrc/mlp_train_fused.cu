// mlp_train_fused.cu -- one training step of the surrogate network in two fused tensor-core
// kernels per batch: the whole forward pass with the loss and the last layer's backward pass,
// then the backward-data chain through the three hidden layers.
//
// k_train_fwd: per tile of 128 rows a CTA of 512 threads runs layer 0 (3 -> 256) on the CUDA
//   cores into the BF16 A tile in shared memory, then the three 256 -> 256 layers on the
//   tensor cores exactly as the fused inference kernel does (weights by bulk copy, 16
//   tcgen05.mma of M 128, N 256, K 16 into a 256-column TMEM accumulator, epilogue by sixteen
//   warps), keeping the activations in shared memory between layers.  The epilogues also
//   store what the later kernels read: the pre-activations z0..z2 in FP32 (tiled: a tile's 8
//   columns k..k+7 of its 128 rows are 4 KB contiguous, so a warp's stores and the backward
//   pass's loads of one 8-column group are 1 KB contiguous) and the activations H1..H4 as BF16
//   operand images (tc_common.cuh), and x as a 16-column image.  The last layer (256 -> 12)
//   comes out of the third epilogue's partial sums; the loss and its gradient g4 follow per row
//   (g4 stored as a 16-column image, its column sums added to db4), and the last layer's
//   backward data pass g3 = (g4 W4^T) gelu'(z3) re-reads z3 from tensor memory, stores g3 as a
//   BF16 image and adds its column sums to the bias gradient db3.
// k_train_bwd: per tile, the g3 image by bulk copy as the A tile, then for the hidden layers
//   3, 2, 1 the backward images B[n][k] = W[n][k] by bulk copy, 16 tcgen05.mma (N 256) and an
//   epilogue g_{l-1} = (g_l W_l^T) gelu'(z_{l-1}) that stores g_{l-1} as a BF16 image, adds
//   its column sums to db_{l-1} and, but for the last, feeds it back as the next A tile.
// Arithmetic is that of the per-layer path: BF16 operands (weights, activations and
// gradients rounded to BF16 where they enter a product), FP32 products and sums, FP32 bias,
// GELU and GELU'; bias gradients are sums of the unrounded FP32 g.  A batch's last, partial
// tile is computed whole: its rows past n have zero output gradients, so they add nothing to
// any gradient.  Every mbarrier wait is bounded (the surrogate's wait limit); a CTA that gives
// up sets the error flag, waits (with the default bound) for the work it issued, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "rp_internal.h"
#include "tc_common.cuh"

namespace rph {

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kThreads = 512;            // 16 warps: lane quarter (warp % 4) x column group (warp / 4)
constexpr int kGroups = kThreads / 128;  // column groups of a row
constexpr int kGroupCols = 256 / kGroups;
constexpr uint32_t kWBytes = (uint32_t)kPackW;
// shared memory map (bytes): A tile, B tile, FP32 constants, barriers
constexpr uint32_t SM_A = 0;
constexpr uint32_t SM_B = 65536;
constexpr uint32_t SM_F = SM_B + kWBytes;
constexpr uint32_t SM_BAR = SM_F + kPackF * 4;  // barriers: B image, MMAs, A tile (backward)
constexpr uint32_t SM_SLOT = SM_BAR + 32;        // TMEM address, then the abort word
constexpr uint32_t SM_TOTAL = SM_BAR + 64;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory map exceeds a CTA's limit");
static_assert(SM_F % 16 == 0 && SM_BAR % 8 == 0, "alignment");
// after the last MMA of a tile the A tile holds the last layer's partial sums (3 groups x 128
// rows x 12) and then the rows' output gradients g4 (128 x 12)
constexpr uint32_t SM_P = 0, SM_G4 = (kGroups - 1) * kTile * 12 * 4;
static_assert(SM_G4 + kTile * 12 * 4 <= 65536, "partial sums and g4 fit in the A tile");

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void load_image(uint32_t b_base, const unsigned char *src, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kWBytes)
                 : "memory");
#pragma unroll
    for (int c = 0; c < 4; ++c)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                b_base + c * 32768u),
            "l"(src + c * 32768), "r"(32768u), "r"(bar)
            : "memory");
}

// 16 MMAs of one 256 x 256 layer (A tile x B image) into the accumulator, committed to bar_mma
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t a_base, uint32_t b_base,
                                            uint32_t bar_mma)
{
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const uint64_t ad = sdesc(a_base + s * 4096u, 2048u, 128u);
        const uint64_t bd = sdesc(b_base + s * 8192u, 4096u, 128u);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(s)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar_mma)
                 : "memory");
}

__device__ __forceinline__ void store8(float *dst, const float (&v)[8])
{
    reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}
// the 8 FP32 values of columns k0..k0+7 (k0 % 8 == 0) of row `row` of tile `tile` in a tiled
// pre-activation buffer
__device__ __forceinline__ float *zt_at(float *Z, long long tile, int row, int k0)
{
    return Z + tile * (128LL * 256) + (k0 >> 3) * 1024 + row * 8;
}
__device__ __forceinline__ const float *zt_at(const float *Z, long long tile, int row, int k0)
{
    return Z + tile * (128LL * 256) + (k0 >> 3) * 1024 + row * 8;
}

// Shared setup of both kernels: barriers, abort word, tensor memory (256 columns).
__device__ __forceinline__ uint32_t setup_cta(unsigned char *sm, int tid, int warp)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + SM_SLOT);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_cta = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    return *slot;
}

// Shared teardown: on failure record it and drain the issued work, then free tensor memory.
__device__ __forceinline__ void teardown_cta(unsigned char *sm, int tid, int warp, uint32_t tmem,
                                             bool failed, bool ld_pending, uint32_t ph_ld,
                                             bool mma_pending, uint32_t ph_mma, int *flag,
                                             bool a_pending = false, uint32_t ph_a = 0)
{
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    if (failed && tid == 0) {
        atomicExch(flag, 1);
        if (ld_pending) mbar_wait(su32(&bar[0]), ph_ld);
        if (mma_pending) mbar_wait(su32(&bar[1]), ph_mma);
        if (a_pending) mbar_wait(su32(&bar[2]), ph_a);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

// Forward pass, loss and last-layer backward of n rows (x (n, 3), targets y (n, 2), t (n, 10)).
// Writes z0, z1, z2 (tiled FP32), the images of x, H1..H4, g4 and g3, adds the loss sum to
// *loss and the column sums of g4 and g3 to db4 and db3.
__global__ void __launch_bounds__(kThreads, 1)
    k_train_fwd(const unsigned char *__restrict__ pack, const float *__restrict__ x,
                const float *__restrict__ y, const float *__restrict__ t, long long n,
                float *__restrict__ Z0, float *__restrict__ Z1, float *__restrict__ Z2,
                unsigned char *__restrict__ H1, unsigned char *__restrict__ H2,
                unsigned char *__restrict__ H3, unsigned char *__restrict__ H4,
                unsigned char *__restrict__ Xi, unsigned char *__restrict__ G4,
                unsigned char *__restrict__ G3, float *__restrict__ db4,
                float *__restrict__ db3, double *loss, int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + SM_A;
    float *sF = reinterpret_cast<float *>(sm + SM_F);
    float *sP = reinterpret_cast<float *>(sm + SM_P);
    float *sG = reinterpret_cast<float *>(sm + SM_G4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]);
    const uint32_t a_base = su32(sm + SM_A), b_base = su32(sm + SM_B);

    const float4 *gF = reinterpret_cast<const float4 *>(pack + 3 * kPackW);
    for (int i = tid; i < kPackF / 4; i += kThreads) reinterpret_cast<float4 *>(sF)[i] = gF[i];
    const uint32_t tmem = setup_cta(sm, tid, warp);

    uint32_t ph_ld = 0, ph_mma = 0;
    bool ld_pending = false, mma_pending = false;
    const long long n_tiles = (n + kTile - 1) / kTile;
    const int row0 = tid & 127, grp0 = tid >> 7;
    const int q = warp & 3, ch = warp >> 2;
    const int erow = q * 32 + lane;
    const float inv_n = 1.0f / (float)n;
    float *Zs[2] = {Z1, Z2};
    unsigned char *Hs[3] = {H2, H3, H4};
    bool failed = false;
    if (tid == 0 && blockIdx.x < n_tiles) {
        load_image(b_base, pack, bar_ld);
        ld_pending = true;
    }

    for (long long tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const long long g0 = tile * kTile;
        {  // layer 0 on the CUDA cores: z0, and gelu(z0) in BF16 to the A tile and the H1 image
            const long long gr = g0 + row0;
            float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
            if (gr < n) {
                x0 = bf16r(x[3 * gr]);
                x1 = bf16r(x[3 * gr + 1]);
                x2 = bf16r(x[3 * gr + 2]);
            }
            if (grp0 < 2) {  // the x image: columns 0..2, zero-padded to 16
                const uint4 pk = grp0 == 0 ? make_uint4(pack2(x0, x1), pack2(x2, 0.0f), 0u, 0u)
                                           : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(Xi + tile * kImage16 + a_off(row0, grp0 * 8)) = pk;
            }
#pragma unroll 1
            for (int c = 0; c < kGroupCols / 8; ++c) {
                const int k0 = grp0 * kGroupCols + c * 8;
                float zz[8], hh[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = k0 + e;
                    float z = x0 * sF[PF_W0 + j];
                    z = fmaf(x1, sF[PF_W0 + 256 + j], z);
                    z = fmaf(x2, sF[PF_W0 + 512 + j], z);
                    zz[e] = z + sF[PF_B0 + j];
                    hh[e] = gelu(zz[e]);
                }
                store8(zt_at(Z0, tile, row0, k0), zz);
                const uint4 pk = pack8(hh);
                *reinterpret_cast<uint4 *>(sA + a_off(row0, k0)) = pk;
                *reinterpret_cast<uint4 *>(H1 + tile * kImage + a_off(row0, k0)) = pk;
            }
        }
        float acc[12];
#pragma unroll
        for (int o = 0; o < 12; ++o) acc[o] = 0.0f;

        for (int l = 0; l < 3; ++l) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();
            fence_after();
            if (tid == 0) {
                if (mbar_wait(bar_ld, ph_ld, wait)) {
                    ld_pending = false;
                    issue_layer(tmem, a_base, b_base, bar_mma);
                    mma_pending = true;
                } else {
                    *abort_cta = 1;
                }
            }
            ph_ld ^= 1u;
            if (!mbar_wait(bar_mma, ph_mma, wait)) *abort_cta = 1;
            ph_mma ^= 1u;
            fence_after();
            __syncthreads();
            if (*abort_cta) {
                failed = true;
                break;
            }
            if (tid == 0) {
                mma_pending = false;
                if (l < 2) {
                    load_image(b_base, pack + (l + 1) * kPackW, bar_ld);
                    ld_pending = true;
                } else if (tile + gridDim.x < n_tiles) {
                    load_image(b_base, pack, bar_ld);
                    ld_pending = true;
                }
            }
            const float *bias = sF + PF_B1 + l * 256;
            unsigned char *Hl = Hs[l] + tile * kImage;
#pragma unroll 1
            for (int c = 0; c < kGroupCols / 32; ++c) {
                const int col0 = ch * kGroupCols + c * 32;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k0 = col0 + e * 8;
                    float zz[8], hh[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        zz[u] = __uint_as_float(v[e * 8 + u]) + bias[k0 + u];
                        hh[u] = gelu(zz[u]);
                    }
                    const uint4 pk = pack8(hh);
                    *reinterpret_cast<uint4 *>(Hl + a_off(erow, k0)) = pk;
                    if (l < 2) {
                        store8(zt_at(Zs[l], tile, erow, k0), zz);
                        *reinterpret_cast<uint4 *>(sA + a_off(erow, k0)) = pk;
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float h = bf16r(hh[u]);
                            const float *w4 = sF + PF_W4 + (k0 + u) * 12;
#pragma unroll
                            for (int o = 0; o < 12; ++o) acc[o] = fmaf(h, w4[o], acc[o]);
                        }
                    }
                }
            }
            fence_before();
        }
        if (failed) break;
        // last layer: the column groups' partial sums of each row meet in shared memory
        if (ch > 0) {
#pragma unroll
            for (int o = 0; o < 12; ++o) sP[((ch - 1) * kTile + erow) * 12 + o] = acc[o];
        }
        __syncthreads();
        if (ch == 0) {
            // output, loss and its gradient g4 per row (logistic loss of the existence logits,
            // half the squared error of the regression outputs of existing slots, over n)
            const long long gr = g0 + erow;
            float L = 0.0f;
            float gg[12];
#pragma unroll
            for (int o = 0; o < 12; ++o) gg[o] = 0.0f;
            if (gr < n) {
                float out[12];
#pragma unroll
                for (int o = 0; o < 12; ++o) {
                    float v = acc[o];
                    for (int g = 1; g < kGroups; ++g) v += sP[((g - 1) * kTile + erow) * 12 + o];
                    out[o] = v + sF[PF_B4 + o];
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float z = out[6 * k], yk = y[gr * 2 + k];
                    L += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - yk * z;
                    gg[6 * k] = (1.0f / (1.0f + expf(-z)) - yk) * inv_n;
#pragma unroll
                    for (int j = 0; j < 5; ++j) {
                        const float d = out[6 * k + 1 + j] - t[gr * 10 + 5 * k + j];
                        L += 0.5f * yk * d * d;
                        gg[6 * k + 1 + j] = yk * d * inv_n;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 12; ++o) sG[erow * 12 + o] = bf16r(gg[o]);
            {  // g4 as a 16-column image, and its column sums
                float cs[16];
#pragma unroll
                for (int o = 0; o < 16; ++o) cs[o] = o < 12 ? gg[o] : 0.0f;
                unsigned char *G4t = G4 + tile * kImage16;
                *reinterpret_cast<uint4 *>(G4t + a_off(erow, 0)) =
                    make_uint4(pack2(gg[0], gg[1]), pack2(gg[2], gg[3]), pack2(gg[4], gg[5]),
                               pack2(gg[6], gg[7]));
                *reinterpret_cast<uint4 *>(G4t + a_off(erow, 8)) =
                    make_uint4(pack2(gg[8], gg[9]), pack2(gg[10], gg[11]), 0u, 0u);
                const float sum = warp_colsum<16>(cs, lane);
                if (lane < 12) atomicAdd(db4 + lane, sum);
            }
            for (int d = 16; d > 0; d >>= 1) L += __shfl_xor_sync(0xffffffffu, L, d);
            if (lane == 0) atomicAdd(loss, (double)L);
        }
        __syncthreads();
        fence_after();
        {  // last layer backward: g3 = (g4 W4^T) gelu'(z3), z3 read again from tensor memory
            const float *bias = sF + PF_B1 + 2 * 256;
            unsigned char *G3t = G3 + tile * kImage;
            float gr4[12];
#pragma unroll
            for (int o = 0; o < 12; ++o) gr4[o] = sG[erow * 12 + o];
#pragma unroll 1
            for (int c = 0; c < kGroupCols / 32; ++c) {
                const int col0 = ch * kGroupCols + c * 32;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
                float cs[32];  // this row's g3 of the 32 columns, for the column sums
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float gg[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int col = col0 + e * 8 + u;
                        const float *w4 = sF + PF_W4 + col * 12;
                        float s = 0.0f;
#pragma unroll
                        for (int o = 0; o < 12; ++o) s = fmaf(gr4[o], w4[o], s);
                        gg[u] = s * gelu_prime(__uint_as_float(v[e * 8 + u]) + bias[col]);
                        cs[e * 8 + u] = gg[u];
                    }
                    *reinterpret_cast<uint4 *>(G3t + a_off(erow, col0 + e * 8)) = pack8(gg);
                }
                atomicAdd(db3 + col0 + lane, warp_colsum<32>(cs, lane));
            }
        }
        fence_before();
        __syncthreads();
    }
    teardown_cta(sm, tid, warp, tmem, failed, ld_pending, ph_ld ^ 1u, mma_pending, ph_mma ^ 1u, flag);
}

// Backward-data chain of the hidden layers for n rows: from the g3 image and the tiled
// pre-activations z0..z2, writes the images of g2, g1, g0 with g_{l-1} = (g_l W_l^T)
// gelu'(z_{l-1}) and adds their column sums to db2, db1, db0.  pack_t: the backward images of
// W1, W2, W3 (B[n][k] = W[n][k]).
__global__ void __launch_bounds__(kThreads, 1)
    k_train_bwd(const unsigned char *__restrict__ pack_t, const unsigned char *__restrict__ G3,
                const float *__restrict__ Z0, const float *__restrict__ Z1,
                const float *__restrict__ Z2, long long n, unsigned char *__restrict__ G2,
                unsigned char *__restrict__ G1, unsigned char *__restrict__ G0,
                float *__restrict__ db2, float *__restrict__ db1, float *__restrict__ db0,
                int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + SM_A;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_SLOT + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]), bar_a = su32(&bar[2]);
    const uint32_t a_base = su32(sm + SM_A), b_base = su32(sm + SM_B);
    const uint32_t tmem = setup_cta(sm, tid, warp);

    uint32_t ph_ld = 0, ph_mma = 0, ph_a = 0;
    bool ld_pending = false, mma_pending = false, a_pending = false;
    const long long n_tiles = (n + kTile - 1) / kTile;
    const int q = warp & 3, ch = warp >> 2;
    const int erow = q * 32 + lane;
    const float *Zin[3] = {Z2, Z1, Z0};  // gelu' of the layer below layers 3, 2, 1
    unsigned char *Gout[3] = {G2, G1, G0};
    float *dbs[3] = {db2, db1, db0};
    bool failed = false;
    if (tid == 0 && blockIdx.x < n_tiles) {  // layer 3's image first
        load_image(b_base, pack_t + 2 * kPackW, bar_ld);
        ld_pending = true;
    }

    for (long long tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        if (tid == 0) {  // the tile's g3 image is the first A tile
            mbar_expect(bar_a, kImage);
            bulk_g2s(a_base, G3 + tile * kImage, kImage / 2, bar_a);
            bulk_g2s(a_base + kImage / 2, G3 + tile * kImage + kImage / 2, kImage / 2, bar_a);
            a_pending = true;
        }
        for (int l = 0; l < 3; ++l) {  // hidden layers 3, 2, 1
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();
            fence_after();
            if (tid == 0) {
                bool ok = true;
                if (l == 0) {
                    ok = mbar_wait(bar_a, ph_a, wait);
                    if (ok) {
                        a_pending = false;
                        ph_a ^= 1u;
                    }
                }
                if (ok && mbar_wait(bar_ld, ph_ld, wait)) {
                    ld_pending = false;
                    issue_layer(tmem, a_base, b_base, bar_mma);
                    mma_pending = true;
                } else {
                    *abort_cta = 1;
                }
            }
            ph_ld ^= 1u;
            if (!mbar_wait(bar_mma, ph_mma, wait)) *abort_cta = 1;
            ph_mma ^= 1u;
            fence_after();
            __syncthreads();
            if (*abort_cta) {
                failed = true;
                break;
            }
            if (tid == 0) {
                mma_pending = false;
                if (l < 2) {
                    load_image(b_base, pack_t + (1 - l) * kPackW, bar_ld);
                    ld_pending = true;
                } else if (tile + gridDim.x < n_tiles) {
                    load_image(b_base, pack_t + 2 * kPackW, bar_ld);
                    ld_pending = true;
                }
            }
            const float *Zl = Zin[l];
            unsigned char *Gl = Gout[l] + tile * kImage;
            float *dbl = dbs[l];
#pragma unroll 1
            for (int c = 0; c < kGroupCols / 32; ++c) {
                const int col0 = ch * kGroupCols + c * 32;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
                float cs[32];  // this row's g of the 32 columns, for the column sums
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k0 = col0 + e * 8;
                    const float4 *zs = reinterpret_cast<const float4 *>(zt_at(Zl, tile, erow, k0));
                    const float4 z0 = __ldg(zs), z1 = __ldg(zs + 1);
                    const float z[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
                    float gg[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        gg[u] = __uint_as_float(v[e * 8 + u]) * gelu_prime(z[u]);
                        cs[e * 8 + u] = gg[u];
                    }
                    const uint4 pk = pack8(gg);
                    *reinterpret_cast<uint4 *>(Gl + a_off(erow, k0)) = pk;
                    if (l < 2) *reinterpret_cast<uint4 *>(sA + a_off(erow, k0)) = pk;
                }
                atomicAdd(dbl + col0 + lane, warp_colsum<32>(cs, lane));
            }
            fence_before();
        }
        if (failed) break;
        __syncthreads();  // the next tile's copy overwrites the A tile
    }
    teardown_cta(sm, tid, warp, tmem, failed, ld_pending, ph_ld ^ 1u, mma_pending, ph_mma ^ 1u, flag,
                 a_pending, ph_a);
}

}  // namespace

int train_fwd(rp_surrogate_s *s, long long n, const float *x, const float *y, const float *t,
              float *db3, float *db4, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    RP_CUDA_TRY(cudaFuncSetAttribute(k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SM_TOTAL));
    const long long tiles = (n + kTile - 1) / kTile;
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count(dev));
    k_train_fwd<<<grid, kThreads, SM_TOTAL, st>>>(s->pack, x, y, t, n, s->Z[0], s->Z[1], s->Z[2],
                                                  s->H[1], s->H[2], s->H[3], s->H[4], s->ximg,
                                                  s->g4img, s->gl[3], db4, db3, s->loss, s->fflag,
                                                  wait_cycles(s));
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

int train_bwd(rp_surrogate_s *s, long long n, float *db2, float *db1, float *db0, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    RP_CUDA_TRY(cudaFuncSetAttribute(k_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SM_TOTAL));
    const long long tiles = (n + kTile - 1) / kTile;
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count(dev));
    k_train_bwd<<<grid, kThreads, SM_TOTAL, st>>>(s->pack_t, s->gl[3], s->Z[0], s->Z[1], s->Z[2],
                                                  n, s->gl[2], s->gl[1], s->gl[0], db2, db1, db0,
                                                  s->fflag, wait_cycles(s));
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

}  // namespace rph
