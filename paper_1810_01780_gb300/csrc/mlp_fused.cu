// mlp_fused.cu -- surrogate inference in one persistent kernel on the 5th-generation tensor
// cores.
//
// Per tile of 128 rows a CTA of 512 threads computes all five layers without the activations
// leaving the SM:
//   layer 0 (3 -> 256) on the CUDA cores, written as BF16 into the A operand tile (64 KB);
//   layers 1..3 (256 -> 256): the layer's packed BF16 weights (128 KB) arrive in shared memory
//     by bulk copy (cp.async.bulk, completion on an mbarrier), issued as soon as the previous
//     layer's MMAs have released the B tile so that the copy overlaps the epilogue; one thread
//     issues 2 x 16 tcgen05.mma (M = 128, N = 128 (one half of the output columns each),
//     K = 16, FP32 accumulators in tensor memory, 256 columns) and commits them to a second
//     mbarrier; the sixteen warps read the accumulators back
//     (tcgen05.ld, warp w reads lanes 32 (w % 4) .. + 31 and columns 64 (w / 4) .. + 63),
//     add the bias, apply GELU and write the BF16 result into the A tile for the next layer;
//   layer 4 (256 -> 12) on the CUDA cores from the last layer's BF16-rounded activations.
// Operand images use the no-swizzle K-major layout of the tensor cores: 8 x 8 core matrices of
// 128 contiguous bytes; for A (128 rows x 256 k) core (k/8, row/8) sits at
// ((k/8) * 16 + row/8) * 128 (K-direction stride 2048 B, 8-row stride 128 B); B (256 n x 256 k)
// holds its two halves of n one after the other, each laid out like A.  Arithmetic is that of the
// unfused path: BF16 operands, FP32 products and sums, FP32 bias and GELU.
// Every wait on an mbarrier is bounded (by default about two seconds; rp_surrogate_set_wait_limit
// sets it); a CTA that gives up sets the error flag, waits (with the default bound) for its work
// in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "rp_internal.h"
#include "tc_common.cuh"

namespace rph {

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kThreads = 512;             // 16 warps: 4 column groups per TMEM lane quarter
constexpr int kGroups = kThreads / 128;   // column groups of a row
constexpr int kGroupCols = 256 / kGroups;
constexpr uint32_t kWBytes = (uint32_t)kPackW;
// shared memory map (bytes)
constexpr uint32_t SM_A = 0;
constexpr uint32_t SM_B = 65536;
constexpr uint32_t SM_F = SM_B + kWBytes;
constexpr uint32_t SM_BAR = SM_F + kPackF * 4;
constexpr uint32_t SM_TOTAL = SM_BAR + 32;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory map exceeds a CTA's limit");
static_assert(SM_F % 16 == 0 && SM_BAR % 8 == 0, "alignment");
static_assert((kGroups - 1) * kTile * 12 * 4 <= 65536, "layer-4 partial sums reuse the A tile");
static_assert(PF_W4 % 4 == 0, "W4 rows load as float4");

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 128 (one half of the
// layer's output columns), M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);

// one hidden layer's packed weights (kWBytes) into the B tile, completion on `bar`
__device__ __forceinline__ void load_weights(uint32_t b_base, const unsigned char *src, uint32_t bar)
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

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_fused(const unsigned char *__restrict__ pack, const float *__restrict__ x,
                float *__restrict__ out, long long n, int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm + SM_A;
    float *sF = reinterpret_cast<float *>(sm + SM_F);
    float *sP = reinterpret_cast<float *>(sm + SM_A);  // layer-4 partials, after the last MMA
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + SM_BAR);  // [0] weights in, [1] MMAs done
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + SM_BAR + 16);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + SM_BAR + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]);
    const uint32_t a_base = su32(sm + SM_A), b_base = su32(sm + SM_B);

    const float4 *gF = reinterpret_cast<const float4 *>(pack + 3 * kPackW);
    for (int i = tid; i < kPackF / 4; i += kThreads) reinterpret_cast<float4 *>(sF)[i] = gF[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_ld) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma) : "memory");
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
    const uint32_t tmem = *slot;

    uint32_t ph_ld = 0, ph_mma = 0;
    bool ld_pending = false, mma_pending = false;  // thread 0: async work not yet waited for
    const long long n_tiles = (n + kTile - 1) / kTile;
    const int row0 = tid & 127, grp0 = tid >> 7;  // layer 0: row and column group
    const int q = warp & 3, ch = warp >> 2;       // epilogue: lane quarter and column group
    const int erow = q * 32 + lane;
    bool failed = false;
    if (tid == 0 && blockIdx.x < n_tiles) {  // the first layer's weights, during layer 0
        load_weights(b_base, pack, bar_ld);
        ld_pending = true;
    }

    for (long long tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const long long g0 = tile * kTile;
        {  // layer 0 on the CUDA cores
            const long long gr = g0 + row0;
            float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
            if (gr < n) {
                x0 = bf16r(x[3 * gr]);
                x1 = bf16r(x[3 * gr + 1]);
                x2 = bf16r(x[3 * gr + 2]);
            }
#pragma unroll 2
            for (int c = 0; c < kGroupCols / 8; ++c) {
                const int k0 = grp0 * kGroupCols + c * 8;
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float h[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int j = k0 + 2 * e + u;
                        float z = x0 * sF[PF_W0 + j];
                        z = fmaf(x1, sF[PF_W0 + 256 + j], z);
                        z = fmaf(x2, sF[PF_W0 + 512 + j], z);
                        h[u] = gelu(z + sF[PF_B0 + j]);
                    }
                    w[e] = pack2(h[0], h[1]);
                }
                *reinterpret_cast<uint4 *>(sA + a_off(row0, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        float2 acc2[6];  // the 12 outputs of the last layer as pairs (o, o + 1)
#pragma unroll
        for (int o = 0; o < 6; ++o) acc2[o] = make_float2(0.0f, 0.0f);

        for (int l = 0; l < 3; ++l) {
            // the A tile written by this CTA's threads becomes visible to the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();
            fence_after();
            if (tid == 0) {
                if (mbar_wait(bar_ld, ph_ld, wait)) {
                    ld_pending = false;
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {  // output columns 128 hf .. 128 hf + 127
#pragma unroll
                        for (int s = 0; s < 16; ++s) {
                            const uint64_t ad = sdesc(a_base + s * 4096u, 2048u, 128u);
                            const uint64_t bd = sdesc(b_base + hf * 65536u + s * 4096u, 2048u, 128u);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                    tmem + hf * 128u),
                                "l"(ad), "l"(bd), "r"(kIdesc), "r"(s)
                                : "memory");
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            bar_mma)
                        : "memory");
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
                // the B tile is free: the next weights load during this epilogue
                if (l < 2) {
                    load_weights(b_base, pack + (l + 1) * kPackW, bar_ld);
                    ld_pending = true;
                } else if (tile + gridDim.x < n_tiles) {
                    load_weights(b_base, pack, bar_ld);
                    ld_pending = true;
                }
            }

            const float *bias = sF + PF_B1 + l * 256;
#pragma unroll 1
            for (int c = 0; c < kGroupCols / 32; ++c) {
                const int col0 = ch * kGroupCols + c * 32;
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
                if (l < 2) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        uint32_t w[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = e * 8 + 2 * u;
                            const float2 g = gelu2(__fadd2_rn(
                                make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])),
                                make_float2(bias[col0 + j], bias[col0 + j + 1])));
                            w[u] = pack2(g.x, g.y);
                        }
                        *reinterpret_cast<uint4 *>(sA + a_off(erow, col0 + e * 8)) =
                            make_uint4(w[0], w[1], w[2], w[3]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const float2 g = gelu2(__fadd2_rn(
                            make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])),
                            make_float2(bias[col0 + j], bias[col0 + j + 1])));
                        const float hs[2] = {bf16r(g.x), bf16r(g.y)};
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            // W4 row col0 + j + s: 12 floats, 16-byte aligned (PF_W4 % 4 == 0)
                            const float4 *w4 =
                                reinterpret_cast<const float4 *>(sF + PF_W4 + (col0 + j + s) * 12);
                            const float2 h2 = make_float2(hs[s], hs[s]);
#pragma unroll
                            for (int c4 = 0; c4 < 3; ++c4) {
                                const float4 w = w4[c4];
                                acc2[2 * c4] = __ffma2_rn(h2, make_float2(w.x, w.y), acc2[2 * c4]);
                                acc2[2 * c4 + 1] =
                                    __ffma2_rn(h2, make_float2(w.z, w.w), acc2[2 * c4 + 1]);
                            }
                        }
                    }
                }
            }
            fence_before();  // the next __syncthreads orders these reads before the next MMA
        }
        if (failed) break;
        // layer 4: the column groups' partial sums of each row meet in shared memory (the A
        // tile, free once the last MMA has completed)
        if (ch > 0) {
#pragma unroll
            for (int o = 0; o < 12; ++o)
                sP[((ch - 1) * kTile + erow) * 12 + o] = (o & 1) ? acc2[o >> 1].y : acc2[o >> 1].x;
        }
        __syncthreads();
        if (ch == 0) {
            const long long gr = g0 + erow;
            if (gr < n) {
#pragma unroll
                for (int o = 0; o < 12; ++o) {
                    float v = (o & 1) ? acc2[o >> 1].y : acc2[o >> 1].x;
                    for (int g = 1; g < kGroups; ++g) v += sP[((g - 1) * kTile + erow) * 12 + o];
                    out[gr * 12 + o] = v + sF[PF_B4 + o];
                }
            }
        }
        __syncthreads();
    }

    if (failed && tid == 0) {
        atomicExch(flag, 1);
        // let work already issued finish before the memory it targets goes away
        if (ld_pending) mbar_wait(bar_ld, ph_ld ^ 1u);
        if (mma_pending) mbar_wait(bar_mma, ph_mma ^ 1u);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

}  // namespace

int forward_fused(rp_surrogate_s *s, long long n, const float *x, float *out, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int rc = ensure_pack(s, st);
    if (rc) return rc;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    RP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SM_TOTAL));
    RP_CUDA_TRY(cudaMemsetAsync(s->fflag, 0, sizeof(int), st));
    const long long tiles = (n + kTile - 1) / kTile;
    const int grid = (int)std::min<long long>(tiles, (long long)sm_count(dev));
    k_mlp_fused<<<grid, kThreads, SM_TOTAL, st>>>(s->pack, x, out, n, s->fflag, wait_cycles(s));
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

int fused_status(rp_surrogate_s *s, cudaStream_t st)
{
    int f = 0;
    RP_CUDA_TRY(cudaMemcpyAsync(&f, s->fflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RP_CUDA_TRY(cudaStreamSynchronize(st));
    if (f) {
        set_error("surrogate: a bounded wait of a tensor-core kernel gave up after %lld SM "
                  "cycles (its work did not complete in time)", wait_cycles(s));
        return RP_ERR_TIMEOUT;
    }
    return RP_OK;
}

}  // namespace rph
