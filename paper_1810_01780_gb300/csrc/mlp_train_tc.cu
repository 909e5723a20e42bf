// mlp_train_tc.cu -- the weight gradients of the surrogate's three hidden 256 x 256 layers in
// training, on the 5th-generation tensor cores (tcgen05), all three layers in one launch.
//
//   k_tc_wgrad: dW[in][out] += sum over rows s of H[s][in] g[s][out]: M = in (two halves of
//     128), N = out (one half of 128 per CTA), K = rows; blockIdx.z selects the layer.  A CTA
//     runs over chunks of 128 rows, staging H^T and its half of g^T as BF16 K-major images (each
//     thread gathers 8 rows of one column into a 16-byte core row), accumulating both M halves
//     in tensor memory (256 columns), and adds its sums to dW with vector atomics at the end;
//     the bias gradient (column sums of g) comes along from the staging loads.
//   k_pack_t: the backward data pass's B images of W1..W3 (B[n][k] = W[n][k]).
// Arithmetic: BF16 operands, FP32 products and sums.  Every mbarrier wait is bounded (the
// surrogate's wait limit); a CTA that gives up sets the error flag, waits (with the default
// bound) for its work in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "rp_internal.h"
#include "tc_common.cuh"

namespace rph {

namespace {

using namespace tc;

constexpr int kThreads = 512;  // 16 warps: lane quarter (warp % 4) x column group (warp / 4)
constexpr int kRows = 128;     // rows per tile (M of one MMA)
constexpr uint32_t kImgB = 256u * 256u * 2u;  // a packed 256 x 256 BF16 B image

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128 (each CTA
// computes one half of the 256 output columns)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// shared memory map of k_tc_wgrad (bytes): A = H^T chunk as two 128 x 128 halves (32 KB each;
// core (k/8, m/8) at ((k/8) * 16 + m/8) * 128), B = the CTA's 128 columns of g^T, 128 x 128
// (32 KB, same core layout)
constexpr uint32_t WG_A = 0;
constexpr uint32_t WG_B = 65536;
constexpr uint32_t WG_BAR = WG_B + 32768;
constexpr uint32_t WG_TOTAL = WG_BAR + 32;
constexpr int kChunk = 128;  // rows (K) per chunk

// dW[:, 128 h .. 128 h + 127] (h = blockIdx.y) over the chunks blockIdx.x, + gridDim.x, ...
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_wgrad(const WgradArgs args, long long n, int *flag, long long wait)
{
    const float *__restrict__ H = args.H[blockIdx.z];
    const float *__restrict__ G = args.G[blockIdx.z];
    float *__restrict__ dW = args.dW[blockIdx.z];
    float *__restrict__ db = args.db[blockIdx.z];
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + WG_BAR);  // MMAs done
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + WG_BAR + 16);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + WG_BAR + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_mma = su32(&bar[0]);
    const uint32_t a_base = su32(sm + WG_A), b_base = su32(sm + WG_B);
    const long long n_chunks = (n + kChunk - 1) / kChunk;
    const int half = (int)blockIdx.y;

    if (tid == 0) {
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
    uint32_t ph = 0;
    bool mma_pending = false, failed = false;
    // staging: H^T, column col (all 256) and 8-row chunks kc_a + 2 i; g^T, column gcol of the
    // half and 8-row chunks kc_g + 4 i
    const int col = tid & 255, kc_a = tid >> 8;
    const int gl = tid & 127, gcol = half * 128 + gl, kc_g = tid >> 7;
    float gsum = 0.0f;  // this thread's part of the bias gradient sum_s g[s][gcol]
    int it = 0;
    for (long long chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x, ++it) {
        const long long r0 = chunk * kChunk;
#pragma unroll 2
        for (int i = 0; i < 8; ++i) {
            const int kc = kc_a + 2 * i;  // 8-row chunk 0..15
            float h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const long long r = r0 + kc * 8 + e;
                h[e] = r < n ? __ldg(H + r * 256 + col) : 0.0f;
            }
            const int mh = col >> 7, m = col & 127;
            *reinterpret_cast<uint4 *>(sm + WG_A + mh * 32768 + (kc * 16 + (m >> 3)) * 128 + (m & 7) * 16) =
                make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
        }
#pragma unroll 2
        for (int i = 0; i < 4; ++i) {
            const int kc = kc_g + 4 * i;
            float g[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const long long r = r0 + kc * 8 + e;
                g[e] = r < n ? __ldg(G + r * 256 + gcol) : 0.0f;
                gsum += g[e];
            }
            *reinterpret_cast<uint4 *>(sm + WG_B + (kc * 16 + (gl >> 3)) * 128 + (gl & 7) * 16) =
                make_uint4(pack2(g[0], g[1]), pack2(g[2], g[3]), pack2(g[4], g[5]), pack2(g[6], g[7]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
#pragma unroll
            for (int mh = 0; mh < 2; ++mh)
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    mma_f16(tmem + (uint32_t)(mh * 128),
                            sdesc(a_base + mh * 32768u + s * 4096u, 2048u, 128u),
                            sdesc(b_base + s * 4096u, 2048u, 128u), (uint32_t)(it > 0 || s > 0));
            mma_commit(bar_mma);
            mma_pending = true;
        }
        // the images are rewritten for the next chunk only after these MMAs have read them
        if (!mbar_wait(bar_mma, ph, wait)) *abort_cta = 1;
        ph ^= 1u;
        fence_after();
        __syncthreads();
        if (*abort_cta) {
            failed = true;
            break;
        }
        if (tid == 0) mma_pending = false;
    }
    if (!failed && it > 0) {
        // TMEM column t: M half t / 128, output column 128 half + t % 128; rows m of the half
        // are the lanes (lane quarter q = warp % 4)
        const int q = warp & 3, ch = warp >> 2;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const int tcol = ch * 64 + c * 32, mh = tcol >> 7;
            const int m = mh * 128 + q * 32 + lane, n0 = half * 128 + (tcol & 127);
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)tcol, v);
            float *d = dW + (long long)m * 256 + n0;  // 16-byte aligned: n0 % 32 == 0
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d + j),
                             "f"(__uint_as_float(v[j])), "f"(__uint_as_float(v[j + 1])),
                             "f"(__uint_as_float(v[j + 2])), "f"(__uint_as_float(v[j + 3]))
                             : "memory");
        }
        atomicAdd(db + gcol, gsum);
    }
    if (failed && tid == 0) {
        atomicExch(flag, 1);
        if (mma_pending) mbar_wait(bar_mma, ph ^ 1u);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                     : "memory");
    }
}

// Backward images of the hidden layers: B[n][k] = W[n][k] for W = W1..W3 ([in][out], so that
// C = g W^T), in the same K-major image as the inference pack.
__global__ void k_pack_t(const float *__restrict__ p, unsigned char *__restrict__ img,
                         long long w1, long long w2, long long w3)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 3 * 65536) return;
    const int l = (int)(i / 65536), e = (int)(i % 65536), nn = e / 256, k = e % 256;
    const long long w = l == 0 ? w1 : (l == 1 ? w2 : w3);
    const float v = p[w + (long long)nn * 256 + k];
    const long long off = l * (long long)kImgB + ((k >> 3) * 32 + (nn >> 3)) * 128 + (nn & 7) * 16 + (k & 7) * 2;
    *(__nv_bfloat16 *)(img + off) = __float2bfloat16_rn(v);
}

}  // namespace

int tc_pack_backward(const float *p, unsigned char *img, long long w1, long long w2, long long w3,
                     cudaStream_t st)
{
    k_pack_t<<<(3 * 65536 + 255) / 256, 256, 0, st>>>(p, img, w1, w2, w3);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

int tc_wgrad3(const WgradArgs &a, long long n, int *flag, long long wait, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    const long long chunks = (n + kChunk - 1) / kChunk;
    // chunks x column halves x layers
    const dim3 grid((unsigned)std::min<long long>(chunks, (long long)sm_count(dev)), 2, 3);
    RP_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WG_TOTAL));
    k_tc_wgrad<<<grid, kThreads, WG_TOTAL, st>>>(a, n, flag, wait);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

}  // namespace rph
