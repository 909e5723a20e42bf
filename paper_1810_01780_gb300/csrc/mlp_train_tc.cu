// mlp_train_tc.cu -- the surrogate's 256 x 256 layers in training, on the 5th-generation
// tensor cores (tcgen05).
//
// Two kernels cover the three hidden 256 -> 256 layers:
//   k_tc_dense<EPI>: C[128 rows x 128 columns] = A[128 x 256] B^T per CTA (one row tile and one
//     half of the 256 output columns each), with the FP32 rows of A converted to BF16 into the
//     no-swizzle K-major image in shared memory, the packed BF16 B image (256 n x 256 k, 128 KB)
//     brought in by bulk copy, 16 tcgen05.mma (M 128, N 128, K 16, reading the half's n-cores)
//     into a 128-column tensor-memory accumulator, and an epilogue per
//     row: forward (EPI_FWD) z = C + b, keeping z and gelu(z); backward (EPI_BWD)
//     C * gelu'(z) of the layer below.  Forward takes B[n][k] = W[k][n] (the inference
//     image), backward B[n][k] = W[n][k] (so that C = g W^T).
//   k_tc_wgrad: dW[in][out] += sum over rows s of H[s][in] g[s][out]: M = in (two halves of
//     128), N = out (one half of 128 per CTA), K = rows.  A CTA runs over chunks of 128 rows,
//     staging H^T and its half of g^T as BF16 K-major images (each thread gathers 8 rows of one
//     column into a 16-byte core row), accumulating both M halves in tensor memory (256
//     columns), and adds its sums to dW with vector atomics at the end; the bias gradient
//     (column sums of g) comes along from the staging loads.
// Arithmetic is that of the CUDA-core GEMMs they replace: BF16 operands, FP32 products and
// sums, FP32 bias, GELU and GELU'.  Every mbarrier wait is bounded (the surrogate's wait limit);
// a CTA that gives up sets the error flag, waits (with the default bound) for its work in
// flight, frees its tensor memory and returns.
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

enum { EPI_FWD = 0, EPI_BWD = 1 };

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128 (each CTA
// computes one half of the 256 output columns)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

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

// shared memory map of k_tc_dense (bytes)
constexpr uint32_t DN_A = 0;                  // 128 x 256 BF16 A image (64 KB)
constexpr uint32_t DN_B = 65536;              // 256 x 256 BF16 B image (128 KB)
constexpr uint32_t DN_BAR = DN_B + kImgB;     // two mbarriers, TMEM slot, abort word
constexpr uint32_t DN_TOTAL = DN_BAR + 32;
static_assert(DN_TOTAL <= 227 * 1024, "shared memory map exceeds a CTA's limit");

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_dense(const float *__restrict__ A, long long n, const unsigned char *__restrict__ Bimg,
               const float *__restrict__ bias, const float *__restrict__ Zin,
               float *__restrict__ Zout, float *__restrict__ Out, int *flag, long long wait)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + DN_BAR);  // [0] B in, [1] MMAs done
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + DN_BAR + 16);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + DN_BAR + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_ld = su32(&bar[0]), bar_mma = su32(&bar[1]);
    const uint32_t a_base = su32(sm + DN_A), b_base = su32(sm + DN_B);
    const long long g0 = (long long)blockIdx.x * kRows;
    const int half = (int)blockIdx.y;  // output columns 128 half .. + 127

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_ld) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_cta = 0;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_ld), "r"(kImgB)
                     : "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    b_base + c * 32768u),
                "l"(Bimg + c * 32768), "r"(32768u), "r"(bar_ld)
                : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A rows -> BF16 K-major image: 128 rows x 32 chunks of 8 columns, 8 chunks per thread
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
        const int c = tid + i * kThreads, row = c >> 5, k0 = (c & 31) * 8;
        const long long gr = g0 + row;
        float4 lo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), hi = lo;
        if (gr < n) {
            const float4 *src = reinterpret_cast<const float4 *>(A + gr * 256 + k0);
            lo = __ldg(src);
            hi = __ldg(src + 1);
        }
        *reinterpret_cast<uint4 *>(sm + DN_A + a_off(row, k0)) =
            make_uint4(pack2(lo.x, lo.y), pack2(lo.z, lo.w), pack2(hi.x, hi.y), pack2(hi.z, hi.w));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *slot;
    bool ld_pending = tid == 0, mma_pending = false;
    if (tid == 0) {
        if (mbar_wait(bar_ld, 0, wait)) {
            ld_pending = false;
            // the half's 16 n-cores of each k-core row of the B image: start 2048 B further
#pragma unroll
            for (int s = 0; s < 16; ++s)
                mma_f16(tmem, sdesc(a_base + s * 4096u, 2048u, 128u),
                        sdesc(b_base + (uint32_t)half * 2048u + s * 8192u, 4096u, 128u), (uint32_t)s);
            mma_commit(bar_mma);
            mma_pending = true;
        } else {
            *abort_cta = 1;
        }
    }
    __syncthreads();
    bool failed = *abort_cta != 0;
    if (!failed && !mbar_wait(bar_mma, 0, wait)) *abort_cta = 1;
    fence_after();
    __syncthreads();
    failed = *abort_cta != 0;
    if (!failed) {
        if (tid == 0) mma_pending = false;
        const int q = warp & 3, ch = warp >> 2, row = q * 32 + lane;
        const long long gr = g0 + row;
        {
            const int tcol = ch * 32, col0 = half * 128 + tcol;
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)tcol, v);
            if (gr < n) {
                float *o = Out + gr * 256 + col0;
                if (EPI == EPI_FWD) {
                    float *zo = Zout + gr * 256 + col0;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        float4 z, h;
                        z.x = __uint_as_float(v[j]) + bias[col0 + j];
                        z.y = __uint_as_float(v[j + 1]) + bias[col0 + j + 1];
                        z.z = __uint_as_float(v[j + 2]) + bias[col0 + j + 2];
                        z.w = __uint_as_float(v[j + 3]) + bias[col0 + j + 3];
                        h.x = gelu(z.x);
                        h.y = gelu(z.y);
                        h.z = gelu(z.z);
                        h.w = gelu(z.w);
                        if (zo) *reinterpret_cast<float4 *>(zo + j) = z;
                        *reinterpret_cast<float4 *>(o + j) = h;
                    }
                } else {
                    const float *zi = Zin + gr * 256 + col0;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 z = *reinterpret_cast<const float4 *>(zi + j);
                        float4 g;
                        g.x = __uint_as_float(v[j]) * gelu_grad(z.x);
                        g.y = __uint_as_float(v[j + 1]) * gelu_grad(z.y);
                        g.z = __uint_as_float(v[j + 2]) * gelu_grad(z.z);
                        g.w = __uint_as_float(v[j + 3]) * gelu_grad(z.w);
                        *reinterpret_cast<float4 *>(o + j) = g;
                    }
                }
            }
        }
    }
    if (failed && tid == 0) {
        atomicExch(flag, 1);
        // let work already issued finish before the memory it targets goes away
        if (ld_pending) mbar_wait(bar_ld, 0);
        if (mma_pending) mbar_wait(bar_mma, 0);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u)
                     : "memory");
    }
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
    k_tc_wgrad(const float *__restrict__ H, const float *__restrict__ G, long long n,
               float *__restrict__ dW, float *__restrict__ db, int *flag, long long wait)
{
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

int tc_dense(bool forward, const float *A, long long n, const unsigned char *Bimg,
             const float *bias, const float *Zin, float *Zout, float *Out, int *flag,
             long long wait, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    const dim3 grid((unsigned)((n + kRows - 1) / kRows), 2);  // row tiles x column halves
    if (forward) {
        RP_CUDA_TRY(cudaFuncSetAttribute(k_tc_dense<EPI_FWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DN_TOTAL));
        k_tc_dense<EPI_FWD><<<grid, kThreads, DN_TOTAL, st>>>(A, n, Bimg, bias, Zin, Zout, Out, flag, wait);
    } else {
        RP_CUDA_TRY(cudaFuncSetAttribute(k_tc_dense<EPI_BWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DN_TOTAL));
        k_tc_dense<EPI_BWD><<<grid, kThreads, DN_TOTAL, st>>>(A, n, Bimg, bias, Zin, Zout, Out, flag, wait);
    }
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

int tc_wgrad(const float *H, const float *G, long long n, float *dW, float *db, int *flag,
             long long wait, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    const long long chunks = (n + kChunk - 1) / kChunk;
    // chunks x column halves, at most two CTAs per SM in all
    const dim3 grid((unsigned)std::min<long long>(chunks, (long long)sm_count(dev)), 2);
    RP_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WG_TOTAL));
    k_tc_wgrad<<<grid, kThreads, WG_TOTAL, st>>>(H, G, n, dW, db, flag, wait);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

}  // namespace rph
