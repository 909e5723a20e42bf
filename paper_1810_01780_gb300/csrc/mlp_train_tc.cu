// mlp_train_tc.cu -- the weight gradients of all five layers of the surrogate in training, on
// the 5th-generation tensor cores (tcgen05), in one launch.
//
//   k_tc_wgrad: D = A^T B over the batch's rows with M = A's 256 columns (one half of 128 per
//     CTA), N = B's columns (one half of 128 per CTA for the hidden layers), K = rows;
//     blockIdx.z selects the job, blockIdx.y the M half and N half, and
//     blockIdx.x one of the job's interleaved shares of the 128-row tiles (CTAs past a job's
//     shares return at once).  The jobs: dW_l = H_l^T g_l of the hidden layers (N 256), the
//     last layer's dW4 = H4^T g4 (N 16: g4's 12 columns zero-padded) and the first layer's
//     dW0^T = g0^T x (N 16: x's 3 columns zero-padded).  The forward and backward passes leave
//     these matrices as BF16 operand images (tc_common.cuh), which are the MN-major no-swizzle
//     images of their transposes: a CTA bulk-copies its half of each tile's A image (32 KB) and
//     its part of the B image (32 or 4 KB) into one of several shared-memory stages, so the
//     copies of the next tiles overlap the MMAs of this one, accumulates over its tiles in
//     tensor memory and adds its sums to dW with atomics at the end (the fewer tile shares, the
//     less atomic traffic: it is one copy of dW per share).  (The bias gradients are summed by the passes
//     that produce the g.)
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
constexpr uint32_t kImgB = 256u * 256u * 2u;  // a packed 256 x 256 BF16 B image

// instruction descriptor: D FP32, A and B BF16, both MN-major (bits 15 and 16), M = 128; N
// (bits 17..22, N / 8) per job
constexpr uint32_t kIdescT = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((128u >> 4) << 24);

// shared memory map of k_tc_wgrad (bytes): stages of (the A image's M half, 32 KB; the B
// image's N half, 32 KB, or the 16-column image, 4 KB): three of 64 KB for the hidden layers,
// five of 36 KB for the thin ones (whose short MMAs leave the copies' latency exposed unless
// more tiles are in flight); then the barriers full[s] (the copies into stage s landed) and
// done[s] (the MMAs have read stage s)
constexpr uint32_t WG_HALF = kImage / 2;
constexpr uint32_t WG_STAGE = WG_HALF + kImage;
constexpr int kStagesWide = 3, kStagesThin = 5, kMaxStages = 6;
constexpr uint32_t WG_BAR = 2 * WG_STAGE;
constexpr uint32_t WG_SLOT = WG_BAR + 2 * kMaxStages * 8;  // TMEM address, abort word
constexpr uint32_t WG_TOTAL = WG_SLOT + 32;
static_assert(kStagesThin * (WG_HALF + kImage16) <= WG_BAR && kStagesWide * 2 * WG_HALF <= WG_BAR,
              "the stages fit");
static_assert(WG_TOTAL <= 227 * 1024, "shared memory map exceeds a CTA's limit");

// rows 128 h .. 128 h + 127 (h = blockIdx.y % 2) of D, and for the hidden layers columns
// 128 nh .. 128 nh + 127 (nh = blockIdx.y / 2), over the tiles blockIdx.x, + shares, ...
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_wgrad(const WgradArgs args, long long n_tiles, int *flag, long long wait)
{
    const WgradJob &J = args.job[blockIdx.z];
    const long long shares = J.shares;
    const bool wide = J.n == 256;
    const int half = (int)(blockIdx.y & 1), nh = (int)(blockIdx.y >> 1);
    if ((long long)blockIdx.x >= shares || (!wide && nh)) return;  // uniform over the CTA
    const unsigned char *__restrict__ H = J.A;
    const unsigned char *__restrict__ G = J.B;
    float *__restrict__ dW = J.dW;
    const uint32_t b_bytes = wide ? WG_HALF : kImage16;  // the B operand of a tile
    const uint32_t b_stride = wide ? kImage : kImage16;  // bytes per tile of the B image
    const uint32_t b_skip = wide ? (uint32_t)nh * WG_HALF : 0u;
    const uint32_t idesc = kIdescT | ((wide ? 128u : 16u) >> 3) << 17;
    const int S = wide ? kStagesWide : kStagesThin;  // pipeline stages
    const uint32_t stage_bytes = WG_HALF + b_bytes;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + WG_BAR);  // full[0..S), done at +kMaxStages
    uint64_t *done = bar + kMaxStages;
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + WG_SLOT);
    volatile int *abort_cta = reinterpret_cast<volatile int *>(sm + WG_SLOT + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long cnt = (n_tiles - blockIdx.x + shares - 1) / shares;  // >= 1

    if (tid == 0) {
        for (int b = 0; b < 2 * kMaxStages; ++b)
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
    const uint32_t tmem = *slot;
    chain_wait_release();  // the images come from the forward and backward passes

    if (tid == 0) {
        // One thread copies and issues.  Tile i (the i-th of this CTA) uses stage i % S, as
        // that stage's (i / S)-th use: its copies complete phase i / S of full[i % S] and its
        // MMAs commit phase i / S of done[i % S].  ld[s] / mm[s]: the tile whose copies / MMAs
        // on stage s are in flight, -1 if none (drained on failure).
        long long ld[kMaxStages], mm[kMaxStages];
        for (int s2 = 0; s2 < kMaxStages; ++s2) ld[s2] = mm[s2] = -1;
        bool failed = false;
        auto load = [&](long long i) {
            const int st = (int)(i % S);
            const long long t = blockIdx.x + i * shares;
            const uint32_t base = su32(sm + st * stage_bytes), fb = su32(&bar[st]);
            mbar_expect(fb, stage_bytes);
            bulk_g2s(base, H + t * kImage + half * WG_HALF, WG_HALF, fb);
            bulk_g2s(base + WG_HALF, G + t * b_stride + b_skip, b_bytes, fb);
            ld[st] = i;
        };
        auto par = [S](long long i) { return (uint32_t)((i / S) & 1); };
        for (long long j = 0; j < cnt && j < S; ++j) load(j);
        for (long long i = 0; i < cnt && !failed; ++i) {
            const int st = (int)(i % S);
            if (!mbar_wait(su32(&bar[st]), par(i), wait)) {
                failed = true;
                break;
            }
            ld[st] = -1;
            const uint32_t a0 = su32(sm + st * stage_bytes), b0 = a0 + WG_HALF;
            // K step k: rows 16 k .. 16 k + 15, two 8-row core groups 128 bytes apart (the
            // K-direction stride); 8-column groups 2048 bytes apart (the M / N-direction stride)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint64_t ad = sdesc(a0 + k * 256u, 128u, 2048u);
                const uint64_t bd = sdesc(b0 + k * 256u, 128u, 2048u);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(i > 0 || k > 0))
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&done[st]))
                         : "memory");
            mm[st] = i;
            // the stage of tile i - 1, once its MMAs are done, takes tile i - 1 + S
            if (i >= 1 && i - 1 + S < cnt) {
                const int o = (int)((i - 1) % S);
                if (!mbar_wait(su32(&done[o]), par(i - 1), wait)) {
                    failed = true;
                    break;
                }
                mm[o] = -1;
                load(i - 1 + S);
            }
        }
        if (!failed) {  // the last tile's MMAs, and with them all before, done
            if (mbar_wait(su32(&done[(cnt - 1) % S]), par(cnt - 1), wait)) {
                for (int s2 = 0; s2 < kMaxStages; ++s2) mm[s2] = -1;
            } else {
                failed = true;
            }
        }
        if (failed) {
            atomicExch(flag, 1);
            *abort_cta = 1;
            for (int s2 = 0; s2 < S; ++s2) {  // drain with the default bound
                if (ld[s2] >= 0) mbar_wait(su32(&bar[s2]), par(ld[s2]));
                if (mm[s2] >= 0) mbar_wait(su32(&done[s2]), par(mm[s2]));
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (!*abort_cta) {
        // TMEM lane m: row 128 half + m of D; column c: column c (quarter q = warp % 4 reads
        // lanes 32 q .. 32 q + 31)
        const int q = warp & 3, ch = warp >> 2;
        const int m = half * 128 + q * 32 + lane;
        if (wide) {  // column group warp / 4: columns 128 nh + 32 (warp / 4) ..
            const int n0 = nh * 128 + ch * 32;
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32), v);
            float *d = dW + (long long)m * 256 + n0;  // 16-byte aligned: n0 % 32 == 0
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d + j),
                             "f"(__uint_as_float(v[j])), "f"(__uint_as_float(v[j + 1])),
                             "f"(__uint_as_float(v[j + 2])), "f"(__uint_as_float(v[j + 3]))
                             : "memory");
        } else if (ch == 0) {  // 16 columns, warps 0..3
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16), v);
            if (J.out == WG_OUT_LAST) {
                float *d = dW + (long long)m * 12;  // 16-byte aligned: 48 m bytes
#pragma unroll
                for (int j = 0; j < 12; j += 4)
                    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d + j),
                                 "f"(__uint_as_float(v[j])), "f"(__uint_as_float(v[j + 1])),
                                 "f"(__uint_as_float(v[j + 2])), "f"(__uint_as_float(v[j + 3]))
                                 : "memory");
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(dW + c * 256 + m, __uint_as_float(v[c]));
            }
        }
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
    const long long off = l * (long long)kImgB + bimg_off(k, nn);
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

int tc_wgrad(WgradArgs &a, long long n, int *flag, long long wait, cudaStream_t st)
{
    if (n <= 0) return RP_OK;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    const long long tiles = (n + 127) / 128;
    // one CTA per SM: a few for each thin job (little to copy and multiply), the rest split
    // evenly among the three hidden layers' four (M half, N half) blocks
    const long long sms = sm_count(dev);
    const long long thin = std::max(1LL, std::min(tiles, std::min(8LL, sms / 19)));
    const long long wide = std::max(1LL, std::min(tiles, (sms - 4 * thin) / 12));
    for (int j = 0; j < 5; ++j) a.job[j].shares = (int32_t)(j < 3 ? wide : thin);
    const dim3 grid((unsigned)std::max(wide, thin), 4, 5);  // y: M half + 2 x N half
    RP_CUDA_TRY(cudaFuncSetAttribute(k_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WG_TOTAL));
    return launch_chained(k_tc_wgrad, grid, dim3(kThreads), WG_TOTAL, st, (const WgradArgs)a,
                          tiles, flag, wait);
}

}  // namespace rph
