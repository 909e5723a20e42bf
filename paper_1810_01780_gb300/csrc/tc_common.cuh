// tc_common.cuh -- helpers shared by the kernels that run on the 5th-generation tensor cores
// (tcgen05): shared-memory matrix descriptors of the no-swizzle K-major layout, bounded
// mbarrier waits, tensor-memory loads, BF16 packing and the erf-form GELU and its derivative.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace rph {
namespace tc {

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at the maximum SM clock

// Programmatic dependent launch (a kernel launched with launch_chained): waits until the
// kernel before this one in the stream has completed and its writes are visible, then lets the
// next chained kernel be scheduled, so that its launch and its CTAs' setup overlap this
// kernel's work.  Every thread calls it before its first access to global memory that earlier
// work in the stream writes or reads; in a kernel launched without the attribute it returns at
// once.  As each chained kernel releases its successor only after its own wait, a kernel past
// the wait also follows every earlier kernel of the stream.
__device__ __forceinline__ void chain_wait_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t su32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle: start, K-direction core stride (lbo), 8-row
// core stride (sbo), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Waits until the mbarrier `bar` has completed phase `phase`; false once `limit` SM cycles
// have passed without it (the caller then records the failure and drains its work in flight
// with a wait of the default limit before it returns).  Each round first tests the phase
// without blocking, then checks the limit, then waits with mbarrier.try_wait (which may
// suspend the thread for a while): so a limit shorter than the work it waits for always runs
// out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit = kWaitCycles)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The erf-form GELU, gelu(z) = z Phi(z) with Phi the standard normal distribution function,
// and its derivative gelu'(z) = Phi(z) + z phi(z), phi(z) = exp(-z^2 / 2) / sqrt(2 pi) the
// normal density.  Phi is taken from Abramowitz and Stegun, Handbook of Mathematical
// Functions, formula 26.2.17 (Hastings' rational approximation, absolute error < 7.5e-8): for
// x >= 0,
//   1 - Phi(x) = phi(x) t (b1 + t (b2 + t (b3 + t (b4 + t b5)))),  t = 1 / (1 + p x),
// so one density phi(z) = 2^(-z^2 log2(e) / 2 - log2 sqrt(2 pi)) serves both Phi and gelu'.
// Every activation is rounded to BF16 (relative precision 2^-9) before it enters a product,
// far coarser than this error.
struct PhiE {
    float phi;  // Phi(z)
    float d;    // phi(z), the normal density
};
__device__ __forceinline__ PhiE phi_e(float z)
{
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.2316419f, fabsf(z), 1.0f)));
    float p = fmaf(t, 1.330274429f, -1.821255978f);
    p = fmaf(t, p, 1.781477937f);
    p = fmaf(t, p, -0.356563782f);
    p = fmaf(t, p, 0.319381530f);
    p *= t;
    float d;
    asm("ex2.approx.ftz.f32 %0, %1;"
        : "=f"(d)
        : "f"(fmaf(z * z, -0.72134752044448170f, -1.3257480647361594f)));
    const float q = p * d;  // 1 - Phi(|z|)
    PhiE r;
    r.phi = z >= 0.0f ? 1.0f - q : q;
    r.d = d;
    return r;
}
// phi_e of two values with the same operations, the FMA-pipe ones as packed FP32 pairs (one
// instruction for both lanes, each rounded as the scalar operation): the same results
__device__ __forceinline__ void phi_e2(float2 z, float2 &phi, float2 &d)
{
    float2 t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.x) : "f"(fmaf(0.2316419f, fabsf(z.x), 1.0f)));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.y) : "f"(fmaf(0.2316419f, fabsf(z.y), 1.0f)));
    float2 p = __ffma2_rn(t, make_float2(1.330274429f, 1.330274429f),
                          make_float2(-1.821255978f, -1.821255978f));
    p = __ffma2_rn(t, p, make_float2(1.781477937f, 1.781477937f));
    p = __ffma2_rn(t, p, make_float2(-0.356563782f, -0.356563782f));
    p = __ffma2_rn(t, p, make_float2(0.319381530f, 0.319381530f));
    p = __fmul2_rn(p, t);
    const float2 a = __ffma2_rn(__fmul2_rn(z, z), make_float2(-0.72134752044448170f, -0.72134752044448170f),
                                make_float2(-1.3257480647361594f, -1.3257480647361594f));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(d.x) : "f"(a.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(d.y) : "f"(a.y));
    const float2 q = __fmul2_rn(p, d);  // 1 - Phi(|z|)
    const float2 r = __ffma2_rn(q, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
    phi.x = z.x >= 0.0f ? r.x : q.x;
    phi.y = z.y >= 0.0f ? r.y : q.y;
}
__device__ __forceinline__ float gelu(float z) { return z * phi_e(z).phi; }
__device__ __forceinline__ float2 gelu2(float2 z)
{
    float2 phi, d;
    phi_e2(z, phi, d);
    return __fmul2_rn(z, phi);
}
__device__ __forceinline__ float gelu_prime(float z)
{
    const PhiE r = phi_e(z);
    return fmaf(z, r.d, r.phi);
}
__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
// Byte offset of the 8 consecutive k (k0 % 8 == 0) of row `row` in the A tile: 128 rows x 256
// BF16 columns as 8 x 8 core matrices of 128 contiguous bytes (a row's 8 columns in 16 bytes),
// core (row / 8, k / 8) at ((k / 8) * 16 + row / 8) * 128.  Read as an operand with K = row
// and M (or N) = column, the same bytes are the MN-major no-swizzle image of the transposed
// tile, so training stores each 128-row tile of activations and gradients in this layout
// ("operand image", 64 KB): the forward and backward passes write it with coalesced 16-byte
// stores (a warp's 32 rows of one 8-column group are 512 contiguous bytes) and the weight
// gradients load it whole with bulk copies.
__device__ __forceinline__ uint32_t a_off(int row, int k0)
{
    return (uint32_t)(((k0 >> 3) * 16 + (row >> 3)) * 128 + (row & 7) * 16);
}
constexpr uint32_t kImage = 128u * 256u * 2u;  // bytes of one 128-row operand image
constexpr uint32_t kImage16 = 128u * 16u * 2u;  // the same of 16 columns (x and g4, zero-padded)

// Column sums over a warp's 32 lanes of W (16 or 32) columns: lane L returns the sum over the
// lanes of v[L % W] (recursive halving: at each round a lane keeps the half of its columns its
// lane bit selects and adds the partner's copy of them; for W = 16 a last exchange adds the
// other 16 lanes).  v is consumed.
template <int W>
__device__ __forceinline__ float warp_colsum(float (&v)[W], int lane)
{
#pragma unroll
    for (int k = W / 2; k >= 1; k >>= 1) {
        const bool up = (lane & k) != 0;
#pragma unroll
        for (int j = 0; j < k; ++j) {
            const float send = up ? v[j] : v[j + k];
            const float keep = up ? v[j + k] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, k);
        }
    }
#pragma unroll
    for (int k = W; k < 32; k <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], k);
    return v[0];
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global memory
// to shared memory, completing on the mbarrier `bar` (whose transaction count the caller arms).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace rph
