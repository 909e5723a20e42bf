// mlp.cu -- the surrogate network: 3 -> 256 -> 256 -> 256 -> 256 -> 12, GELU (erf form),
// BF16 weights and activations into the tensor cores, FP32 accumulation, FP32 master weights
// with Adam.  Forward, loss, backward and the optimiser step are all kernels of this file.
//
// The three hidden 256 x 256 layers train on the 5th-generation tensor cores
// (mlp_train_tc.cu).  The thin first (3 -> 256) and last (256 -> 12) layers use the GEMM
// below: C[M x N] = A[M x K] * B[K x N] with arbitrary strides for A and B (so that the same
// kernel computes X W, dZ W^T and X^T dZ), 64 x 64 x 32 block tiles staged in shared memory
// as BF16, four warps of 32 x 32, mma.sync m16n8k16 (bf16 x bf16 -> f32).  Epilogues: bias,
// bias + GELU (keeping the pre-activation for the backward pass), times GELU'(Z), or split-K
// accumulation with atomics (weight gradients, K = batch).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rp_internal.h"

namespace {

constexpr int kLayers = 5;
constexpr int kDims[kLayers + 1] = {3, 256, 256, 256, 256, 12};
constexpr int BM = 64, BN = 64, BK = 32, kThreads = 128;

enum { EPI_BIAS = 0, EPI_BIAS_GELU = 1, EPI_GELU_GRAD = 2, EPI_ATOMIC = 3 };

struct GemmArgs {
    int M, N, K;
    const float *A;
    long long sAi, sAk;
    const void *B;
    long long sBk, sBj;
    int b_bf16;
    float *C;
    long long ldc;
    const float *bias;
    float *Z;  // EPI_BIAS_GELU: pre-activation out (may be null); EPI_GELU_GRAD: Z in
    float *H;  // EPI_BIAS_GELU: activation out
    int k_chunk;
};

__device__ __forceinline__ float gelu_f(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm(const GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + 8];
    __shared__ __align__(16) __nv_bfloat16 Bt[BN][BK + 8];  // B tile stored n-major
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    int k_begin = 0, k_end = g.K;
    if (EPI == EPI_ATOMIC) {
        k_begin = blockIdx.z * g.k_chunk;
        k_end = min(g.K, k_begin + g.k_chunk);
    }
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const bool a_rows = g.sAi == 1;  // A's rows are contiguous: map threads along i
    const bool b_cols = g.sBj == 1;  // B's columns are contiguous: map threads along j
    const int gq = lane >> 2, q = lane & 3;

    for (int k0 = k_begin; k0 < k_end; k0 += BK) {
#pragma unroll 4
        for (int r = 0; r < (BM * BK) / kThreads; ++r) {
            const int e = tid + r * kThreads;
            const int row = a_rows ? (e % BM) : (e / BK), col = a_rows ? (e / BM) : (e % BK);
            const int i = m0 + row, k = k0 + col;
            float v = 0.0f;
            if (i < g.M && k < k_end) v = g.A[(long long)i * g.sAi + (long long)k * g.sAk];
            As[row][col] = __float2bfloat16_rn(v);
        }
#pragma unroll 4
        for (int r = 0; r < (BN * BK) / kThreads; ++r) {
            const int e = tid + r * kThreads;
            const int col = b_cols ? (e % BN) : (e / BK), kr = b_cols ? (e / BN) : (e % BK);
            const int j = n0 + col, k = k0 + kr;
            __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
            if (j < g.N && k < k_end) {
                const long long o = (long long)k * g.sBk + (long long)j * g.sBj;
                v = g.b_bf16 ? ((const __nv_bfloat16 *)g.B)[o]
                             : __float2bfloat16_rn(((const float *)g.B)[o]);
            }
            Bt[col][kr] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + gq;
                af[mt][0] = *(const uint32_t *)&As[r][kk + 2 * q];
                af[mt][1] = *(const uint32_t *)&As[r + 8][kk + 2 * q];
                af[mt][2] = *(const uint32_t *)&As[r][kk + 2 * q + 8];
                af[mt][3] = *(const uint32_t *)&As[r + 8][kk + 2 * q + 8];
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = wn * 32 + nt * 8 + gq;
                bf[nt][0] = *(const uint32_t *)&Bt[c][kk + 2 * q];
                bf[nt][1] = *(const uint32_t *)&Bt[c][kk + 2 * q + 8];
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
        }
        __syncthreads();
    }
    // epilogue: accumulator (row gq / gq+8, columns 2q, 2q+1) of each 16 x 8 tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = m0 + wm * 32 + mt * 16 + gq + (h >= 2 ? 8 : 0);
                const int j = n0 + wn * 32 + nt * 8 + 2 * q + (h & 1);
                if (i >= g.M || j >= g.N) continue;
                float v = acc[mt][nt][h];
                const long long o = (long long)i * g.ldc + j;
                if (EPI == EPI_ATOMIC) {
                    atomicAdd(&g.C[o], v);
                } else if (EPI == EPI_BIAS) {
                    g.C[o] = v + g.bias[j];
                } else if (EPI == EPI_BIAS_GELU) {
                    v += g.bias[j];
                    if (g.Z) g.Z[o] = v;
                    g.H[o] = gelu_f(v);
                } else {  // EPI_GELU_GRAD
                    g.C[o] = v * gelu_grad_f(g.Z[o]);
                }
            }
}

// Loss (per sample: logistic loss of each slot's existence logit + y times half the squared
// error of its five regression outputs) and its gradient with respect to the outputs.
__global__ void k_loss(const float *out, const float *y, const float *t, long long n, float *g,
                       double *loss)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float L = 0.0f;
    if (b < n) {
        const float inv_n = 1.0f / (float)n;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float z = out[b * 12 + 6 * k], yk = y[b * 2 + k];
            L += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - yk * z;
            g[b * 12 + 6 * k] = (1.0f / (1.0f + expf(-z)) - yk) * inv_n;
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const float d = out[b * 12 + 6 * k + 1 + j] - t[b * 10 + 5 * k + j];
                L += 0.5f * yk * d * d;
                g[b * 12 + 6 * k + 1 + j] = yk * d * inv_n;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)L);
}

// db[j] += sum over rows of g[row, j]
__global__ void k_colsum(const float *g, long long n, int N, float *db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const long long per = (n + gridDim.y - 1) / gridDim.y;
    const long long lo = blockIdx.y * per, hi = lo + per < n ? lo + per : n;
    float s = 0.0f;
    for (long long r = lo; r < hi; ++r) s += g[r * N + j];
    atomicAdd(&db[j], s);
}

__global__ void k_adam(float *p, __nv_bfloat16 *pb, const float *gr, float *m, float *v,
                       long long n, float lr, float c1, float c2)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gr[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

long long layer_w(int l)
{
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)kDims[i] * kDims[i + 1] + kDims[i + 1];
    return o;
}
long long layer_b(int l) { return layer_w(l) + (long long)kDims[l] * kDims[l + 1]; }

struct LayerOffs {
    long long w[kLayers], b[kLayers];  // offsets of W_l and b_l in the flat parameter vector
};

// Inference operands of the fused kernel (layout: kPackW, kPackF and PF_* in rp_internal.h):
// the hidden layers' weights W1..W3 as BF16 B operands (B[n][k] = W[k][n]) in the tensor
// cores' no-swizzle K-major shared-memory image (8 x 8 core matrices of 128 contiguous bytes;
// core (k/8, n/8) at ((k/8) * 32 + n/8) * 128), then the FP32 block.
using rph::kPackF;
using rph::kPackW;
__global__ void k_pack(const float *__restrict__ p, unsigned char *__restrict__ pack, const LayerOffs L)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < 3 * 65536) {
        const int l = (int)(i / 65536), e = (int)(i % 65536), k = e / 256, n = e % 256;
        const float w = p[L.w[l + 1] + (long long)k * 256 + n];
        const long long off = l * kPackW + ((k >> 3) * 32 + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
        *(__nv_bfloat16 *)(pack + off) = __float2bfloat16_rn(w);
        return;
    }
    const long long j = i - 3 * 65536;
    if (j >= kPackF) return;
    float v = 0.0f;
    if (j < rph::PF_B0)
        v = __bfloat162float(__float2bfloat16_rn(p[L.w[0] + (j - rph::PF_W0)]));
    else if (j < rph::PF_B1)
        v = p[L.b[0] + (j - rph::PF_B0)];
    else if (j < rph::PF_W4)
        v = p[L.b[1 + (int)((j - rph::PF_B1) / 256)] + (j - rph::PF_B1) % 256];
    else if (j < rph::PF_B4)
        v = __bfloat162float(__float2bfloat16_rn(p[L.w[4] + (j - rph::PF_W4)]));
    else if (j < rph::PF_B4 + 12)
        v = p[L.b[4] + (j - rph::PF_B4)];
    ((float *)(pack + 3 * kPackW))[j] = v;
}
long long n_params() { return layer_w(kLayers); }

}  // namespace

namespace rph {

static void free_acts(rp_surrogate_s *s)
{
    for (int l = 0; l < 4; ++l) {
        cudaFree(s->Z[l]);
        s->Z[l] = nullptr;
    }
    for (int l = 1; l < 5; ++l) {
        cudaFree(s->H[l]);
        s->H[l] = nullptr;
    }
    cudaFree(s->out);
    cudaFree(s->g0);
    cudaFree(s->g1);
    s->out = s->g0 = s->g1 = nullptr;
    s->cap = 0;
}

int ensure_acts(rp_surrogate_s *s, long long n)
{
    if (n <= s->cap) return RP_OK;
    RP_CUDA_TRY(cudaDeviceSynchronize());
    free_acts(s);
    const long long cap = n + n / 4;
    for (int l = 0; l < 4; ++l) RP_CUDA_TRY(cudaMalloc(&s->Z[l], sizeof(float) * cap * 256));
    for (int l = 1; l < 5; ++l) RP_CUDA_TRY(cudaMalloc(&s->H[l], sizeof(float) * cap * 256));
    RP_CUDA_TRY(cudaMalloc(&s->out, sizeof(float) * cap * 12));
    RP_CUDA_TRY(cudaMalloc(&s->g0, sizeof(float) * cap * 256));
    RP_CUDA_TRY(cudaMalloc(&s->g1, sizeof(float) * cap * 256));
    s->cap = cap;
    return RP_OK;
}

template <int EPI>
static int gemm(const GemmArgs &g, cudaStream_t st)
{
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, 1);
    if (EPI == EPI_ATOMIC) grid.z = (g.K + g.k_chunk - 1) / g.k_chunk;
    k_gemm<EPI><<<grid, kThreads, 0, st>>>(g);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

// forward pass of n rows for training, keeping the pre-activations: layers 1..3 (256 -> 256)
// on the tensor cores, layers 0 (3 -> 256) and 4 (256 -> 12) with the kernel above
int forward(rp_surrogate_s *s, long long n, const float *x, float *out, bool train,
                   cudaStream_t st)
{
    int rc = ensure_pack(s, st);
    if (rc) return rc;
    const float *h = x;
    for (int l = 0; l < kLayers; ++l) {
        if (l >= 1 && l <= 3) {
            if ((rc = tc_dense(true, h, n, s->pack + (l - 1) * kPackW, s->p + layer_b(l), nullptr,
                               train ? s->Z[l] : nullptr, s->H[l + 1], s->fflag, st)))
                return rc;
            h = s->H[l + 1];
            continue;
        }
        GemmArgs g;
        memset(&g, 0, sizeof g);
        g.M = (int)n;
        g.N = kDims[l + 1];
        g.K = kDims[l];
        g.A = h;
        g.sAi = kDims[l];
        g.sAk = 1;
        g.B = s->pb + layer_w(l);
        g.sBk = kDims[l + 1];
        g.sBj = 1;
        g.b_bf16 = 1;
        g.ldc = kDims[l + 1];
        g.bias = s->p + layer_b(l);
        if (l < kLayers - 1) {
            g.Z = train ? s->Z[l] : nullptr;
            g.H = s->H[l + 1];
            g.C = s->H[l + 1];
            rc = gemm<EPI_BIAS_GELU>(g, st);
            h = s->H[l + 1];
        } else {
            g.C = out;
            rc = gemm<EPI_BIAS>(g, st);
        }
        if (rc) return rc;
    }
    return RP_OK;
}

// loss and parameter gradient (into s->grad) of n rows
static int loss_grad(rp_surrogate_s *s, long long n, const float *x, const float *y,
                     const float *t, double *loss_host, cudaStream_t st)
{
    int rc = ensure_acts(s, n);
    if (rc) return rc;
    if ((rc = forward(s, n, x, s->out, true, st))) return rc;
    RP_CUDA_TRY(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
    RP_CUDA_TRY(cudaMemsetAsync(s->grad, 0, sizeof(float) * n_params(), st));
    float *g_cur = s->g0, *g_next = s->g1;
    k_loss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->out, y, t, n, g_cur, s->loss);
    RP_CUDA_TRY(cudaGetLastError());
    const int k_chunk = 512;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int in = kDims[l], outd = kDims[l + 1];
        const float *h = l == 0 ? x : s->H[l];
        if (l >= 1 && l <= 3) {
            // hidden 256 x 256 layers on the tensor cores: dW_l = H_l^T g, then
            // g_{l-1} = (g W_l^T) * GELU'(Z_{l-1})
            if ((rc = tc_wgrad(h, g_cur, n, s->grad + layer_w(l), s->fflag, st))) return rc;
            dim3 cg((outd + 127) / 128, 64);
            k_colsum<<<cg, 128, 0, st>>>(g_cur, n, outd, s->grad + layer_b(l));
            RP_CUDA_TRY(cudaGetLastError());
            if ((rc = tc_dense(false, g_cur, n, s->pack_t + (l - 1) * kPackW, nullptr, s->Z[l - 1],
                               nullptr, g_next, s->fflag, st)))
                return rc;
            float *tmp = g_cur;
            g_cur = g_next;
            g_next = tmp;
            continue;
        }
        // dW_l = H_l^T g  (split over the batch)
        GemmArgs g;
        memset(&g, 0, sizeof g);
        g.M = in;
        g.N = outd;
        g.K = (int)n;
        g.A = h;
        g.sAi = 1;
        g.sAk = in;
        g.B = g_cur;
        g.sBk = outd;
        g.sBj = 1;
        g.b_bf16 = 0;
        g.C = s->grad + layer_w(l);
        g.ldc = outd;
        g.k_chunk = k_chunk;
        if ((rc = gemm<EPI_ATOMIC>(g, st))) return rc;
        dim3 cg((outd + 127) / 128, 64);
        k_colsum<<<cg, 128, 0, st>>>(g_cur, n, outd, s->grad + layer_b(l));
        RP_CUDA_TRY(cudaGetLastError());
        if (l == 0) break;
        // g_{l-1} = (g W_l^T) * GELU'(Z_{l-1})
        GemmArgs d;
        memset(&d, 0, sizeof d);
        d.M = (int)n;
        d.N = in;
        d.K = outd;
        d.A = g_cur;
        d.sAi = outd;
        d.sAk = 1;
        d.B = s->pb + layer_w(l);
        d.sBk = 1;
        d.sBj = outd;
        d.b_bf16 = 1;
        d.C = g_next;
        d.ldc = in;
        d.Z = s->Z[l - 1];
        if ((rc = gemm<EPI_GELU_GRAD>(d, st))) return rc;
        float *tmp = g_cur;
        g_cur = g_next;
        g_next = tmp;
    }
    if (loss_host) {
        RP_CUDA_TRY(cudaMemcpyAsync(loss_host, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        if ((rc = fused_status(s, st))) return rc;  // syncs st
        *loss_host /= (double)n;
    }
    return RP_OK;
}

// loss[1] += loss[0] / n: the running sum of batch losses of an epoch
__global__ void k_acc_loss(double *loss, double inv_n) { loss[1] += loss[0] * inv_n; }

int ensure_pack(rp_surrogate_s *s, cudaStream_t st)
{
    if (!s->pack) {
        RP_CUDA_TRY(cudaMalloc(&s->pack, 3 * kPackW + sizeof(float) * kPackF));
        s->pack_version = -1;
    }
    if (!s->pack_t) {
        RP_CUDA_TRY(cudaMalloc(&s->pack_t, 3 * kPackW));
        s->pack_version = -1;
    }
    if (s->pack_version == s->version) return RP_OK;
    const long long total = 3 * 65536 + kPackF;
    LayerOffs L;
    for (int l = 0; l < kLayers; ++l) {
        L.w[l] = layer_w(l);
        L.b[l] = layer_b(l);
    }
    k_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s->p, s->pack, L);
    RP_CUDA_TRY(cudaGetLastError());
    int rc = tc_pack_backward(s->p, s->pack_t, L.w[1], L.w[2], L.w[3], st);
    if (rc) return rc;
    s->pack_version = s->version;
    return RP_OK;
}

// one Adam step at learning rate lr on the gradient in s->grad
static int adam_step(rp_surrogate_s *s, float lr, cudaStream_t st)
{
    s->step += 1;
    s->version += 1;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)s->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)s->step)));
    const long long np = n_params();
    k_adam<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(s->p, s->pb, s->grad, s->m, s->v, np, lr,
                                                          c1, c2);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
static uint64_t splitmix64(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static const char kMagic[8] = {'R', 'P', 'S', 'U', 'R', '0', '0', '1'};

}  // namespace rph

using namespace rph;

extern "C" {

int rp_surrogate_n_params(void) { return (int)n_params(); }

int rp_surrogate_create(const float *params, rp_surrogate_t *out)
{
    if (!params || !out) {
        set_error("rp_surrogate_create: null argument");
        return RP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    rp_surrogate_s *s = new (std::nothrow) rp_surrogate_s();
    if (!s) return RP_ERR_OOM;
    memset(s, 0, sizeof *s);
    cudaGetDevice(&s->device);
    const long long np = n_params();
    cudaError_t e = cudaMalloc(&s->p, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&s->m, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&s->v, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&s->grad, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&s->pb, sizeof(__nv_bfloat16) * np);
    if (e == cudaSuccess) e = cudaMalloc(&s->loss, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->fflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->fflag, 0, sizeof(int));
    if (e != cudaSuccess) {
        rp_surrogate_destroy(s);
        return cuda_fail(e, "rp_surrogate_create");
    }
    int rc = rp_surrogate_set_params(s, params);
    if (rc) {
        rp_surrogate_destroy(s);
        return rc;
    }
    *out = s;
    return RP_OK;
}

int rp_surrogate_destroy(rp_surrogate_t s)
{
    if (!s) return RP_OK;
    free_pipe(s);
    free_acts(s);
    cudaFree(s->p);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->grad);
    cudaFree(s->pb);
    cudaFree(s->loss);
    cudaFree(s->pack);
    cudaFree(s->pack_t);
    cudaFree(s->fflag);
    delete s;
    return RP_OK;
}

int rp_surrogate_set_params(rp_surrogate_t s, const float *params)
{
    if (!s || !params) {
        set_error("rp_surrogate_set_params: null argument");
        return RP_ERR_INVALID_ARG;
    }
    const long long np = n_params();
    RP_CUDA_TRY(cudaMemcpy(s->p, params, sizeof(float) * np, cudaMemcpyDefault));
    RP_CUDA_TRY(cudaMemset(s->m, 0, sizeof(float) * np));
    RP_CUDA_TRY(cudaMemset(s->v, 0, sizeof(float) * np));
    k_to_bf16<<<(unsigned)((np + 255) / 256), 256>>>(s->p, s->pb, np);
    RP_CUDA_TRY(cudaGetLastError());
    RP_CUDA_TRY(cudaDeviceSynchronize());
    s->step = 0;
    s->version += 1;
    return RP_OK;
}

int rp_surrogate_get_params(rp_surrogate_t s, float *params)
{
    if (!s || !params) {
        set_error("rp_surrogate_get_params: null argument");
        return RP_ERR_INVALID_ARG;
    }
    RP_CUDA_TRY(cudaDeviceSynchronize());
    RP_CUDA_TRY(cudaMemcpy(params, s->p, sizeof(float) * n_params(), cudaMemcpyDefault));
    return RP_OK;
}

int rp_surrogate_forward(rp_surrogate_t s, int64_t n, const float *x, float *out, void *stream)
{
    if (!s || n < 0 || (n > 0 && (!x || !out))) {
        set_error("rp_surrogate_forward: bad arguments");
        return RP_ERR_INVALID_ARG;
    }
    if (n == 0) return RP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = forward_fused(s, n, x, out, st);
    if (rc) return rc;
    return fused_status(s, st);
}

int rp_surrogate_loss_grad(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                           const float *t, double *loss, float *grad, void *stream)
{
    if (!s || n <= 0 || !x || !y || !t) {
        set_error("rp_surrogate_loss_grad: bad arguments");
        return RP_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double L = 0.0;
    int rc = loss_grad(s, n, x, y, t, &L, st);
    if (rc) return rc;
    if (loss) *loss = L;
    if (grad) {
        RP_CUDA_TRY(cudaMemcpyAsync(grad, s->grad, sizeof(float) * n_params(), cudaMemcpyDefault,
                                    st));
        RP_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return RP_OK;
}

int rp_surrogate_train_step(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                            const float *t, float lr, double *loss, void *stream)
{
    if (!s || n <= 0 || !x || !y || !t || !(lr > 0.0f)) {
        set_error("rp_surrogate_train_step: bad arguments");
        return RP_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = loss_grad(s, n, x, y, t, loss, st);
    if (rc) return rc;
    if ((rc = adam_step(s, lr, st))) return rc;
    if (!loss) return fused_status(s, st);  // syncs st
    return RP_OK;
}

int rp_surrogate_train(rp_surrogate_t s, int64_t n, const float *x, const float *y,
                       const float *t, const rp_train_params *p, double *loss, void *stream)
{
    if (!s || !p || !x || !y || !t || p->epochs < 1 || p->batch < 1 || n < p->batch ||
        !(p->lr > 0.0f) || !(p->lr_final >= 0.0f)) {
        set_error("rp_surrogate_train: bad arguments (need epochs >= 1, 1 <= batch <= n, lr > 0)");
        return RP_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long nb = n / p->batch, B = p->batch;
    int rc = ensure_acts(s, B);
    if (rc) return rc;
    std::vector<long long> order(nb);
    for (long long b = 0; b < nb; ++b) order[b] = b;
    uint64_t rng = p->seed;
    const double total = (double)p->epochs * (double)nb;
    long long k = 0;
    for (int e = 0; e < p->epochs; ++e) {
        for (long long b = nb - 1; b > 0; --b) {  // Fisher-Yates shuffle of the batch order
            const long long j = (long long)(splitmix64(rng) % (uint64_t)(b + 1));
            std::swap(order[b], order[j]);
        }
        RP_CUDA_TRY(cudaMemsetAsync(s->loss + 1, 0, sizeof(double), st));
        for (long long b = 0; b < nb; ++b, ++k) {
            const long long r0 = order[b] * B;
            const double c = 0.5 * (1.0 + cos(3.14159265358979323846 * (double)k / total));
            const float lr = (float)(p->lr_final + (p->lr - p->lr_final) * c);
            if ((rc = loss_grad(s, B, x + 3 * r0, y + 2 * r0, t + 10 * r0, nullptr, st))) return rc;
            k_acc_loss<<<1, 1, 0, st>>>(s->loss, 1.0 / ((double)B * (double)nb));
            RP_CUDA_TRY(cudaGetLastError());
            if ((rc = adam_step(s, lr, st))) return rc;
        }
    }
    double L = 0.0;
    RP_CUDA_TRY(cudaMemcpyAsync(&L, s->loss + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    if ((rc = fused_status(s, st))) return rc;  // syncs st
    if (loss) *loss = L;
    return RP_OK;
}

int rp_surrogate_save(rp_surrogate_t s, const char *path)
{
    if (!s || !path) {
        set_error("rp_surrogate_save: null argument");
        return RP_ERR_INVALID_ARG;
    }
    const long long np = n_params();
    std::vector<float> buf((size_t)(3 * np));
    RP_CUDA_TRY(cudaDeviceSynchronize());
    RP_CUDA_TRY(cudaMemcpy(buf.data(), s->p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    RP_CUDA_TRY(cudaMemcpy(buf.data() + np, s->m, sizeof(float) * np, cudaMemcpyDeviceToHost));
    RP_CUDA_TRY(cudaMemcpy(buf.data() + 2 * np, s->v, sizeof(float) * np, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) {
        set_error("rp_surrogate_save: cannot open %s", path);
        return RP_ERR_INVALID_ARG;
    }
    const int64_t hdr[2] = {(int64_t)np, (int64_t)s->step};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int64_t), 2, f) == 2 &&
              fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("rp_surrogate_save: write to %s failed", path);
        return RP_ERR_INVALID_ARG;
    }
    return RP_OK;
}

int rp_surrogate_load(const char *path, rp_surrogate_t *out)
{
    if (!path || !out) {
        set_error("rp_surrogate_load: null argument");
        return RP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        set_error("rp_surrogate_load: cannot open %s", path);
        return RP_ERR_INVALID_ARG;
    }
    const long long np = n_params();
    char magic[8];
    int64_t hdr[2] = {0, 0};
    std::vector<float> buf((size_t)(3 * np));
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(hdr, sizeof(int64_t), 2, f) == 2 && hdr[0] == np && hdr[1] >= 0 &&
              fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) {
        set_error("rp_surrogate_load: %s is not a surrogate checkpoint of %lld parameters", path,
                  np);
        return RP_ERR_INVALID_ARG;
    }
    rp_surrogate_t s = nullptr;
    int rc = rp_surrogate_create(buf.data(), &s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(s->m, buf.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->v, buf.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rp_surrogate_destroy(s);
        return cuda_fail(e, "rp_surrogate_load");
    }
    s->step = hdr[1];
    *out = s;
    return RP_OK;
}

}  // extern "C"
