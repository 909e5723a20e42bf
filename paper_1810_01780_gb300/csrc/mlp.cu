// mlp.cu -- the surrogate network: 3 -> 256 -> 256 -> 256 -> 256 -> 12, GELU (erf form),
// BF16 weights and operands, FP32 accumulation, FP32 master weights with Adam: the operand
// images of the weights, the optimiser step, the loss-and-gradient driver, the native training
// loop and checkpoints.
//
// Inference runs in one fused kernel (mlp_fused.cu: the hidden 256 x 256 layers on the
// 5th-generation tensor cores, the thin first (3 -> 256) and last (256 -> 12) layers on the
// CUDA cores).  A training step runs every layer on the tensor cores (the thin ones with their
// narrow side zero-padded to 16): the forward and backward kernels of mlp_train_fused.cu, the
// weight gradients of mlp_train_tc.cu, then one Adam kernel here.  Arithmetic everywhere:
// BF16-rounded operands, FP32 products and sums.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rp_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int kLayers = 5;
// widths of the network's layers: 3 -> 256 -> 256 -> 256 -> 256 -> 12
__host__ __device__ constexpr int kDim(int i) { return i == 0 ? 3 : (i == kLayers ? 12 : 256); }


__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

__host__ __device__ constexpr long long layer_w(int l)
{
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)kDim(i) * kDim(i + 1) + kDim(i + 1);
    return o;
}
__host__ __device__ constexpr long long layer_b(int l)
{
    return layer_w(l) + (long long)kDim(l) * kDim(l + 1);
}

struct LayerOffs {
    long long w[kLayers], b[kLayers];  // offsets of W_l and b_l in the flat parameter vector
};

// Operands of the fused kernels (layout: kPackW, kPackF, PF_* and kPackW4F / kPackW4B in
// rp_internal.h): the hidden layers' weights W1..W3 as BF16 B operands (B[n][k] = W[k][n]) in
// the tensor cores' no-swizzle K-major shared-memory image, the two halves of n one after the
// other (bimg_off), then the FP32 block, then the last layer's two BF16 images and the first
// layer's (their padding stays zero from the pack's allocation).
using rph::kPackF;
using rph::kPackW;
__global__ void k_pack(const float *__restrict__ p, unsigned char *__restrict__ pack, const LayerOffs L)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < 3 * 65536) {
        const int l = (int)(i / 65536), e = (int)(i % 65536), k = e / 256, n = e % 256;
        const float w = p[L.w[l + 1] + (long long)k * 256 + n];
        *(__nv_bfloat16 *)(pack + l * kPackW + rph::bimg_off(k, n)) = __float2bfloat16_rn(w);
        return;
    }
    const long long j = i - 3 * 65536;
    if (j >= kPackF) {
        const long long e = j - kPackF;  // the last layer's images
        if (e >= 256 * 12) return;
        const int k = (int)(e / 12), o = (int)(e % 12);
        const __nv_bfloat16 b = __float2bfloat16_rn(p[L.w[4] + e]);
        *(__nv_bfloat16 *)(pack + rph::kPackW4F + rph::w4f_off(k, o)) = b;
        *(__nv_bfloat16 *)(pack + rph::kPackW4B + rph::w4b_off(k, o)) = b;
        return;
    }
    float v = 0.0f;
    if (j < rph::PF_B0) {
        const __nv_bfloat16 b = __float2bfloat16_rn(p[L.w[0] + (j - rph::PF_W0)]);
        v = __bfloat162float(b);
        const int e = (int)(j - rph::PF_W0);
        *(__nv_bfloat16 *)(pack + rph::kPackW0 + rph::w0_off(e >> 8, e & 255)) = b;
    }
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

// One Adam step that also leaves behind what the next training step reads: the BF16 copy of
// the weights, both operand images of the hidden layers (the inference pack of k_pack and the
// backward image of k_pack_t, same layouts) and the pack's FP32 block, the gradient zeroed for
// the next accumulation, and, for acc != 0, the epoch's loss sum loss[1] += loss[0] acc, with
// loss[0] zeroed.  The pack's padding (after b4) is never written here: zero since the pack
// was allocated.
__global__ void k_adam_pack(float *__restrict__ p, __nv_bfloat16 *__restrict__ pb,
                            float *__restrict__ gr, float *__restrict__ m, float *__restrict__ v,
                            long long n, float lr, float c1, float c2,
                            unsigned char *__restrict__ pack, unsigned char *__restrict__ pack_t,
                            double *loss, double acc)
{
    rph::tc::chain_wait_release();  // the gradient comes from the weight-gradient kernel
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i == 0) {
        if (acc != 0.0) loss[1] += loss[0] * acc;
        loss[0] = 0.0;
    }
    if (i >= n) return;
    const float g = gr[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    p[i] = pi;
    const __nv_bfloat16 b = __float2bfloat16_rn(pi);
    pb[i] = b;
    gr[i] = 0.0f;
    float *pf = reinterpret_cast<float *>(pack + 3 * kPackW);
    constexpr long long kW1 = layer_w(1), kW4 = layer_w(4), kHidden = 256LL * 256 + 256;
    if (i < kW1) {  // W0 (BF16-rounded), b0
        if (i < 3 * 256) {
            pf[rph::PF_W0 + i] = __bfloat162float(b);
            *(__nv_bfloat16 *)(pack + rph::kPackW0 + rph::w0_off((int)(i >> 8), (int)(i & 255))) = b;
        } else
            pf[rph::PF_B0 + (i - 3 * 256)] = pi;
    } else if (i < kW4) {  // W1..W3 as both images, b1..b3
        const int l = (int)((i - kW1) / kHidden), e = (int)((i - kW1) % kHidden);
        if (e < 65536) {
            const int row = e >> 8, col = e & 255;  // W[row][col]: input row, output col
            *(__nv_bfloat16 *)(pack + l * kPackW + rph::bimg_off(row, col)) = b;
            *(__nv_bfloat16 *)(pack_t + l * kPackW + rph::bimg_off(col, row)) = b;
        } else {
            pf[rph::PF_B1 + l * 256 + (e - 65536)] = pi;
        }
    } else {  // W4 (BF16-rounded), b4
        const int e = (int)(i - kW4);
        if (e < 256 * 12) {
            pf[rph::PF_W4 + e] = __bfloat162float(b);
            const int k = e / 12, o = e % 12;
            *(__nv_bfloat16 *)(pack + rph::kPackW4F + rph::w4f_off(k, o)) = b;
            *(__nv_bfloat16 *)(pack + rph::kPackW4B + rph::w4b_off(k, o)) = b;
        } else
            pf[rph::PF_B4 + (e - 256 * 12)] = pi;
    }
}


}  // namespace

namespace rph {

static void free_acts(rp_surrogate_s *s)
{
    for (int l = 0; l < 3; ++l) {
        cudaFree(s->Z[l]);
        s->Z[l] = nullptr;
    }
    for (int l = 1; l < 5; ++l) {
        cudaFree(s->H[l]);
        s->H[l] = nullptr;
    }
    for (int l = 0; l < 4; ++l) {
        cudaFree(s->gl[l]);
        s->gl[l] = nullptr;
    }
    cudaFree(s->ximg);
    cudaFree(s->g4img);
    s->ximg = s->g4img = nullptr;
    s->cap = 0;
}

int ensure_acts(rp_surrogate_s *s, long long n)
{
    if (n <= s->cap) return RP_OK;
    RP_CUDA_TRY(cudaDeviceSynchronize());
    free_acts(s);
    const long long cap = n + n / 4;
    const size_t tiles = (size_t)((cap + 127) / 128);
    for (int l = 0; l < 3; ++l) RP_CUDA_TRY(cudaMalloc(&s->Z[l], tiles * 128 * 256 * 2));
    for (int l = 1; l < 5; ++l) RP_CUDA_TRY(cudaMalloc(&s->H[l], tiles * rph::tc::kImage));
    for (int l = 0; l < 4; ++l) RP_CUDA_TRY(cudaMalloc(&s->gl[l], tiles * rph::tc::kImage));
    RP_CUDA_TRY(cudaMalloc(&s->ximg, tiles * rph::tc::kImage16));
    RP_CUDA_TRY(cudaMalloc(&s->g4img, tiles * rph::tc::kImage16));
    s->cap = cap;
    return RP_OK;
}

// Loss and parameter gradient (into s->grad) of n rows: the fused forward pass with the loss
// and the last layer's backward data pass, the hidden layers' backward data chain (these two
// also sum the bias gradients), and all five layers' weight gradients on the tensor cores (one
// launch).
static int loss_grad(rp_surrogate_s *s, long long n, const float *x, const float *y,
                     const float *t, double *loss_host, cudaStream_t st)
{
    int rc = ensure_acts(s, n);
    if (rc) return rc;
    if ((rc = ensure_pack(s, st))) return rc;
    if (!s->clean) {  // the fused Adam step leaves both zeroed
        RP_CUDA_TRY(cudaMemsetAsync(s->loss, 0, sizeof(double), st));
        RP_CUDA_TRY(cudaMemsetAsync(s->grad, 0, sizeof(float) * n_params(), st));
    }
    s->clean = false;
    float *g = s->grad;
    if ((rc = train_fwd(s, n, x, y, t, g + layer_b(3), g + layer_b(4), st))) return rc;
    if ((rc = train_bwd(s, n, g + layer_b(2), g + layer_b(1), g + layer_b(0), st))) return rc;
    WgradArgs wa;
    memset(&wa, 0, sizeof wa);
    for (int l = 1; l <= 3; ++l)  // layer l: input H_l, output gradient g_l
        wa.job[l - 1] = WgradJob{s->H[l], s->gl[l], g + layer_w(l), 256, WG_OUT_SQUARE, 0, 0};
    wa.job[3] = WgradJob{s->H[4], s->g4img, g + layer_w(4), 16, WG_OUT_LAST, 0, 0};
    wa.job[4] = WgradJob{s->gl[0], s->ximg, g + layer_w(0), 16, WG_OUT_FIRST_T, 0, 0};
    if ((rc = tc_wgrad(wa, n, s->fflag, wait_cycles(s), st))) return rc;
    RP_CUDA_TRY(cudaGetLastError());
    if (loss_host) {
        RP_CUDA_TRY(cudaMemcpyAsync(loss_host, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        if ((rc = fused_status(s, st))) return rc;  // syncs st
        *loss_host /= (double)n;
    }
    return RP_OK;
}

long long wait_cycles(const rp_surrogate_s *s) { return s->wait > 0 ? s->wait : tc::kWaitCycles; }

int ensure_pack(rp_surrogate_s *s, cudaStream_t st)
{
    if (!s->pack) {
        RP_CUDA_TRY(cudaMalloc(&s->pack, kPackBytes));
        RP_CUDA_TRY(cudaMemsetAsync(s->pack, 0, kPackBytes, st));
        s->pack_version = -1;
    }
    if (!s->pack_t) {
        RP_CUDA_TRY(cudaMalloc(&s->pack_t, 3 * kPackW));
        s->pack_version = -1;
    }
    if (s->pack_version == s->version) return RP_OK;
    const long long total = 3 * 65536 + kPackF + 256 * 12;
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

// One Adam step at learning rate lr on the gradient in s->grad.  The fused kernel brings the
// operand images (current before the step: ensure_pack) and the BF16 copy to the new weights
// and zeroes the gradient and the batch loss in the same pass; acc != 0 also adds the batch
// loss, scaled by acc, to the epoch's sum.
static int adam_step(rp_surrogate_s *s, float lr, double acc, cudaStream_t st)
{
    s->step += 1;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)s->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)s->step)));
    const long long np = n_params();
    int rc = ensure_pack(s, st);  // current after a loss_grad: then a no-op
    if (rc) return rc;
    s->version += 1;
    if ((rc = launch_chained(k_adam_pack, dim3((unsigned)((np + 255) / 256)), dim3(256), 0, st,
                             s->p, s->pb, s->grad, s->m, s->v, np, lr, c1, c2, s->pack,
                             s->pack_t, s->loss, acc)))
        return rc;
    s->pack_version = s->version;
    s->clean = true;
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

int rp_surrogate_set_wait_limit(rp_surrogate_t s, int64_t cycles)
{
    if (!s || cycles < 0) {
        set_error("rp_surrogate_set_wait_limit: null handle or negative limit");
        return RP_ERR_INVALID_ARG;
    }
    s->wait = (long long)cycles;
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
    RP_CUDA_TRY(cudaMemsetAsync(s->fflag, 0, sizeof(int), st));
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
    RP_CUDA_TRY(cudaMemsetAsync(s->fflag, 0, sizeof(int), st));
    int rc = loss_grad(s, n, x, y, t, loss, st);
    if (rc) return rc;
    if ((rc = adam_step(s, lr, 0.0, st))) return rc;
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
    RP_CUDA_TRY(cudaMemsetAsync(s->fflag, 0, sizeof(int), st));
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
            if ((rc = adam_step(s, lr, 1.0 / ((double)B * (double)nb), st))) return rc;
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
