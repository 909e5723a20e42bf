// peaks.cu -- roofline denominators of the current device, measured by microkernels
// (rp_measure_peaks): the FP32 and FP64 fused multiply-add rates of the CUDA cores and the read
// bandwidth of a buffer resident in L2.
//
// FMA kernels: every thread runs kChains independent chains a <- a * b + c (no chain waits on
// another, so the pipes stay full whatever the latency); flops = 2 x chains x steps x threads.
// L2 kernel: every thread streams 16-byte loads that bypass L1 (ld.global.cg) over a buffer far
// smaller than L2, read once beforehand, so that every load hits L2; bytes = loads x 16.
// Each rate is the best of three timed launches after one untimed launch, timed with CUDA
// events on the caller's stream.
#include <algorithm>

#include "rp_internal.h"

namespace rph {
namespace {

constexpr int kChains = 8, kUnroll = 16, kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(const T *__restrict__ in, T *out, int iters)
{
    const T b = in[0], c = in[1];
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = in[2] + (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == in[3]) out[0] = s;  // never true for the inputs used; keeps the work
}

__global__ void __launch_bounds__(kThreads) k_l2_read(const float4 *__restrict__ buf, long long n4,
                                                      int passes, float *out)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        for (long long i = i0; i < n4; i += stride) {
            const float4 v = __ldcg(&buf[i]);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.0f) out[0] = acc.x;  // the buffer holds zeros
}

template <class F>
int best_ms(cudaStream_t st, F launch, float *best)
{
    cudaEvent_t e0, e1;
    RP_CUDA_TRY(cudaEventCreate(&e0));
    RP_CUDA_TRY(cudaEventCreate(&e1));
    launch();  // untimed
    *best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "rp_measure_peaks: microkernel");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *best = std::min(*best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RP_CUDA_TRY(cudaGetLastError());
    return RP_OK;
}

}  // namespace
}  // namespace rph

using namespace rph;

extern "C" int rp_measure_peaks(rp_peaks *out, void *stream)
{
    if (!out) {
        set_error("rp_measure_peaks: null output");
        return RP_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev;
    RP_CUDA_TRY(cudaGetDevice(&dev));
    const int sms = sm_count(dev);
    const int grid = sms * 4;  // 1024 threads per SM
    const double threads = (double)grid * kThreads;
    const size_t l2_bytes = (size_t)RP_PEAKS_L2_BUFFER;
    const int f32_iters = 16384, f64_iters = 256, l2_passes = 4000;

    void *mem = nullptr;
    RP_CUDA_TRY(cudaMalloc(&mem, l2_bytes + 4096));
    struct Free {
        void *p;
        ~Free() { cudaFree(p); }
    } guard{mem};
    char *base = (char *)mem;
    float *f_in = (float *)(base + l2_bytes);       // b, c, a0, never-equal sentinel
    double *d_in = (double *)(base + l2_bytes + 64);
    float *sink = (float *)(base + l2_bytes + 1024);
    const float fh[4] = {0.5f, 0.25f, 1.0f, -12345.0f};
    const double dh[4] = {0.5, 0.25, 1.0, -12345.0};
    RP_CUDA_TRY(cudaMemsetAsync(base, 0, l2_bytes, st));
    RP_CUDA_TRY(cudaMemcpyAsync(f_in, fh, sizeof fh, cudaMemcpyHostToDevice, st));
    RP_CUDA_TRY(cudaMemcpyAsync(d_in, dh, sizeof dh, cudaMemcpyHostToDevice, st));
    RP_CUDA_TRY(cudaStreamSynchronize(st));

    float ms32 = 0.f, ms64 = 0.f, msl2 = 0.f;
    int rc = best_ms(st, [&] {
        k_fma_rate<float><<<grid, kThreads, 0, st>>>(f_in, sink, f32_iters);
    }, &ms32);
    if (!rc) rc = best_ms(st, [&] {
        k_fma_rate<double><<<grid, kThreads, 0, st>>>(d_in, (double *)sink, f64_iters);
    }, &ms64);
    const long long n4 = (long long)(l2_bytes / 16);
    if (!rc) rc = best_ms(st, [&] {
        k_l2_read<<<grid, kThreads, 0, st>>>((const float4 *)base, n4, l2_passes, sink);
    }, &msl2);
    if (rc) return rc;
    const double per_thread = 2.0 * kChains * kUnroll;
    out->fp32_tflops = per_thread * f32_iters * threads / (ms32 * 1e-3) / 1e12;
    out->fp64_tflops = per_thread * f64_iters * threads / (ms64 * 1e-3) / 1e12;
    out->l2_gbs = (double)l2_bytes * l2_passes / (msl2 * 1e-3) / 1e9;
    out->fp32_ms = ms32;
    out->fp64_ms = ms64;
    out->l2_ms = msl2;
    out->l2_buffer_bytes = (double)l2_bytes;
    return RP_OK;
}
