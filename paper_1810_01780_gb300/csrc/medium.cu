// medium.cu -- gridded refractivity: FP32 node samples of (n, grad n).
//
// The gradient is taken by central differences of the node values (one-sided on the faces),
// evaluated in FP64 and rounded to FP32, so that n and grad n at any point are trilinear
// interpolations of one float4 per node (a smooth-enough field for the adaptive stepper,
// unlike the piecewise-constant derivative of the trilinear interpolant of n alone).
#include "rp_internal.h"

namespace rph {

__global__ void k_grid_gradient(const float *__restrict__ n, float4 *__restrict__ out, int nx,
                                int ny, int nz, double spacing)
{
    const long long total = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / sz);
        const int ijk[3] = {i, j, k}, dims[3] = {nx, ny, nz};
        const long long stride[3] = {1, sy, sz};
        float g[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double d;
            if (ijk[a] == 0)
                d = ((double)n[c + stride[a]] - (double)n[c]) / spacing;
            else if (ijk[a] == dims[a] - 1)
                d = ((double)n[c] - (double)n[c - stride[a]]) / spacing;
            else
                d = ((double)n[c + stride[a]] - (double)n[c - stride[a]]) / (2.0 * spacing);
            g[a] = (float)d;
        }
        out[c] = make_float4(n[c], g[0], g[1], g[2]);
    }
}

int build_grid(rp_medium_s *m, const float *n_src, double spacing, cudaStream_t st)
{
    const size_t cells = (size_t)m->grid.nx * m->grid.ny * m->grid.nz;
    cudaPointerAttributes attr;
    memset(&attr, 0, sizeof attr);
    bool on_device = cudaPointerGetAttributes(&attr, n_src) == cudaSuccess &&
                     (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    float *tmp = nullptr;
    RP_CUDA_TRY(cudaMalloc(&m->grid_dev, cells * sizeof(float4)));
    const float *src = n_src;
    if (!on_device) {
        RP_CUDA_TRY(cudaMalloc(&tmp, cells * sizeof(float)));
        RP_CUDA_TRY(cudaMemcpyAsync(tmp, n_src, cells * sizeof(float), cudaMemcpyHostToDevice, st));
        src = tmp;
    }
    const int block = 256;
    const int grid = sm_count(m->device) * 8;
    k_grid_gradient<<<grid, block, 0, st>>>(src, m->grid_dev, m->grid.nx, m->grid.ny, m->grid.nz,
                                            spacing);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "grid gradient");
    return RP_OK;
}

}  // namespace rph
