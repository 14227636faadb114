// kf_peak.cu -- FP64 / FP32 fused multiply-add throughput of this GPU, the
// denominators of the fit kernel's roofline.
#include "kf_internal.h"

namespace kfd {

template <class T>
__global__ void __launch_bounds__(256) fma_chains_kernel(int iters, T seed, T *out)
{
    // eight independent chains per thread keep the pipe full
    T a0 = seed + threadIdx.x, a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
    T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
    const T m = T(0.999999), c = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a0 = fma(a0, m, c);
            a1 = fma(a1, m, c);
            a2 = fma(a2, m, c);
            a3 = fma(a3, m, c);
            a4 = fma(a4, m, c);
            a5 = fma(a5, m, c);
            a6 = fma(a6, m, c);
            a7 = fma(a7, m, c);
        }
    }
    const T r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (r == T(-1)) out[blockIdx.x] = r;  // keeps the chains live; never true
}

cudaError_t measure_peak(int which, int sm_count, void *scratch, double *flops_per_s)
{
    const int block = 256, grid = sm_count * 8;
    const int iters = which == 0 ? 256 : 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        if (which == 0)
            fma_chains_kernel<double><<<grid, block>>>(iters, 1.0, reinterpret_cast<double *>(scratch));
        else
            fma_chains_kernel<float><<<grid, block>>>(iters, 1.0f, reinterpret_cast<float *>(scratch));
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first run is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)grid * block * iters * 64.0;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return e;
}

}  // namespace kfd
