// kf_layout.cu -- the layout study of Sec. 4.3 (the paper timed batched 6x6
// matrix products on a GPU for several memory layouts and found its Matriplex
// layout, matrices interleaved element by element, the fastest).  Here the
// product is the covariance transport of every KF step, P' = J P J^T (J a full
// 6x6, P and P' symmetric, 21 packed entries), one matrix per thread with
// every operand in registers, read and written in one of three layouts:
//   AOS    one matrix after another: element k of matrix t at t * K + k;
//   SOA    one plane per element: element k of matrix t at k * n + t (the
//          layout of this library's kernels);
//   BLOCK  Matriplex-like: blocks of 32 matrices, element-major inside a
//          block: (t / 32) * K * 32 + k * 32 + t % 32.
// The arithmetic is identical in the three; only the addresses a warp touches
// differ (AOS: 32 matrices * K * 4 bytes apart; SOA and BLOCK: consecutive).
#include "kf_internal.h"

namespace kfd {

template <int LAYOUT, int K>
__device__ __forceinline__ size_t lidx(int t, int k, int n)
{
    if (LAYOUT == KF_LAYOUT_AOS) return (size_t)t * K + k;
    if (LAYOUT == KF_LAYOUT_SOA) return (size_t)k * n + t;
    return ((size_t)(t >> 5) * K + k) * 32 + (t & 31);
}

template <int LAYOUT>
__global__ void __launch_bounds__(128) transport_layout_kernel(int n, const float *__restrict__ J,
                                                               const float *__restrict__ P, float *__restrict__ Po)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float j[36], p[21];
#pragma unroll
    for (int k = 0; k < 36; ++k) j[k] = J[lidx<LAYOUT, 36>(t, k, n)];
#pragma unroll
    for (int k = 0; k < 21; ++k) p[k] = P[lidx<LAYOUT, 21>(t, k, n)];
    // M = J P (P symmetric, packed lower triangle), then P' = M J^T (lower triangle)
    float m[36];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) s = fmaf(j[a * 6 + c], p[c >= b ? c * (c + 1) / 2 + b : b * (b + 1) / 2 + c], s);
            m[a * 6 + b] = s;
        }
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) s = fmaf(m[a * 6 + c], j[b * 6 + c], s);
            Po[lidx<LAYOUT, 21>(t, a * (a + 1) / 2 + b, n)] = s;
        }
}

cudaError_t launch_transport_layout(int layout, int n, const float *J, const float *P, float *Po, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (n + 127) / 128;
    switch (layout) {
    case KF_LAYOUT_AOS: transport_layout_kernel<KF_LAYOUT_AOS><<<grid, 128, 0, st>>>(n, J, P, Po); break;
    case KF_LAYOUT_SOA: transport_layout_kernel<KF_LAYOUT_SOA><<<grid, 128, 0, st>>>(n, J, P, Po); break;
    case KF_LAYOUT_BLOCK: transport_layout_kernel<KF_LAYOUT_BLOCK><<<grid, 128, 0, st>>>(n, J, P, Po); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace kfd
