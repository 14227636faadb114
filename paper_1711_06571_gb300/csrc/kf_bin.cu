// kf_bin.cu -- per-layer hit binning into the (phi, z) grid used to select hit
// candidates during building (Sec. 3.1: the hit structures that candidate
// selection searches), as a stable counting sort on the GPU.  Segmented
// versions bin many (event, layer) pairs of one batch in a single pass.
//
//   1. key of every hit, in FP64 with explicit rounding (no contraction), and a
//      histogram of keys (atomics into offsets[1..]): where the single-precision
//      estimate decides the key it is taken at once, the few other hits are
//      listed and a second kernel evaluates them in FP64, so that the slow FP64
//      code runs in full warps instead of in the many warps one such hit would
//      otherwise hold up;
//   2. in-place inclusive scan of the histogram -> CSR offsets;
//   3. scatter by atomic cursors (order inside a bin is arbitrary here) of each
//      hit's record (x, y, z, original index);
//   4. each hit counts the hits of its bin with a smaller original index and
//      moves to that rank, which restores the stable order bit-exactly; its
//      record is the packed copy (x, y, z, index) in binned order, one 16-byte
//      load per candidate in the build kernel.
// Scratch (from the caller): rec[n] float4, key[n] int32, cursor[KF_NBINS]
// int32; rec doubles as the list of FP64 hits and cursor[0] as its length
// before the scan.
#include "kf_internal.h"

namespace kfd {

constexpr double PI_D = 3.14159265358979323846;

// The keys are defined in FP64 with every operation rounded:
//   u = ((atan2(y, x) + pi) * 1024) / (2 pi),   v = ((z + L) * 64) / (2 L).
// A single-precision estimate decides floor() wherever it lies farther than
// BIN_MARGIN from an integer: its error is below 3e-4 bin (atan2f within a few
// ulp of 2^-22 rad, times 1024 / 2 pi = 163, plus the roundings of the sum and
// the product), so the FP64 evaluation, which costs tens of FP64 instructions
// on a GPU whose FP64 rate is 1/64 of FP32, runs only for the ~0.2% of hits
// within BIN_MARGIN of a bin edge.  Either way the result is the FP64 one.
constexpr float BIN_MARGIN = 1e-3f;
constexpr float PI_F_BIN = 3.14159265358979323846f;
constexpr float PHI_SCALE_F = (float)(1024.0 / (2.0 * PI_D));

__device__ __forceinline__ bool bin_decided(float u)
{
    const float f = u - floorf(u);
    return f > BIN_MARGIN && f < 1.f - BIN_MARGIN;
}

// the single-precision estimates of the two bin coordinates
__device__ __forceinline__ void bin_uv32(float x, float y, float z, double half_len, float &u32, float &v32)
{
    u32 = (atan2f(y, x) + PI_F_BIN) * PHI_SCALE_F;
    const float hf = (float)half_len;
    v32 = (z + hf) * (64.f / (2.f * hf));
}

// bin_key where the single-precision estimate decides both floors (then equal
// to it); false where one of them needs the FP64 evaluation
__device__ __forceinline__ bool bin_key_f32(float x, float y, float z, double half_len, int32_t &key)
{
    float u32, v32;
    bin_uv32(x, y, z, half_len, u32, v32);
    if (!bin_decided(u32) || !bin_decided(v32)) return false;
    const int fu = min(max((int)floorf(u32), 0), KF_NPHI - 1);
    const int fv = min(max((int)floorf(v32), 0), KF_NZ - 1);
    key = fv * KF_NPHI + fu;
    return true;
}

__device__ __forceinline__ int32_t bin_key(float x, float y, float z, double half_len)
{
    float u32, v32;
    bin_uv32(x, y, z, half_len, u32, v32);
    double fu, fv;
    if (bin_decided(u32)) {
        fu = (double)floorf(u32);
    } else {
        const double u = __ddiv_rn(__dmul_rn(__dadd_rn(atan2((double)y, (double)x), PI_D), 1024.0), 2.0 * PI_D);
        fu = floor(u);
    }
    if (bin_decided(v32)) {
        fv = (double)floorf(v32);
    } else {
        const double v = __ddiv_rn(__dmul_rn(__dadd_rn((double)z, half_len), 64.0), __dmul_rn(2.0, half_len));
        fv = floor(v);
    }
    fu = fmin(fmax(fu, 0.0), (double)(KF_NPHI - 1));
    fv = fmin(fmax(fv, 0.0), (double)(KF_NZ - 1));
    return (int32_t)fv * KF_NPHI + (int32_t)fu;
}

__global__ void key_kernel(int n, const float *__restrict__ x, const float *__restrict__ y,
                           const float *__restrict__ z, double half_len, int32_t *__restrict__ key,
                           int32_t *__restrict__ counts /* offsets + 1 */, int32_t *__restrict__ undecided,
                           int32_t *__restrict__ n_undecided)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t k;
    if (bin_key_f32(x[i], y[i], z[i], half_len, k)) {
        key[i] = k;
        atomicAdd(&counts[k], 1);
    } else {
        undecided[atomicAdd(n_undecided, 1)] = i;
    }
}

// the listed hits, keyed in FP64 (grid-stride over the device-side count)
__global__ void key_fp64_kernel(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                                double half_len, int32_t *__restrict__ key, int32_t *__restrict__ counts,
                                const int32_t *__restrict__ undecided, const int32_t *__restrict__ n_undecided)
{
    const int m = *n_undecided;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int i = undecided[j];
        const int32_t k = bin_key(x[i], y[i], z[i], half_len);
        key[i] = k;
        atomicAdd(&counts[k], 1);
    }
}

// Inclusive scan of the KF_NBINS counts in place by one block of 1024 threads;
// counts[k] becomes offsets[k + 1] and cursor[k] = offsets[k].  Warp w owns the
// contiguous range [w * 2048, (w + 1) * 2048) and reads it 32 entries at a time
// (coalesced): a first pass sums it, the warp totals are scanned in shared
// memory, a second pass scans the range with shuffles and a running carry.
__device__ __forceinline__ void scan_bins_block(int32_t *__restrict__ counts, int32_t *__restrict__ cursor)
{
    __shared__ int32_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int PER_WARP = KF_NBINS / 32;
    const int base = wid * PER_WARP;
    int32_t s = 0;
    for (int j = lane; j < PER_WARP; j += 32) s += counts[base + j];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) warp_tot[wid] = s;
    __syncthreads();
    if (wid == 0) {
        int32_t w = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int32_t carry = wid > 0 ? warp_tot[wid - 1] : 0;
    for (int j = 0; j < PER_WARP; j += 32) {
        const int i = base + j + lane;
        const int32_t c = counts[i];
        int32_t v = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += o;
        }
        counts[i] = carry + v;
        cursor[i] = carry + v - c;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
}

__global__ void __launch_bounds__(1024) scan_kernel(int32_t *__restrict__ counts, int32_t *__restrict__ cursor)
{
    scan_bins_block(counts, cursor);
}

__global__ void scatter_hits_kernel(int n, const int32_t *__restrict__ key, const float *__restrict__ x,
                                    const float *__restrict__ y, const float *__restrict__ z,
                                    int32_t *__restrict__ cursor, float4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pos = atomicAdd(&cursor[key[i]], 1);
    rec[pos] = make_float4(x[i], y[i], z[i], __int_as_float(i));
}

// the original index of the record at position j
__device__ __forceinline__ int32_t rec_index(const float4 *__restrict__ rec, int j)
{
    return __float_as_int(reinterpret_cast<const float *>(rec)[4 * (size_t)j + 3]);
}

__global__ void rank_kernel(int n, const int32_t *__restrict__ key, const int32_t *__restrict__ offsets,
                            const float4 *__restrict__ rec, int32_t *__restrict__ perm, float4 *__restrict__ packed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float4 h = rec[p];
    const int32_t i = __float_as_int(h.w);
    const int32_t k = key[i];
    const int32_t b0 = offsets[k], b1 = offsets[k + 1];
    int r = 0;
    for (int j = b0; j < b1; ++j) r += rec_index(rec, j) < i;
    perm[b0 + r] = i;
    if (packed) packed[b0 + r] = h;
}

// the grid of the FP64 key pass: enough blocks for the hits, at most 1024
inline int fp64_grid(int n) { return max(1, min((n + 127) / 128, 1024)); }

// scratch layout: rec[n] float4 (16-byte aligned at the base), key[n], cursor[ncursor]
struct BinScratch {
    float4 *rec;
    int32_t *key, *cursor;
};
inline BinScratch carve_bin_scratch(void *scratch, int n)
{
    BinScratch b;
    const size_t m = n > 0 ? (size_t)n : 1;
    b.rec = reinterpret_cast<float4 *>(scratch);
    b.key = reinterpret_cast<int32_t *>(b.rec + m);
    b.cursor = b.key + m;
    return b;
}

size_t bin_scratch_bytes(int n_hits)
{
    const size_t n = n_hits > 0 ? (size_t)n_hits : 1;
    return 16 * n + 4 * n + (size_t)KF_NBINS * sizeof(int32_t) + 256;
}

cudaError_t launch_bin(int n, const float *x, const float *y, const float *z, double half_len, int32_t *perm,
                       int32_t *offsets, float *packed, void *scratch, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(offsets, 0, (KF_NBINS + 1) * sizeof(int32_t), st);
    if (e != cudaSuccess || n <= 0) return e;
    const BinScratch b = carve_bin_scratch(scratch, n);
    // the FP64 list in rec, its length in cursor[0] (both free until the scatter and the scan)
    int32_t *undecided = reinterpret_cast<int32_t *>(b.rec), *n_undecided = b.cursor;
    if ((e = cudaMemsetAsync(n_undecided, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    const int bs = 256, grid = (n + bs - 1) / bs;
    key_kernel<<<grid, bs, 0, st>>>(n, x, y, z, half_len, b.key, offsets + 1, undecided, n_undecided);
    key_fp64_kernel<<<fp64_grid(n), 128, 0, st>>>(x, y, z, half_len, b.key, offsets + 1, undecided, n_undecided);
    scan_kernel<<<1, 1024, 0, st>>>(offsets + 1, b.cursor);
    scatter_hits_kernel<<<grid, bs, 0, st>>>(n, b.key, x, y, z, b.cursor, b.rec);
    rank_kernel<<<grid, bs, 0, st>>>(n, b.key, offsets, b.rec, perm, reinterpret_cast<float4 *>(packed));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ many layers at once
// Segmented form for the serving loop: nseg layers (of several events) with
// their hits concatenated, seg_off[s] .. seg_off[s+1]-1 the hits of layer s;
// one launch per pass for all of them.  Per layer the result equals launch_bin's
// (perm and the packed indices are local to the layer).  Scratch: rec[H] float4,
// key[H], cursor[nseg][NBINS] int32.

__device__ __forceinline__ int seg_of(const int32_t *__restrict__ seg_off, int nseg, int i)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void seg_key_kernel(int H, int nseg, const int32_t *__restrict__ seg_off, const double *__restrict__ half,
                               const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                               int32_t *__restrict__ key, int32_t *__restrict__ offsets,
                               int32_t *__restrict__ undecided, int32_t *__restrict__ n_undecided)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H) return;
    const int s = seg_of(seg_off, nseg, i);
    int32_t k;
    if (bin_key_f32(x[i], y[i], z[i], half[s], k)) {
        key[i] = k;
        atomicAdd(&offsets[(size_t)s * (KF_NBINS + 1) + k + 1], 1);
    } else {
        undecided[atomicAdd(n_undecided, 1)] = i;
    }
}

__global__ void seg_key_fp64_kernel(int nseg, const int32_t *__restrict__ seg_off, const double *__restrict__ half,
                                    const float *__restrict__ x, const float *__restrict__ y,
                                    const float *__restrict__ z, int32_t *__restrict__ key,
                                    int32_t *__restrict__ offsets, const int32_t *__restrict__ undecided,
                                    const int32_t *__restrict__ n_undecided)
{
    const int m = *n_undecided;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int i = undecided[j];
        const int s = seg_of(seg_off, nseg, i);
        const int32_t k = bin_key(x[i], y[i], z[i], half[s]);
        key[i] = k;
        atomicAdd(&offsets[(size_t)s * (KF_NBINS + 1) + k + 1], 1);
    }
}

__global__ void __launch_bounds__(1024) seg_scan_kernel(int32_t *__restrict__ offsets, int32_t *__restrict__ cursor)
{
    // one block per segment: the scan of scan_kernel on that segment's counts
    scan_bins_block(offsets + (size_t)blockIdx.x * (KF_NBINS + 1) + 1, cursor + (size_t)blockIdx.x * KF_NBINS);
}

__global__ void seg_scatter_kernel(int H, int nseg, const int32_t *__restrict__ seg_off,
                                   const int32_t *__restrict__ key, const float *__restrict__ x,
                                   const float *__restrict__ y, const float *__restrict__ z,
                                   int32_t *__restrict__ cursor, float4 *__restrict__ rec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H) return;
    const int s = seg_of(seg_off, nseg, i);
    const int pos = atomicAdd(&cursor[(size_t)s * KF_NBINS + key[i]], 1);
    rec[seg_off[s] + pos] = make_float4(x[i], y[i], z[i], __int_as_float(i - seg_off[s]));
}

__global__ void seg_rank_kernel(int H, int nseg, const int32_t *__restrict__ seg_off, const int32_t *__restrict__ key,
                                const int32_t *__restrict__ offsets, const float4 *__restrict__ rec,
                                int32_t *__restrict__ perm, float4 *__restrict__ packed)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H) return;
    const int s = seg_of(seg_off, nseg, p);
    const int base = seg_off[s];
    const float4 h = rec[p];
    const int32_t i = __float_as_int(h.w);  // local index
    const int32_t k = key[base + i];
    const int32_t *off = offsets + (size_t)s * (KF_NBINS + 1);
    const int32_t b0 = off[k], b1 = off[k + 1];
    int r = 0;
    for (int j = b0; j < b1; ++j) r += rec_index(rec, base + j) < i;
    perm[base + b0 + r] = i;
    if (packed) packed[base + b0 + r] = h;
}

size_t bin_segments_scratch_bytes(int H, int nseg)
{
    const size_t n = H > 0 ? (size_t)H : 1;
    return 16 * n + 4 * n + (size_t)nseg * KF_NBINS * sizeof(int32_t) + 256;
}

cudaError_t launch_bin_segments(int nseg, int H, const int32_t *seg_off, const double *half, const float *x,
                                const float *y, const float *z, int32_t *perm, int32_t *offsets, float *packed,
                                void *scratch, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(offsets, 0, (size_t)nseg * (KF_NBINS + 1) * sizeof(int32_t), st);
    if (e != cudaSuccess || H <= 0 || nseg <= 0) return e;
    const BinScratch b = carve_bin_scratch(scratch, H);
    int32_t *undecided = reinterpret_cast<int32_t *>(b.rec), *n_undecided = b.cursor;
    if ((e = cudaMemsetAsync(n_undecided, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
    const int bs = 256, grid = (H + bs - 1) / bs;
    seg_key_kernel<<<grid, bs, 0, st>>>(H, nseg, seg_off, half, x, y, z, b.key, offsets, undecided, n_undecided);
    seg_key_fp64_kernel<<<fp64_grid(H), 128, 0, st>>>(nseg, seg_off, half, x, y, z, b.key, offsets, undecided,
                                                      n_undecided);
    seg_scan_kernel<<<nseg, 1024, 0, st>>>(offsets, b.cursor);
    seg_scatter_kernel<<<grid, bs, 0, st>>>(H, nseg, seg_off, b.key, x, y, z, b.cursor, b.rec);
    seg_rank_kernel<<<grid, bs, 0, st>>>(H, nseg, seg_off, b.key, offsets, b.rec, perm,
                                         reinterpret_cast<float4 *>(packed));
    return cudaGetLastError();
}

}  // namespace kfd
