// kf_bin_static.cu -- hit binning that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns the whole
// device memory and hands it out itself, or a real-time (trigger) process
// whose memory footprint is fixed when it starts.  kf_bin_hits needs a context
// whose workspace grows with cudaMalloc; this entry point runs the same
// binning kernels with their scratch in a fixed array in device global
// memory, reserved when the library is loaded onto a device.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Only one word of it has to start at zero, the count of hits keyed
// in FP64, and the call clears it; every other scratch word the kernels read is
// written earlier in the same call (the per-bin counts live in the caller's
// offsets array, which the call clears).  Calls whose work overlaps on the GPU
// (two streams, or two threads) race on the array.
#include "kf_internal.h"

namespace {

constexpr int STATIC_MAX_HITS = KF_STATIC_MAX_HITS;
// rec[n] float4 + key[n] + cursor[KF_NBINS] int32, as launch_bin lays them out
constexpr size_t STATIC_SCRATCH_INTS = 5 * (size_t)STATIC_MAX_HITS + KF_NBINS;

static __device__ __align__(256) int32_t g_bin_scratch[STATIC_SCRATCH_INTS];

// Device address of the array on the current device.  Host code cannot use
// g_bin_scratch's name as a device address; cudaGetSymbolAddress gives it with
// the device current.  It is looked up on every call (cheap once the library's
// module is loaded on the device): a cached address would go stale after a
// cudaDeviceReset, when the module is loaded again and the array may move.
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// device memory of GPU dev, or managed memory, at a multiple of align bytes
// (another GPU's memory is refused: without peer access the kernels would fault
// on it; so is a misaligned address: the kernels access whole elements)
bool on_device(const void *p, int dev, uintptr_t align)
{
    cudaPointerAttributes at;
    if (!p || (reinterpret_cast<uintptr_t>(p) & (align - 1)) || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int kf_bin_hits_static(int32_t n_hits, const float *x, const float *y, const float *z, double half_len,
                                  int32_t *perm_out, int32_t *offsets_out, float *packed_out, void *stream)
{
    if (n_hits < 0 || !(half_len > 0)) return KF_EINVAL;
    if (n_hits > STATIC_MAX_HITS) return KF_ESIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KF_ECUDA;
    }
    if (!on_device(offsets_out, dev, 4)) return KF_EINVAL;
    if (n_hits > 0 && (!on_device(x, dev, 4) || !on_device(y, dev, 4) || !on_device(z, dev, 4) ||
                       !on_device(perm_out, dev, 4) || (packed_out && !on_device(packed_out, dev, 16))))
        return KF_EINVAL;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return KF_ECUDA;
    }
    cudaError_t e = kfd::launch_bin(n_hits, x, y, z, half_len, perm_out, offsets_out, packed_out, scratch,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KF_ECUDA;
    }
    return KF_OK;
}
