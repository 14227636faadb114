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
// contents.  Nothing in it has to start at zero: every scratch word the
// kernels read is written earlier in the same call (the per-bin counts live
// in the caller's offsets array, which the call clears).  Calls whose work
// overlaps on the GPU (two streams, or two threads) race on the array.
#include <mutex>

#include "kf_internal.h"

namespace {

constexpr int STATIC_MAX_HITS = KF_STATIC_MAX_HITS;
// key[n] + cursor[KF_NBINS] + tmp[n] int32, as launch_bin lays them out
constexpr size_t STATIC_SCRATCH_INTS = 2 * (size_t)STATIC_MAX_HITS + KF_NBINS;

static __device__ __align__(256) int32_t g_bin_scratch[STATIC_SCRATCH_INTS];

std::mutex g_mu;
void *g_addr[KF_MAX_DEVICES] = {nullptr};

// Device address of the array on the current device, looked up once per device
// (host code cannot use g_bin_scratch's name as a device address).
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int kf_bin_hits_static(int32_t n_hits, const float *x, const float *y, const float *z, double half_len,
                                  int32_t *perm_out, int32_t *offsets_out, float *packed_out, void *stream)
{
    if (n_hits < 0 || !(half_len > 0)) return KF_EINVAL;
    if (n_hits > STATIC_MAX_HITS) return KF_ESIZE;
    if (!on_device(offsets_out)) return KF_EINVAL;
    if (n_hits > 0 && (!on_device(x) || !on_device(y) || !on_device(z) || !on_device(perm_out) ||
                       (packed_out && !on_device(packed_out))))
        return KF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= KF_MAX_DEVICES) {
        cudaGetLastError();
        return KF_ECUDA;
    }
    void *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) {
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
