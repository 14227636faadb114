// kf_server.cu -- serving loop: events of different sizes arrive over time;
// a dispatcher thread admits them as device memory and stream slots free up,
// merges the admitted ones into batches (continuous batching: a batch is formed
// from whatever is queued when a slot frees, while earlier batches still run)
// and runs every batch on its own stream, so batches overlap on the device
// (Sec. 4.2: several events at a time; Sec. 4.3: copies overlapped with
// processing).
//
// Per batch, on its stream: one copy of the batch's tables, a kernel that
// gathers every event's build-layer hits and seed hits from host memory, one
// segmented binning pass over every (event, layer), seeds, best-hit build of
// all events in one launch, gather of the chosen hits, final fit, and a kernel
// that writes every event's results into its caller's arrays.  The host copies
// nothing: on a GPU that reads host memory over the CPU-GPU link (a
// Grace-Blackwell board: pageable memory included, at about 200 GB/s against
// about 15 GB/s for one CPU core's memcpy) the kernels move the data; elsewhere
// the same kernels read page-locked staging.  The per-track arithmetic is that
// of the direct entry points, so a result does not depend on what it was
// batched with.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kf_internal.h"

using namespace kfd;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one page-locked host region.
class PinnedArena {
  public:
    ~PinnedArena()
    {
        if (base_) cudaFreeHost(base_);
    }
    bool init(size_t bytes)
    {
        if (cudaMallocHost(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    // returns nullptr when no block is large enough
    void *alloc(size_t bytes)
    {
        std::lock_guard<std::mutex> lk(mu_);
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_[off] = bytes;
                return static_cast<char *>(base_) + off;
            }
        }
        return nullptr;
    }
    void release(void *p)
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        const size_t off = static_cast<char *>(p) - static_cast<char *>(base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }

  private:
    std::mutex mu_;
    void *base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_, used_;
};

struct Event {
    uint64_t ticket = 0;
    int n = 0, L = 0;
    std::vector<int32_t> surface, n_hits;  // per layer
    int64_t hb = 0;                        // hits of the build layers (3..L-1)
    // where the kernels read the inputs: the caller's arrays (zero-copy) or the staging
    std::vector<const float *> x, y, z;  // per layer (layers 0..2 unused)
    const float *seed_hits = nullptr;    // [n][3][3]
    float *stage = nullptr;              // page-locked staging: x[hb] y[hb] z[hb] seed_hits[9n], or null
    kf_event_result res{};               // the caller's result arrays
    kf_event_result dres{};              // the same as the kernels address them (direct_out)
    bool direct_out = true;              // the kernels write dres directly (else via the batch's staging)
    size_t dev_bytes = 0;
    Clock::time_point t_submit;
};

struct Done {
    int rc = KF_OK;
    double latency_ms = 0;
};

// One segment of the batch's hit arrays (a build layer of one event).
struct SegIn {
    const float *x, *y, *z;
    int32_t count, dst;
};

// One event of a batch: its seed hits and where its results go.
struct EvIO {
    const float *seed_hits;  // [n][3][3]
    int32_t *hit_idx;        // [L][n]
    double *state;           // [6][n]
    double *cov;             // [21][n]
    double *chi2;
    int32_t *ndof;
    uint32_t *status;
    int32_t n, t0;
};

struct Batch {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    bool busy = false;
    std::vector<Event> events;
    void *dev = nullptr;
    char *host = nullptr;  // page-locked: tables, then staged results of events without direct output
    std::vector<size_t> staged_res;  // per event: offset of its staged results in `host` (or SIZE_MAX)
    int N = 0, L = 0;
    const char *err = nullptr;  // CUDA error text of a failed launch
};

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// One event's results staged in page-locked memory: the caller's arrays, each
// starting on a 256-byte boundary (the doubles must be 8-byte aligned whatever
// n and L are).
struct ResLayout {
    size_t idx, st, cov, chi, nd, sts, total;
};
inline ResLayout res_layout(int n, int L)
{
    ResLayout r;
    const size_t m = (size_t)n;
    r.idx = 0;
    r.st = r.idx + al(4 * (size_t)L * m);
    r.cov = r.st + al(48 * m);
    r.chi = r.cov + al(168 * m);
    r.nd = r.chi + al(8 * m);
    r.sts = r.nd + al(4 * m);
    r.total = r.sts + al(4 * m);
    return r;
}
inline size_t result_bytes(int n, int L) { return res_layout(n, L).total; }

// blockIdx.y = segment; the blocks along x stride over its hits
__global__ void gather_hits_kernel(const SegIn *__restrict__ seg, float *__restrict__ x, float *__restrict__ y,
                                   float *__restrict__ z)
{
    const SegIn g = seg[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.count; j += gridDim.x * blockDim.x) {
        x[g.dst + j] = g.x[j];
        y[g.dst + j] = g.y[j];
        z[g.dst + j] = g.z[j];
    }
}

__device__ __forceinline__ int event_of(const int32_t *__restrict__ eoff, int n_events, int t)
{
    int lo = 0, hi = n_events - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// seed hits of every track: CSR arrays (3 hits a track) for the seed estimate
// and the [9][N] planes the build and the gather read
__global__ void gather_seeds_kernel(int N, int E, const EvIO *__restrict__ ev, const int32_t *__restrict__ eoff,
                                    float *__restrict__ sx, float *__restrict__ sy, float *__restrict__ sz,
                                    int32_t *__restrict__ soff, float *__restrict__ sh9)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const EvIO e = ev[event_of(eoff, E, t)];
    const float *h = e.seed_hits + 9 * (size_t)(t - e.t0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float hx = h[3 * k + 0], hy = h[3 * k + 1], hz = h[3 * k + 2];
        sx[3 * t + k] = hx;
        sy[3 * t + k] = hy;
        sz[3 * t + k] = hz;
        sh9[(3 * k + 0) * (size_t)N + t] = hx;
        sh9[(3 * k + 1) * (size_t)N + t] = hy;
        sh9[(3 * k + 2) * (size_t)N + t] = hz;
    }
    soff[t] = 3 * t;
    if (t == N - 1) soff[N] = 3 * N;
}

// every track's results into its event's arrays ([k][n] planes of the event)
__global__ void scatter_results_kernel(int N, int E, int L, const EvIO *__restrict__ ev,
                                       const int32_t *__restrict__ eoff, const int32_t *__restrict__ idx,
                                       const double *__restrict__ st, const double *__restrict__ cov,
                                       const double *__restrict__ chi2, const int32_t *__restrict__ ndof,
                                       const uint32_t *__restrict__ fsts, const uint32_t *__restrict__ bsts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const EvIO e = ev[event_of(eoff, E, t)];
    const size_t n = (size_t)e.n, u = (size_t)(t - e.t0);
    if (e.hit_idx)
        for (int l = 0; l < L; ++l) e.hit_idx[l * n + u] = idx[(size_t)l * N + t];
    if (e.state)
#pragma unroll
        for (int i = 0; i < 6; ++i) e.state[i * n + u] = st[(size_t)i * N + t];
    if (e.cov)
#pragma unroll
        for (int i = 0; i < 21; ++i) e.cov[i * n + u] = cov[(size_t)i * N + t];
    if (e.chi2) e.chi2[u] = chi2[t];
    if (e.ndof) e.ndof[u] = ndof[t];
    if (e.status) e.status[u] = fsts[t] | bsts[t];
}

struct CopyJob {
    char *dst;
    const char *src;
    size_t bytes;
};

// Host copies shared between the calling thread and a few worker threads.
class CopyPool {
  public:
    void start(int workers)
    {
        for (int i = 0; i < workers; ++i) threads_.emplace_back([this] { work(); });
    }
    ~CopyPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    // copy every job; returns when all are done
    void run(const std::vector<CopyJob> &jobs)
    {
        if (jobs.empty()) return;
        {
            std::lock_guard<std::mutex> lk(mu_);
            jobs_ = &jobs;
            next_ = 0;
            left_ = jobs.size();
        }
        cv_.notify_all();
        drain();
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [this] { return left_ == 0; });
        jobs_ = nullptr;
    }

  private:
    void drain()
    {
        for (;;) {
            const CopyJob *j = nullptr;
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (!jobs_ || next_ >= jobs_->size()) return;
                j = &(*jobs_)[next_++];
            }
            memcpy(j->dst, j->src, j->bytes);
            std::lock_guard<std::mutex> lk(mu_);
            if (--left_ == 0) done_.notify_all();
        }
    }
    void work()
    {
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return stop_ || (jobs_ && next_ < jobs_->size()); });
                if (stop_) return;
            }
            drain();
        }
    }
    std::mutex mu_;
    std::condition_variable cv_, done_;
    std::vector<std::thread> threads_;
    const std::vector<CopyJob> *jobs_ = nullptr;
    size_t next_ = 0, left_ = 0;
    bool stop_ = false;
};

}  // namespace

struct kf_server {
    kf_ctx *ctx = nullptr;
    int device = 0;
    Geom geom{};
    bool host_access = false;  // kernels may read and write pageable host memory
    kf_server_params p{};
    cudaMemPool_t pool = nullptr;
    PinnedArena arena;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Event> queue;
    std::vector<Batch> batches;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> pending;  // ticket -> 1 while queued or in flight
    uint64_t next_ticket = 1;
    size_t in_use = 0, peak = 0;
    uint64_t submitted = 0, completed = 0, rejected = 0, n_batches = 0, batch_events = 0;
    std::vector<double> lat;
    uint64_t tracks_done = 0;
    double dev_ms_sum = 0, copy_ms_sum = 0, stage_ms_sum = 0;
    uint64_t timed_batches = 0, staged_events = 0;
    Clock::time_point t_reset;
    std::string err;
    std::atomic<bool> stop{false};
    CopyPool copies;  // declared before the dispatcher thread: destroyed after it is joined
    std::thread worker;

    size_t event_bytes(int n, int L, int64_t hb) const;
    static size_t batch_host_bytes(int n, int L);
    int launch(Batch &b);
    void copy_out(Batch &b);
    void finish(Batch &b, bool ok);
    void loop();
};

// Device address of page-locked host memory p, else null.
static const void *pinned_view(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Address under which a kernel can reach host memory p: p itself where the GPU
// reads pageable memory, the mapped address of page-locked memory, else null.
static const void *device_view(const kf_server *s, const void *p)
{
    if (!p) return nullptr;
    if (s->host_access) return p;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) return at.devicePointer;
    return nullptr;
}

// device_view of an array of floats, or null where either address is not a
// multiple of 4 bytes
static const void *float_view(const kf_server *s, const void *p)
{
    const void *v = device_view(s, p);
    return (reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(v)) & 3 ? nullptr : v;
}

size_t kf_server::event_bytes(int n, int L, int64_t hb) const
{
    const size_t nseg = (size_t)(L - 3);
    size_t b = 0;
    b += 3 * al(4 * (size_t)hb);                                // x, y, z
    b += al(4 * (size_t)hb) + al(16 * (size_t)hb);              // perm, packed
    b += al(4 * nseg * (KF_NBINS + 1));                         // offsets
    b += al(bin_segments_scratch_bytes((int)hb, (int)nseg));     // bin scratch
    b += 3 * al(12 * (size_t)n) + al(36 * (size_t)n);          // seed hits csr, [9][n]
    b += al(24 * (size_t)n) + al((size_t)n) + al(4 * (size_t)n + 4);  // seeds, q, seed offsets
    b += al(4 * (size_t)L * n) + al(4 * (size_t)n);             // idx, build status
    b += al(4 * ((size_t)order_scratch_ints() + n)) * 2;       // two order passes
    b += al(4 * (size_t)n + 4) + al((size_t)L * n) + 3 * al(4 * (size_t)L * n) + al(gather_scratch_bytes(n));
    b += al(24 * (size_t)n) + al((size_t)n);                    // final-fit seeds
    b += al(48 * (size_t)n) + al(168 * (size_t)n) + al(8 * (size_t)n) + 2 * al(4 * (size_t)n);  // outputs
    b += build_seed_scratch_bytes(n);                           // seed fits of the build
    b += fit_carry_bytes(n);                                    // final fit: phase 1 -> phase 2
    b += al(sizeof(LayerDev) * (size_t)L) + al(sizeof(SegIn) * nseg) + al(sizeof(EvIO));  // tables
    // a merged batch rounds each of its (under 48) arrays up once: an event's
    // share of that rounding is below 48 * 256 bytes, so the sum over a batch's
    // events bounds the batch's allocation
    return b + 48 * 256;
}

// Page-locked bytes of a one-event batch (tables, staged results; a bound).
size_t kf_server::batch_host_bytes(int n, int L)
{
    const size_t nseg = (size_t)(L - 3);
    return sizeof(SegIn) * nseg + 12 * nseg + sizeof(EvIO) + sizeof(LayerDev) * (size_t)L + 16 +
           result_bytes(n, L) + 16 * 256;
}

// Launch one batch on its stream (the dispatcher, without the lock).
int kf_server::launch(Batch &b)
{
    const int E = (int)b.events.size();
    const int L = b.events[0].L;
    int N = 0;
    int64_t HB = 0;
    for (auto &e : b.events) {
        N += e.n;
        HB += e.hb;
    }
    const int nseg = E * (L - 3);
    b.N = N;
    b.L = L;
    // ---- device layout: the tables first (one copy), then the work arrays
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += al(bytes);
        return r;
    };
    const size_t d_seg = take(sizeof(SegIn) * (size_t)nseg), d_segoff = take(4 * (size_t)(nseg + 1)),
                 d_half = take(8 * (size_t)nseg), d_ev = take(sizeof(EvIO) * (size_t)E),
                 d_ltab = take(sizeof(LayerDev) * (size_t)E * L), d_eoff = take(4 * (size_t)(E + 1));
    const size_t tables = o;
    const size_t d_x = take(4 * HB), d_y = take(4 * HB), d_z = take(4 * HB), d_perm = take(4 * HB),
                 d_pk = take(16 * HB), d_off = take(4 * (size_t)nseg * (KF_NBINS + 1)),
                 d_bs = take(bin_segments_scratch_bytes((int)HB, nseg)), d_sx = take(12 * (size_t)N),
                 d_sy = take(12 * (size_t)N), d_sz = take(12 * (size_t)N), d_sh9 = take(36 * (size_t)N),
                 d_soff = take(4 * (size_t)(N + 1)), d_seed = take(24 * (size_t)N), d_q = take(N),
                 d_idx = take(4 * (size_t)L * N), d_bsts = take(4 * (size_t)N),
                 d_ord1 = take(4 * (order_scratch_ints() + N)), d_goff = take(4 * (size_t)(N + 1)),
                 d_glay = take((size_t)L * N), d_gx = take(4 * (size_t)L * N), d_gy = take(4 * (size_t)L * N),
                 d_gz = take(4 * (size_t)L * N), d_gsc = take(gather_scratch_bytes(N)), d_fseed = take(24 * (size_t)N),
                 d_fq = take(N), d_ord2 = take(4 * (order_scratch_ints() + N)), d_st = take(48 * (size_t)N),
                 d_cov = take(168 * (size_t)N), d_chi = take(8 * (size_t)N), d_nd = take(4 * (size_t)N),
                 d_sts = take(4 * (size_t)N), d_bseed = take(build_seed_scratch_bytes((int)N)),
                 d_carry = take(fit_carry_bytes((int)N));
    // ---- page-locked host: the tables, then staged results of events the kernels cannot write directly
    size_t h = tables;
    b.staged_res.assign(E, SIZE_MAX);
    for (int ev = 0; ev < E; ++ev)
        if (!b.events[ev].direct_out) {
            b.staged_res[ev] = h;
            h += al(result_bytes(b.events[ev].n, L));
        }
    b.host = static_cast<char *>(arena.alloc(h));
    if (!b.host) return KF_EAGAIN;
    cudaStream_t st = b.stream;
    cudaError_t e = cudaMallocFromPoolAsync(&b.dev, o, pool, st);
    if (e != cudaSuccess) {
        arena.release(b.host);
        b.host = nullptr;
        cudaGetLastError();
        return KF_ENOMEM;
    }
    cudaEventRecord(b.start, st);
    char *D = static_cast<char *>(b.dev);
    char *Hh = b.host;
    auto dp = [&](size_t off) { return D + off; };
    SegIn *seg = reinterpret_cast<SegIn *>(Hh + d_seg);
    int32_t *segoff = reinterpret_cast<int32_t *>(Hh + d_segoff);
    double *half = reinterpret_cast<double *>(Hh + d_half);
    EvIO *eio = reinterpret_cast<EvIO *>(Hh + d_ev);
    LayerDev *ltab = reinterpret_cast<LayerDev *>(Hh + d_ltab);
    int32_t *eoff = reinterpret_cast<int32_t *>(Hh + d_eoff);
    int64_t lpos = 0;
    int sg = 0, tpos = 0, max_count = 0;
    eoff[0] = 0;
    for (int ev = 0; ev < E; ++ev) {
        const Event &x = b.events[ev];
        EvIO &io = eio[ev];
        io.seed_hits = x.seed_hits;
        io.n = x.n;
        io.t0 = tpos;
        if (x.direct_out) {
            io.hit_idx = x.dres.hit_idx;
            io.state = x.dres.state;
            io.cov = x.dres.cov;
            io.chi2 = x.dres.chi2;
            io.ndof = x.dres.ndof;
            io.status = x.dres.status;
        } else {  // the caller's layout inside the batch's page-locked block
            char *r = static_cast<char *>(const_cast<void *>(device_view(this, Hh + b.staged_res[ev])));
            if (!r) r = Hh + b.staged_res[ev];
            const ResLayout rl = res_layout(x.n, L);
            io.hit_idx = reinterpret_cast<int32_t *>(r + rl.idx);
            io.state = reinterpret_cast<double *>(r + rl.st);
            io.cov = reinterpret_cast<double *>(r + rl.cov);
            io.chi2 = reinterpret_cast<double *>(r + rl.chi);
            io.ndof = reinterpret_cast<int32_t *>(r + rl.nd);
            io.status = reinterpret_cast<uint32_t *>(r + rl.sts);
        }
        for (int l = 0; l < L; ++l) {
            LayerDev &ld = ltab[(size_t)ev * L + l];
            ld.surface = x.surface[l];
            if (l < 3) {
                ld.packed = nullptr;
                ld.offsets = nullptr;
                ld.x = ld.y = ld.z = nullptr;
                ld.n_hits = 0;
                continue;
            }
            const int m = x.n_hits[l];
            seg[sg] = SegIn{x.x[l], x.y[l], x.z[l], m, (int32_t)lpos};
            segoff[sg] = (int32_t)lpos;
            half[sg] = geom.s[x.surface[l]].halfd;
            max_count = std::max(max_count, m);
            ld.n_hits = m;
            ld.packed = reinterpret_cast<const float4 *>(dp(d_pk) + 16 * lpos);
            ld.offsets = reinterpret_cast<const int32_t *>(dp(d_off) + 4 * (size_t)sg * (KF_NBINS + 1));
            ld.x = reinterpret_cast<const float *>(dp(d_x) + 4 * lpos);
            ld.y = reinterpret_cast<const float *>(dp(d_y) + 4 * lpos);
            ld.z = reinterpret_cast<const float *>(dp(d_z) + 4 * lpos);
            lpos += m;
            ++sg;
        }
        tpos += x.n;
        eoff[ev + 1] = tpos;
    }
    segoff[nseg] = (int32_t)HB;
    e = cudaMemcpyAsync(D, Hh, tables, cudaMemcpyHostToDevice, st);
    // inputs: every event's build-layer hits and seed hits, read where they are
    if (e == cudaSuccess && HB > 0) {
        dim3 grid((unsigned)std::max(1, std::min((max_count + 1023) / 1024, 64)), (unsigned)nseg);
        gather_hits_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const SegIn *>(dp(d_seg)),
                                                 reinterpret_cast<float *>(dp(d_x)),
                                                 reinterpret_cast<float *>(dp(d_y)),
                                                 reinterpret_cast<float *>(dp(d_z)));
        e = cudaGetLastError();
    }
    const int32_t *deoff = reinterpret_cast<const int32_t *>(dp(d_eoff));
    const EvIO *dev_io = reinterpret_cast<const EvIO *>(dp(d_ev));
    float *sh9 = reinterpret_cast<float *>(dp(d_sh9));
    if (e == cudaSuccess) {
        gather_seeds_kernel<<<(N + 127) / 128, 128, 0, st>>>(
            N, E, dev_io, deoff, reinterpret_cast<float *>(dp(d_sx)), reinterpret_cast<float *>(dp(d_sy)),
            reinterpret_cast<float *>(dp(d_sz)), reinterpret_cast<int32_t *>(dp(d_soff)), sh9);
        e = cudaGetLastError();
    }
    // bin every build layer of every event
    if (e == cudaSuccess)
        e = launch_bin_segments(nseg, (int)HB, reinterpret_cast<int32_t *>(dp(d_segoff)),
                                reinterpret_cast<double *>(dp(d_half)), reinterpret_cast<float *>(dp(d_x)),
                                reinterpret_cast<float *>(dp(d_y)), reinterpret_cast<float *>(dp(d_z)),
                                reinterpret_cast<int32_t *>(dp(d_perm)), reinterpret_cast<int32_t *>(dp(d_off)),
                                reinterpret_cast<float *>(dp(d_pk)), dp(d_bs), st);
    // seeds from the three seed hits
    float *seed = reinterpret_cast<float *>(dp(d_seed));
    int8_t *q = reinterpret_cast<int8_t *>(dp(d_q));
    if (e == cudaSuccess)
        e = launch_seeds(geom, N, N, 0, reinterpret_cast<int32_t *>(dp(d_soff)), reinterpret_cast<float *>(dp(d_sx)),
                         reinterpret_cast<float *>(dp(d_sy)), reinterpret_cast<float *>(dp(d_sz)), seed, q, st);
    // best-hit build of all events
    int32_t *idx = reinterpret_cast<int32_t *>(dp(d_idx));
    int32_t *ord1 = reinterpret_cast<int32_t *>(dp(d_ord1));
    if (e == cudaSuccess)
        e = launch_order(N, nullptr, seed + 3 * (size_t)N, nullptr, nullptr, &geom, 0, ord1,
                         ord1 + order_scratch_ints(), st);
    if (e == cudaSuccess) {
        BuildArgs a;
        memset(&a, 0, sizeof a);
        a.n = N;
        a.n_events = E;
        a.n_layers = L;
        a.n64 = p.fit.n_fp64_updates;
        a.seed_df = p.fit.seed_update == KF_SEED_UD_DF;
        a.seed_cov = p.fit.seed_cov;
        a.ms_on = p.fit.ms_on;
        a.meas_model = p.fit.meas_model;
        a.max_cand = p.build.max_cand;
        a.nsigma = (float)p.build.nsigma;
        a.chi2_cut = (float)p.build.chi2_cut;
        a.layers = reinterpret_cast<const LayerDev *>(dp(d_ltab));
        a.event_off = deoff;
        a.seed_state = seed;
        a.q = q;
        a.seed_hits = sh9;
        a.hit_idx = idx;
        a.order = ord1 + order_scratch_ints();
        a.o_status = reinterpret_cast<uint32_t *>(dp(d_bsts));
        a.seed_scratch = dp(d_bseed);
        e = launch_build(geom, a, p.fit.precision == KF_PREC_FP64, p.build.warp_coop != 0, st);
    }
    // gather the chosen hits and fit them
    int32_t *goff = reinterpret_cast<int32_t *>(dp(d_goff));
    uint8_t *glay = reinterpret_cast<uint8_t *>(dp(d_glay));
    float *gx = reinterpret_cast<float *>(dp(d_gx)), *gy = reinterpret_cast<float *>(dp(d_gy)),
          *gz = reinterpret_cast<float *>(dp(d_gz));
    if (e == cudaSuccess)
        e = launch_gather(N, E, L, reinterpret_cast<const LayerDev *>(dp(d_ltab)), deoff, sh9, idx, goff, glay, gx,
                          gy, gz, dp(d_gsc), st);
    float *fseed = reinterpret_cast<float *>(dp(d_fseed));
    int8_t *fq = reinterpret_cast<int8_t *>(dp(d_fq));
    int32_t *ord2 = reinterpret_cast<int32_t *>(dp(d_ord2));
    if (e == cudaSuccess) e = launch_seeds(geom, N, N, 0, goff, gx, gy, gz, fseed, fq, st);
    if (e == cudaSuccess)
        e = launch_order(N, goff, fseed + 3 * (size_t)N, fseed + 5 * (size_t)N, glay, &geom,
                         std::max(3, p.fit.n_fp64_updates), ord2, ord2 + order_scratch_ints(), st);
    if (e == cudaSuccess) {
        FitArgs a;
        memset(&a, 0, sizeof a);
        a.n = N;
        a.t_begin = 0;
        a.count = N;
        a.n64 = p.fit.n_fp64_updates;
        a.seed_df = p.fit.seed_update == KF_SEED_UD_DF;
        a.seed_cov = p.fit.seed_cov;
        a.ms_on = p.fit.ms_on;
        a.meas_model = p.fit.meas_model;
        a.seed_state = fseed;
        a.q = fq;
        a.off = goff;
        a.layer = glay;
        a.hx = gx;
        a.hy = gy;
        a.hz = gz;
        a.o_state = reinterpret_cast<double *>(dp(d_st));
        a.o_cov = reinterpret_cast<double *>(dp(d_cov));
        a.o_chi2 = reinterpret_cast<double *>(dp(d_chi));
        a.o_ndof = reinterpret_cast<int32_t *>(dp(d_nd));
        a.o_status = reinterpret_cast<uint32_t *>(dp(d_sts));
        a.order = ord2 + order_scratch_ints();
        if (p.fit.precision != KF_PREC_FP64) fit_carve_carry(a.carry, dp(d_carry), N);
        e = launch_fit(geom, a, p.fit.precision == KF_PREC_FP64, 128, st);
    }
    // results: every event's slice into its arrays
    if (e == cudaSuccess) {
        scatter_results_kernel<<<(N + 127) / 128, 128, 0, st>>>(
            N, E, L, dev_io, deoff, idx, reinterpret_cast<const double *>(dp(d_st)),
            reinterpret_cast<const double *>(dp(d_cov)), reinterpret_cast<const double *>(dp(d_chi)),
            reinterpret_cast<const int32_t *>(dp(d_nd)), reinterpret_cast<const uint32_t *>(dp(d_sts)),
            reinterpret_cast<const uint32_t *>(dp(d_bsts)));
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(b.dev, st);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    if (e != cudaSuccess) {
        b.err = cudaGetErrorString(e);
        cudaGetLastError();
        cudaStreamSynchronize(st);  // nothing may still read b.host when it is reused
        cudaGetLastError();
        arena.release(b.host);
        b.host = nullptr;
        return KF_ECUDA;
    }
    return KF_OK;
}

// Copy the staged results of a finished batch's events into their callers'
// arrays (events whose arrays are not page-locked).  Runs without the lock:
// only the dispatcher touches a busy batch and its events.  The copies are cut
// into pieces shared with the copy threads (one core copies about 15 GB/s).
void kf_server::copy_out(Batch &b)
{
    const int L = b.L;
    std::vector<CopyJob> jobs;
    auto add = [&](void *dst, const char *src, size_t bytes) {
        constexpr size_t PIECE = (size_t)1 << 20;
        for (size_t o = 0; o < bytes; o += PIECE)
            jobs.push_back(CopyJob{static_cast<char *>(dst) + o, src + o, std::min(PIECE, bytes - o)});
    };
    for (size_t ev = 0; ev < b.events.size(); ++ev) {
        if (b.staged_res[ev] == SIZE_MAX) continue;
        const Event &x = b.events[ev];
        const kf_event_result &r = x.res;
        const size_t n = (size_t)x.n;
        const char *src = b.host + b.staged_res[ev];
        const ResLayout rl = res_layout(x.n, L);
        if (r.hit_idx) add(r.hit_idx, src + rl.idx, 4 * L * n);
        if (r.state) add(r.state, src + rl.st, 48 * n);
        if (r.cov) add(r.cov, src + rl.cov, 168 * n);
        if (r.chi2) add(r.chi2, src + rl.chi, 8 * n);
        if (r.ndof) add(r.ndof, src + rl.nd, 4 * n);
        if (r.status) add(r.status, src + rl.sts, 4 * n);
    }
    copies.run(jobs);
}

// Report the events of a finished batch and free its staging (lock held).
void kf_server::finish(Batch &b, bool ok)
{
    const auto now = Clock::now();
    for (auto &x : b.events) {
        const int n = x.n;
        Done d;
        d.rc = ok ? KF_OK : KF_ECUDA;
        d.latency_ms = std::chrono::duration<double, std::milli>(now - x.t_submit).count();
        done[x.ticket] = d;
        pending.erase(x.ticket);
        if (ok) {
            lat.push_back(d.latency_ms);
            ++completed;
            tracks_done += (uint64_t)n;
        }
        in_use -= x.dev_bytes;
        arena.release(x.stage);
        x.stage = nullptr;
    }
    arena.release(b.host);
    b.host = nullptr;
    b.events.clear();
    b.busy = false;
    cv.notify_all();
}

void kf_server::loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    bool single = false;
    while (!stop) {
        bool progress = false;
        // completions
        for (auto &b : batches) {
            if (!b.busy) continue;
            cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                err = cudaGetErrorString(q);
                cudaGetLastError();
            } else {
                float dms = 0.f;
                if (cudaEventElapsedTime(&dms, b.start, b.done) != cudaSuccess) cudaGetLastError();
                lk.unlock();
                const auto c0 = Clock::now();
                copy_out(b);
                const double cms = std::chrono::duration<double, std::milli>(Clock::now() - c0).count();
                lk.lock();
                dev_ms_sum += dms;
                copy_ms_sum += cms;
                ++timed_batches;
            }
            finish(b, q == cudaSuccess);
            progress = true;
        }
        // admission: a free slot takes the queued events that fit the memory left,
        // once the oldest has waited the batch window or a full batch is queued
        const auto now = Clock::now();
        const bool ripe =
            !queue.empty() && ((int)queue.size() >= p.max_batch_events ||
                               std::chrono::duration<double, std::milli>(now - queue.front().t_submit).count() >=
                                   p.batch_window_ms);
        for (auto &b : batches) {
            if (b.busy || queue.empty() || !ripe) continue;
            const int L = queue.front().L;
            size_t bytes = 0;
            std::vector<Event> take;
            const int cap = single ? 1 : p.max_batch_events;
            single = false;
            for (auto it = queue.begin(); it != queue.end() && (int)take.size() < cap;) {
                if (it->L != L) {
                    ++it;
                    continue;
                }
                if (in_use + bytes + it->dev_bytes > p.mem_budget_bytes) break;  // keep arrival order
                bytes += it->dev_bytes;
                take.push_back(std::move(*it));
                it = queue.erase(it);
            }
            if (take.empty()) break;
            b.events = std::move(take);
            b.busy = true;  // owned by this thread while unlocked
            lk.unlock();
            int rc = launch(b);
            lk.lock();
            if (rc != KF_OK) {
                b.busy = false;
                if (b.err) err = b.err;
                // back to the front of the queue, in order
                for (auto it = b.events.rbegin(); it != b.events.rend(); ++it) queue.push_front(std::move(*it));
                const size_t tried = b.events.size();
                b.events.clear();
                bool busy = false;
                for (auto &c : batches) busy = busy || c.busy;
                if (rc == KF_ECUDA || (!busy && tried == 1)) {
                    // a CUDA error, or one event that cannot get memory with nothing else
                    // in flight: it can never run, so it fails instead of waiting forever
                    Event &x = queue.front();
                    done[x.ticket] = Done{rc, 0.0};
                    pending.erase(x.ticket);
                    arena.release(x.stage);
                    queue.pop_front();
                    cv.notify_all();
                    progress = true;
                } else if (!busy) {
                    single = true;  // retry with the first event alone
                    progress = true;
                }
                // else: wait for a batch in flight to return its memory
                break;
            }
            in_use += bytes;
            peak = std::max(peak, in_use);
            ++n_batches;
            batch_events += b.events.size();
            progress = true;
        }
        if (!progress) cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

extern "C" {

int kf_server_create(kf_ctx *ctx, const kf_geometry *geom, const kf_server_params *params, kf_server **out)
{
    if (!ctx || !geom || !out) return KF_EINVAL;
    *out = nullptr;
    kf_server_params P;
    memset(&P, 0, sizeof P);
    if (params) P = *params;
    if (P.mem_budget_bytes == 0) P.mem_budget_bytes = (size_t)40 << 30;
    if (P.host_staging_bytes == 0) P.host_staging_bytes = (size_t)1 << 30;
    if (P.max_batches <= 0) P.max_batches = 4;
    if (P.max_batch_events <= 0) P.max_batch_events = 16;
    if (P.max_batches > 16 || P.max_batch_events > 64 || !(P.batch_window_ms >= 0 && P.batch_window_ms <= 1e5))
        return ctx_fail(ctx, KF_EINVAL, "max_batches <= 16, max_batch_events <= 64, 0 <= batch_window_ms <= 1e5");
    kf_fit_params F, Fin = P.fit;
    Fin.schedule = KF_SCHED_GRID;  // the server's fits run on the grid schedule
    int rc = ctx_fit_params(ctx, P.fit.seed_cov == 0 ? nullptr : &Fin, F);
    if (rc) return rc;
    P.fit = F;
    if (P.build.nsigma == 0) P.build = kf_build_params{3.0, 30.0, 32, 0, nullptr};
    P.build.debug_pred = nullptr;  // a diagnostic of kf_build_besthit calls, not of the server
    if (!(P.build.nsigma > 0) || !(P.build.chi2_cut > 0) || P.build.max_cand < 1 || P.build.max_cand > 64)
        return ctx_fail(ctx, KF_EINVAL, "build params: nsigma > 0, chi2_cut > 0, 1 <= max_cand <= 64");
    Geom G;
    if ((rc = ctx_geom(ctx, geom, G))) return rc;
    const int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, KF_ECUDA, "cudaSetDevice");
    }
    kf_server *s = new kf_server();
    s->ctx = ctx;
    s->p = P;
    s->device = dev;
    s->geom = G;
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        pageable = 0;
    }
    s->host_access = pageable != 0;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess || !s->arena.init(P.host_staging_bytes)) {
        cudaGetLastError();
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return ctx_fail(ctx, KF_ENOMEM, "memory pool or pinned staging arena");
    }
    uint64_t keep = P.mem_budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->batches.resize(P.max_batches);
    for (auto &b : s->batches) {
        if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&b.start) != cudaSuccess || cudaEventCreate(&b.done) != cudaSuccess) {
            cudaGetLastError();
            for (auto &c : s->batches) {
                if (c.stream) cudaStreamDestroy(c.stream);
                if (c.start) cudaEventDestroy(c.start);
                if (c.done) cudaEventDestroy(c.done);
            }
            cudaMemPoolDestroy(s->pool);
            delete s;
            return ctx_fail(ctx, KF_ECUDA, "stream or event creation");
        }
    }
    s->t_reset = Clock::now();
    s->copies.start(3);
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return KF_OK;
}

int kf_server_submit(kf_server *s, const kf_event *ev, const kf_event_result *res, uint64_t *ticket)
{
    if (!s || !ev || !ticket) return KF_EINVAL;
    const auto t_submit = Clock::now();
    const int n = ev->n_tracks, L = ev->n_layers;
    if (n <= 0 || L < 4 || L > KF_MAX_SURFACES || !ev->surface || !ev->n_hits || !ev->x || !ev->y || !ev->z ||
        !ev->seed_hits || (ev->flags & ~KF_EVENT_ZERO_COPY))
        return KF_EINVAL;
    int64_t hb = 0;
    for (int l = 0; l < L; ++l) {
        if (ev->surface[l] < 0 || ev->surface[l] >= s->geom.n || s->geom.s[ev->surface[l]].kind != 0 ||
            ev->n_hits[l] < 0)
            return KF_EINVAL;
        if (l >= 3) {
            if (ev->n_hits[l] > 0 && (!ev->x[l] || !ev->y[l] || !ev->z[l])) return KF_EINVAL;
            hb += ev->n_hits[l];
        }
    }
    if (hb > (int64_t)1 << 30) return KF_EINVAL;
    Event x;
    x.n = n;
    x.L = L;
    x.surface.assign(ev->surface, ev->surface + L);
    x.n_hits.assign(ev->n_hits, ev->n_hits + L);
    x.hb = hb;
    x.res = res ? *res : kf_event_result{};
    x.dev_bytes = s->event_bytes(n, L, hb);
    x.t_submit = t_submit;
    x.x.assign(L, nullptr);
    x.y.assign(L, nullptr);
    x.z.assign(L, nullptr);
    // results: written by the kernels into page-locked arrays; pageable arrays get
    // them from staging (a GPU write into pageable memory faults every fresh page
    // in through the host, which measured slower than a host copy), and so do
    // arrays not aligned to their element size (the kernels store whole 4- and
    // 8-byte elements, and a misaligned store faults the GPU; the host copy out
    // of staging takes any alignment)
    {
        const void *r[6] = {x.res.hit_idx, x.res.state, x.res.cov, x.res.chi2, x.res.ndof, x.res.status};
        const uintptr_t a[6] = {4, 8, 8, 8, 4, 4};
        const void *v[6];
        bool all = true;
        for (int i = 0; i < 6; ++i) {
            v[i] = pinned_view(r[i]);
            const bool al_ok = !((reinterpret_cast<uintptr_t>(r[i]) | reinterpret_cast<uintptr_t>(v[i])) & (a[i] - 1));
            all = all && (!r[i] || (v[i] && al_ok));
        }
        x.direct_out = all;
        x.dres = kf_event_result{(int32_t *)v[0], (double *)v[1], (double *)v[2], (double *)v[3], (int32_t *)v[4],
                                 (uint32_t *)v[5]};
    }
    // inputs: read in place (zero-copy) where the kernels can reach them at
    // float alignment, else staged (the host copy takes any alignment)
    bool in_place = (ev->flags & KF_EVENT_ZERO_COPY) != 0;
    if (in_place) {
        x.seed_hits = static_cast<const float *>(float_view(s, ev->seed_hits));
        in_place = x.seed_hits != nullptr;
        for (int l = 3; l < L && in_place; ++l) {
            if (ev->n_hits[l] == 0) continue;
            x.x[l] = static_cast<const float *>(float_view(s, ev->x[l]));
            x.y[l] = static_cast<const float *>(float_view(s, ev->y[l]));
            x.z[l] = static_cast<const float *>(float_view(s, ev->z[l]));
            in_place = x.x[l] && x.y[l] && x.z[l];
        }
    }
    const size_t stage_bytes = in_place ? 0 : 4 * (3 * (size_t)hb + 9 * (size_t)n);
    const size_t host_need = stage_bytes + s->batch_host_bytes(n, L);
    if (x.dev_bytes > s->p.mem_budget_bytes || host_need > s->p.host_staging_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->rejected;
        return KF_EBUSY;
    }
    if (!in_place) {
        x.stage = static_cast<float *>(s->arena.alloc(stage_bytes));
        if (!x.stage) return KF_EAGAIN;  // staging full: retry after earlier events complete
        float *base = static_cast<float *>(const_cast<void *>(device_view(s, x.stage)));
        if (!base) base = x.stage;  // the arena is page-locked: always reachable
        float *px = x.stage, *py = px + hb, *pz = py + hb;
        int64_t pos = 0;
        for (int l = 3; l < L; ++l) {
            const int m = ev->n_hits[l];
            memcpy(px + pos, ev->x[l], 4 * (size_t)m);
            memcpy(py + pos, ev->y[l], 4 * (size_t)m);
            memcpy(pz + pos, ev->z[l], 4 * (size_t)m);
            x.x[l] = base + pos;
            x.y[l] = base + hb + pos;
            x.z[l] = base + 2 * hb + pos;
            pos += m;
        }
        memcpy(x.stage + 3 * hb, ev->seed_hits, 36 * (size_t)n);
        x.seed_hits = base + 3 * hb;
    }
    const double sms = std::chrono::duration<double, std::milli>(Clock::now() - t_submit).count();
    std::lock_guard<std::mutex> lk(s->mu);
    s->stage_ms_sum += sms;
    ++s->staged_events;
    x.ticket = s->next_ticket++;
    *ticket = x.ticket;
    s->pending[x.ticket] = 1;
    ++s->submitted;
    s->queue.push_back(std::move(x));
    s->cv.notify_all();
    return KF_OK;
}

int kf_server_poll(kf_server *s, uint64_t ticket, double *latency_ms)
{
    if (!s) return KF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return s->pending.count(ticket) ? KF_EAGAIN : KF_EINVAL;
    const Done d = it->second;
    s->done.erase(it);
    if (latency_ms) *latency_ms = d.latency_ms;
    return d.rc;
}

int kf_server_wait(kf_server *s, uint64_t ticket, double timeout_ms, double *latency_ms)
{
    if (!s) return KF_EINVAL;
    const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        auto it = s->done.find(ticket);
        if (it != s->done.end()) {
            const Done d = it->second;
            s->done.erase(it);
            if (latency_ms) *latency_ms = d.latency_ms;
            return d.rc;
        }
        if (!s->pending.count(ticket)) return KF_EINVAL;
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && Clock::now() >= deadline)
            return KF_ETIMEOUT;
    }
}

int kf_server_stats_get(kf_server *s, kf_server_stats *out, int reset)
{
    if (!s || !out) return KF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->queued = (int32_t)s->queue.size();
    int evs = 0, bs = 0;
    for (auto &b : s->batches)
        if (b.busy) {
            ++bs;
            evs += (int)b.events.size();
        }
    out->in_flight_events = evs;
    out->in_flight_batches = bs;
    out->bytes_in_use = s->in_use;
    out->peak_bytes_in_use = s->peak;
    out->batches = s->n_batches;
    out->mean_batch_events = s->n_batches ? (double)s->batch_events / (double)s->n_batches : 0.0;
    std::vector<double> v = s->lat;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * (double)(v.size() - 1)));
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
    }
    const double secs = std::chrono::duration<double>(Clock::now() - s->t_reset).count();
    out->events_per_s = secs > 0 ? (double)v.size() / secs : 0.0;
    out->tracks_per_s = secs > 0 ? (double)s->tracks_done / secs : 0.0;
    out->batch_device_ms = s->timed_batches ? s->dev_ms_sum / (double)s->timed_batches : 0.0;
    out->copy_out_ms = s->timed_batches ? s->copy_ms_sum / (double)s->timed_batches : 0.0;
    out->stage_ms = s->staged_events ? s->stage_ms_sum / (double)s->staged_events : 0.0;
    if (reset) {
        s->dev_ms_sum = s->copy_ms_sum = s->stage_ms_sum = 0;
        s->timed_batches = s->staged_events = 0;
        s->lat.clear();
        s->tracks_done = 0;
        s->t_reset = Clock::now();
        s->peak = s->in_use;
        s->n_batches = 0;
        s->batch_events = 0;
    }
    if (!s->err.empty()) return KF_ECUDA;
    return KF_OK;
}

void kf_server_destroy(kf_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &b : s->batches) {
        if (b.stream) cudaStreamSynchronize(b.stream);
        if (b.host) s->arena.release(b.host);
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.start) cudaEventDestroy(b.start);
        if (b.done) cudaEventDestroy(b.done);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // extern "C"
