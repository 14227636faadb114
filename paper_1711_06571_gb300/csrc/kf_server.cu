// kf_server.cu -- serving loop: events of different sizes arrive over time;
// a dispatcher thread admits them as device memory and stream slots free up,
// merges the admitted ones into batches (continuous batching: a batch is formed
// from whatever is queued when a slot frees, while earlier batches still run)
// and runs every batch on its own stream, so batches overlap on the device and
// their copies overlap other batches' kernels (Sec. 4.2: several events at a
// time; Sec. 4.3: copies overlapped with processing).
//
// Per batch, on its stream: copy the events' build-layer hits and seed hits in,
// bin every (event, layer) in one segmented pass, seed, best-hit build of all
// events in one launch, gather the chosen hits, final fit, copy the results
// out, release the batch memory.  The per-track arithmetic is the same as in
// the direct entry points, so a result does not depend on what it was batched
// with.
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
    int64_t hb = 0;                       // hits of the build layers (3..L-1)
    float *stage = nullptr;               // pinned: x[hb] y[hb] z[hb] sx[3n] sy[3n] sz[3n]
    kf_event_result res{};
    size_t dev_bytes = 0;
    Clock::time_point t_submit;
};

struct Done {
    int rc = KF_OK;
    double latency_ms = 0;
};

struct Batch {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    bool busy = false;
    std::vector<Event> events;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    char *host = nullptr;  // pinned: tables in, results out
    int N = 0, L = 0;
    // offsets of the results inside `host`
    size_t o_idx = 0, o_st = 0, o_cov = 0, o_chi = 0, o_nd = 0, o_sts = 0, o_bsts = 0;
    const char *err = nullptr;  // CUDA error text of a failed launch
};

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

__global__ void seed_soa_kernel(int n, const float *__restrict__ sx, const float *__restrict__ sy,
                                const float *__restrict__ sz, float *__restrict__ sh9)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sh9[(3 * k + 0) * (size_t)n + t] = sx[3 * t + k];
        sh9[(3 * k + 1) * (size_t)n + t] = sy[3 * t + k];
        sh9[(3 * k + 2) * (size_t)n + t] = sz[3 * t + k];
    }
}

}  // namespace

struct kf_server {
    kf_ctx *ctx = nullptr;
    int device = 0;
    Geom geom{};
    std::vector<kf_surface> surfaces;
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
    std::thread worker;

    size_t event_bytes(int n, int L, int64_t hb) const;
    static size_t batch_host_bytes(int n, int L);
    int launch(Batch &b);
    void copy_out(Batch &b);
    void finish(Batch &b, bool ok);
    void loop();
};

size_t kf_server::event_bytes(int n, int L, int64_t hb) const
{
    const size_t nseg = (size_t)(L - 3);
    size_t b = 0;
    b += 3 * al(4 * (size_t)hb);                                // x, y, z
    b += al(4 * (size_t)hb) + al(16 * (size_t)hb);              // perm, packed
    b += al(4 * nseg * (KF_NBINS + 1));                         // offsets
    b += al(4 * (2 * (size_t)hb + nseg * KF_NBINS));            // bin scratch
    b += 3 * al(12 * (size_t)n) + al(36 * (size_t)n);          // seed hits csr, [9][n]
    b += al(24 * (size_t)n) + al((size_t)n) + al(4 * (size_t)n + 4);  // seeds, q, seed offsets
    b += al(4 * (size_t)L * n) + al(4 * (size_t)n);             // idx, build status
    b += al(4 * ((size_t)order_scratch_ints() + n)) * 2;       // two order passes
    b += al(4 * (size_t)n + 4) + al((size_t)L * n) + 3 * al(4 * (size_t)L * n) + al(gather_scratch_bytes(n));
    b += al(24 * (size_t)n) + al((size_t)n);                    // final-fit seeds
    b += al(48 * (size_t)n) + al(168 * (size_t)n) + al(8 * (size_t)n) + 2 * al(4 * (size_t)n);  // outputs
    b += al(sizeof(LayerDev) * (size_t)L);                      // layer table
    // a merged batch rounds each of its ~40 arrays up once: an event's share of
    // that rounding is below 40 * 256 bytes, so the sum over a batch's events
    // bounds the batch's allocation
    return b + 40 * 256;
}

// Pinned bytes of a one-event batch's tables and results (a bound: the batch
// layout below rounds each of its arrays up to 256 bytes).
size_t kf_server::batch_host_bytes(int n, int L)
{
    return (size_t)n * (4 * (size_t)L + 48 + 168 + 8 + 4 + 4 + 4 + 4) + 4 * (size_t)L * 8 +
           sizeof(LayerDev) * (size_t)L + 13 * 256 + 64;
}

// Launch one batch on its stream (called with the lock held).
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
    // ---- device layout
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += al(bytes);
        return r;
    };
    const size_t d_x = take(4 * HB), d_y = take(4 * HB), d_z = take(4 * HB), d_perm = take(4 * HB),
                 d_pk = take(16 * HB), d_off = take(4 * (size_t)nseg * (KF_NBINS + 1)),
                 d_bs = take(bin_segments_scratch_bytes((int)HB, nseg)), d_segoff = take(4 * (size_t)(nseg + 1)),
                 d_half = take(8 * (size_t)nseg), d_sx = take(12 * (size_t)N), d_sy = take(12 * (size_t)N),
                 d_sz = take(12 * (size_t)N), d_sh9 = take(36 * (size_t)N), d_soff = take(4 * (size_t)(N + 1)),
                 d_seed = take(24 * (size_t)N), d_q = take(N), d_idx = take(4 * (size_t)L * N),
                 d_bsts = take(4 * (size_t)N), d_ord1 = take(4 * (order_scratch_ints() + N)),
                 d_ltab = take(sizeof(LayerDev) * (size_t)E * L), d_eoff = take(4 * (size_t)(E + 1)),
                 d_goff = take(4 * (size_t)(N + 1)), d_glay = take((size_t)L * N), d_gx = take(4 * (size_t)L * N),
                 d_gy = take(4 * (size_t)L * N), d_gz = take(4 * (size_t)L * N), d_gsc = take(gather_scratch_bytes(N)),
                 d_fseed = take(24 * (size_t)N), d_fq = take(N), d_ord2 = take(4 * (order_scratch_ints() + N)),
                 d_st = take(48 * (size_t)N), d_cov = take(168 * (size_t)N), d_chi = take(8 * (size_t)N),
                 d_nd = take(4 * (size_t)N), d_sts = take(4 * (size_t)N);
    b.dev_bytes = o;
    // ---- pinned host: tables in, results out
    size_t h = 0;
    auto htake = [&](size_t bytes) {
        size_t r = h;
        h += al(bytes);
        return r;
    };
    const size_t h_segoff = htake(4 * (size_t)(nseg + 1)), h_half = htake(8 * (size_t)nseg),
                 h_soff = htake(4 * (size_t)(N + 1)), h_ltab = htake(sizeof(LayerDev) * (size_t)E * L),
                 h_eoff = htake(4 * (size_t)(E + 1));
    b.o_idx = htake(4 * (size_t)L * N);
    b.o_st = htake(48 * (size_t)N);
    b.o_cov = htake(168 * (size_t)N);
    b.o_chi = htake(8 * (size_t)N);
    b.o_nd = htake(4 * (size_t)N);
    b.o_sts = htake(4 * (size_t)N);
    b.o_bsts = htake(4 * (size_t)N);
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
    int32_t *segoff = reinterpret_cast<int32_t *>(Hh + h_segoff);
    double *half = reinterpret_cast<double *>(Hh + h_half);
    int32_t *soff = reinterpret_cast<int32_t *>(Hh + h_soff);
    LayerDev *ltab = reinterpret_cast<LayerDev *>(Hh + h_ltab);
    int32_t *eoff = reinterpret_cast<int32_t *>(Hh + h_eoff);
    // tables
    int64_t hpos = 0;
    int seg = 0, tpos = 0;
    eoff[0] = 0;
    for (int ev = 0; ev < E; ++ev) {
        Event &x = b.events[ev];
        // copies of this event's build-layer hits and seed hits into the batch arrays
        e = cudaMemcpyAsync(dp(d_x) + 4 * hpos, x.stage, 4 * x.hb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp(d_y) + 4 * hpos, x.stage + x.hb, 4 * x.hb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp(d_z) + 4 * hpos, x.stage + 2 * x.hb, 4 * x.hb, cudaMemcpyHostToDevice, st);
        const float *sbase = x.stage + 3 * x.hb;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp(d_sx) + 12 * (size_t)tpos, sbase, 12 * (size_t)x.n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp(d_sy) + 12 * (size_t)tpos, sbase + 3 * x.n, 12 * (size_t)x.n,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp(d_sz) + 12 * (size_t)tpos, sbase + 6 * x.n, 12 * (size_t)x.n,
                                cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) break;
        int64_t lpos = hpos;
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
            segoff[seg] = (int32_t)lpos;
            half[seg] = geom.s[x.surface[l]].halfd;
            ld.n_hits = x.n_hits[l];
            ld.packed = reinterpret_cast<const float4 *>(dp(d_pk) + 16 * lpos);
            ld.offsets = reinterpret_cast<const int32_t *>(dp(d_off) + 4 * (size_t)seg * (KF_NBINS + 1));
            ld.x = reinterpret_cast<const float *>(dp(d_x) + 4 * lpos);
            ld.y = reinterpret_cast<const float *>(dp(d_y) + 4 * lpos);
            ld.z = reinterpret_cast<const float *>(dp(d_z) + 4 * lpos);
            lpos += x.n_hits[l];
            ++seg;
        }
        hpos += x.hb;
        tpos += x.n;
        eoff[ev + 1] = tpos;
    }
    segoff[nseg] = (int32_t)HB;
    for (int t = 0; t <= N; ++t) soff[t] = 3 * t;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp(d_segoff), segoff, 4 * (size_t)(nseg + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp(d_half), half, 8 * (size_t)nseg, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp(d_soff), soff, 4 * (size_t)(N + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp(d_ltab), ltab, sizeof(LayerDev) * (size_t)E * L, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp(d_eoff), eoff, 4 * (size_t)(E + 1), cudaMemcpyHostToDevice, st);
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
    float *sh9 = reinterpret_cast<float *>(dp(d_sh9));
    if (e == cudaSuccess)
        e = launch_seeds(geom, N, N, 0, reinterpret_cast<int32_t *>(dp(d_soff)), reinterpret_cast<float *>(dp(d_sx)),
                         reinterpret_cast<float *>(dp(d_sy)), reinterpret_cast<float *>(dp(d_sz)), seed, q, st);
    if (e == cudaSuccess) {
        seed_soa_kernel<<<(N + 127) / 128, 128, 0, st>>>(N, reinterpret_cast<float *>(dp(d_sx)),
                                                         reinterpret_cast<float *>(dp(d_sy)),
                                                         reinterpret_cast<float *>(dp(d_sz)), sh9);
        e = cudaGetLastError();
    }
    // best-hit build of all events
    int32_t *idx = reinterpret_cast<int32_t *>(dp(d_idx));
    int32_t *ord1 = reinterpret_cast<int32_t *>(dp(d_ord1));
    if (e == cudaSuccess) e = launch_order(N, nullptr, seed + 3 * (size_t)N, ord1, ord1 + order_scratch_ints(), st);
    if (e == cudaSuccess) {
        BuildArgs a;
        memset(&a, 0, sizeof a);
        a.n = N;
        a.n_events = E;
        a.n_layers = L;
        a.n64 = p.fit.n_fp64_updates;
        a.seed_cov = p.fit.seed_cov;
        a.ms_on = p.fit.ms_on;
        a.max_cand = p.build.max_cand;
        a.nsigma = (float)p.build.nsigma;
        a.chi2_cut = (float)p.build.chi2_cut;
        a.layers = reinterpret_cast<const LayerDev *>(dp(d_ltab));
        a.event_off = reinterpret_cast<const int32_t *>(dp(d_eoff));
        a.seed_state = seed;
        a.q = q;
        a.seed_hits = sh9;
        a.hit_idx = idx;
        a.order = ord1 + order_scratch_ints();
        a.o_status = reinterpret_cast<uint32_t *>(dp(d_bsts));
        e = launch_build(geom, a, p.fit.precision == KF_PREC_FP64, p.build.warp_coop != 0, st);
    }
    // gather the chosen hits and fit them
    int32_t *goff = reinterpret_cast<int32_t *>(dp(d_goff));
    uint8_t *glay = reinterpret_cast<uint8_t *>(dp(d_glay));
    float *gx = reinterpret_cast<float *>(dp(d_gx)), *gy = reinterpret_cast<float *>(dp(d_gy)),
          *gz = reinterpret_cast<float *>(dp(d_gz));
    if (e == cudaSuccess)
        e = launch_gather(N, E, L, reinterpret_cast<const LayerDev *>(dp(d_ltab)),
                          reinterpret_cast<const int32_t *>(dp(d_eoff)), sh9, idx, goff, glay, gx, gy, gz, dp(d_gsc),
                          st);
    float *fseed = reinterpret_cast<float *>(dp(d_fseed));
    int8_t *fq = reinterpret_cast<int8_t *>(dp(d_fq));
    int32_t *ord2 = reinterpret_cast<int32_t *>(dp(d_ord2));
    if (e == cudaSuccess) e = launch_seeds(geom, N, N, 0, goff, gx, gy, gz, fseed, fq, st);
    if (e == cudaSuccess) e = launch_order(N, goff, fseed + 3 * (size_t)N, ord2, ord2 + order_scratch_ints(), st);
    if (e == cudaSuccess) {
        FitArgs a;
        memset(&a, 0, sizeof a);
        a.n = N;
        a.t_begin = 0;
        a.count = N;
        a.n64 = p.fit.n_fp64_updates;
        a.seed_cov = p.fit.seed_cov;
        a.ms_on = p.fit.ms_on;
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
        e = launch_fit(geom, a, p.fit.precision == KF_PREC_FP64, 128, st);
    }
    // results out
    struct {
        size_t d, h, bytes;
    } outs[] = {{d_idx, b.o_idx, 4 * (size_t)L * N}, {d_st, b.o_st, 48 * (size_t)N},
                {d_cov, b.o_cov, 168 * (size_t)N}, {d_chi, b.o_chi, 8 * (size_t)N},
                {d_nd, b.o_nd, 4 * (size_t)N},    {d_sts, b.o_sts, 4 * (size_t)N},
                {d_bsts, b.o_bsts, 4 * (size_t)N}};
    for (auto &c : outs)
        if (e == cudaSuccess) e = cudaMemcpyAsync(Hh + c.h, dp(c.d), c.bytes, cudaMemcpyDeviceToHost, st);
    cudaError_t ef = cudaFreeAsync(b.dev, st);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaEventRecord(b.done, st);
    if (e != cudaSuccess) {
        b.err = cudaGetErrorString(e);
        cudaGetLastError();
        cudaStreamSynchronize(st);  // the copies out of b.host must end before it is reused
        cudaGetLastError();
        arena.release(b.host);
        b.host = nullptr;
        return KF_ECUDA;
    }
    return KF_OK;
}

// Copy a finished batch's results into the callers' arrays.  Runs without the
// lock: only the dispatcher touches a busy batch and its events.
void kf_server::copy_out(Batch &b)
{
    const int N = b.N, L = b.L;
    int t0 = 0;
    for (auto &x : b.events) {
        const int n = x.n;
        {
            const kf_event_result &r = x.res;
            if (r.hit_idx)
                for (int l = 0; l < L; ++l)
                    memcpy(r.hit_idx + (size_t)l * n, b.host + b.o_idx + 4 * ((size_t)l * N + t0), 4 * (size_t)n);
            if (r.state)
                for (int i = 0; i < 6; ++i)
                    memcpy(r.state + (size_t)i * n, b.host + b.o_st + 8 * ((size_t)i * N + t0), 8 * (size_t)n);
            if (r.cov)
                for (int i = 0; i < 21; ++i)
                    memcpy(r.cov + (size_t)i * n, b.host + b.o_cov + 8 * ((size_t)i * N + t0), 8 * (size_t)n);
            if (r.chi2) memcpy(r.chi2, b.host + b.o_chi + 8 * (size_t)t0, 8 * (size_t)n);
            if (r.ndof) memcpy(r.ndof, b.host + b.o_nd + 4 * (size_t)t0, 4 * (size_t)n);
            if (r.status) {
                const uint32_t *fs = reinterpret_cast<const uint32_t *>(b.host + b.o_sts) + t0;
                const uint32_t *bs = reinterpret_cast<const uint32_t *>(b.host + b.o_bsts) + t0;
                for (int t = 0; t < n; ++t) r.status[t] = fs[t] | bs[t];
            }
        }
        t0 += n;
    }
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
    kf_fit_params F;
    int rc = ctx_fit_params(ctx, P.fit.seed_cov == 0 ? nullptr : &P.fit, F);
    if (rc) return rc;
    P.fit = F;
    if (P.build.nsigma == 0) P.build = kf_build_params{3.0, 30.0, 32, 0};
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
        !ev->seed_hits)
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
    const size_t stage_bytes = 4 * (3 * (size_t)hb + 9 * (size_t)n);
    if (x.dev_bytes > s->p.mem_budget_bytes ||
        stage_bytes + s->batch_host_bytes(n, L) > s->p.host_staging_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->rejected;
        return KF_EBUSY;
    }
    x.stage = static_cast<float *>(s->arena.alloc(stage_bytes));
    if (!x.stage) return KF_EAGAIN;  // host staging full: retry after results come back
    // stage the event: build-layer x, y, z, then the seed hits as three CSR arrays
    float *px = x.stage, *py = px + hb, *pz = py + hb;
    int64_t pos = 0;
    for (int l = 3; l < L; ++l) {
        const int m = ev->n_hits[l];
        memcpy(px + pos, ev->x[l], 4 * (size_t)m);
        memcpy(py + pos, ev->y[l], 4 * (size_t)m);
        memcpy(pz + pos, ev->z[l], 4 * (size_t)m);
        pos += m;
    }
    float *sx = x.stage + 3 * hb, *sy = sx + 3 * n, *sz = sy + 3 * n;
    for (int t = 0; t < n; ++t)
        for (int k = 0; k < 3; ++k) {
            sx[3 * t + k] = ev->seed_hits[9 * t + 3 * k + 0];
            sy[3 * t + k] = ev->seed_hits[9 * t + 3 * k + 1];
            sz[3 * t + k] = ev->seed_hits[9 * t + 3 * k + 2];
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
