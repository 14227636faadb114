// kf_api.cu -- the extern "C" entry points of libkf.so (declared in include/kf.h):
// argument checking, geometry upload by value, per-stream workspaces, the
// graph-captured persistent fit and its autotuner.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "kf_internal.h"

using namespace kfd;

namespace {

struct Buf {
    void *p = nullptr;
    size_t n = 0;
};

struct Tuned {
    int block = 128, grid = 0, chunk = 1;  // chunk: tracks per thread per queue grab
    float ms = 0.f;
};

struct GraphKey {
    std::vector<uint8_t> bytes;
    bool operator==(const GraphKey &o) const { return bytes == o.bytes; }
};

}  // namespace

struct kf_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    size_t used = 0;
    std::string err;
    std::mutex mu;
    std::map<cudaStream_t, Buf> ws;  // one workspace per stream: calls on one stream are ordered
    cudaStream_t cap_stream = nullptr;
    // autotune results: key = (fp64, n bucket)
    std::map<std::pair<int, int>, Tuned> tuned;
    // one cached graph of the persistent fit
    GraphKey gkey;
    cudaGraphExec_t gexec = nullptr;
    // end-to-end host path: device buffers and the streams of kf_fit_host's
    // copy/compute pipeline, used by one kf_fit_host call at a time (host_mu)
    Buf host_ws;
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
    std::mutex host_mu;
    // kf_fit_timing: a ring of event triples around the phase kernels of the
    // grid-schedule kf_fit calls since timing was enabled
    static constexpr int TRING = 1024;
    std::vector<std::array<cudaEvent_t, 3>> tev;
    int tcalls = 0;  // timed calls since enabled
    bool timing = false;
};

namespace {

int fail(kf_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(kf_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, KF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// device memory of GPU dev (where the context's kernels run) or managed memory,
// at an address that is a multiple of align; another GPU's memory is refused
// (without peer access the kernels would fault on it), and so is a misaligned
// address: the kernels load and store whole elements (16-byte float4 for packed
// hits), and a misaligned element access faults the GPU
bool is_device_ptr_on(const void *p, int dev, size_t align = 1)
{
    if (!p || (reinterpret_cast<uintptr_t>(p) & (align - 1))) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

// alignment of the element type a pointer points to (1 for void)
template <class T>
constexpr size_t elem_align(const T *)
{
    if constexpr (std::is_void_v<T>)
        return 1;
    else
        return alignof(T);
}

#define NEED_DEV_AL(ptr, name, al)                                                                  \
    do {                                                                                            \
        if (!is_device_ptr_on(ptr, ctx->device, al))                                                \
            return fail(ctx, KF_EINVAL, "%s must be device memory aligned to %zu bytes", name, (size_t)(al)); \
    } while (0)
#define OPT_DEV_AL(ptr, name, al)                                                                   \
    do {                                                                                            \
        if ((ptr) && !is_device_ptr_on(ptr, ctx->device, al))                                       \
            return fail(ctx, KF_EINVAL, "%s must be device memory aligned to %zu bytes", name, (size_t)(al)); \
    } while (0)
#define NEED_DEV(ptr, name) NEED_DEV_AL(ptr, name, elem_align(ptr))
#define OPT_DEV(ptr, name) OPT_DEV_AL(ptr, name, elem_align(ptr))

int to_geom(kf_ctx *ctx, const kf_geometry *g, Geom &G)
{
    if (!g || !g->surfaces || g->n_surfaces <= 0 || g->n_surfaces > KF_MAX_SURFACES)
        return fail(ctx, KF_EINVAL, "geometry: need 1..%d surfaces", KF_MAX_SURFACES);
    memset(&G, 0, sizeof G);
    G.n = g->n_surfaces;
    G.kbd = KAPPA * g->bz;
    G.kb = (float)G.kbd;
    G.mass2d = g->mass * g->mass;
    G.mass2 = (float)G.mass2d;
    for (int i = 0; i < G.n; ++i) {
        const kf_surface &s = g->surfaces[i];
        if (s.kind != 0 && s.kind != 1) return fail(ctx, KF_EINVAL, "surface %d: kind must be 0 or 1", i);
        if (!(s.sig_n > 0) || !(s.sig_rphi > 0) || !(s.sig_3 > 0) || !(s.x_x0 >= 0))
            return fail(ctx, KF_EINVAL, "surface %d: resolutions must be > 0 and x/X0 >= 0", i);
        if (s.kind == 0 && !(s.pos > 0 && s.half_or_rin > 0))
            return fail(ctx, KF_EINVAL, "surface %d: barrel needs R > 0 and half length > 0", i);
        if (!(s.dr >= 0) || (s.kind == 0 && !(s.dr < s.pos)))
            return fail(ctx, KF_EINVAL, "surface %d: dr must be >= 0 and below the radius", i);
        Surf &d = G.s[i];
        d.kind = s.kind;
        d.posd = s.pos;
        d.pos = (float)s.pos;
        d.pos2 = (float)(s.pos * s.pos);
        d.pos2lo = (float)(s.pos * s.pos - (double)d.pos2);
        d.halfd = s.half_or_rin;
        d.half = (float)s.half_or_rin;
        d.rout = (float)s.r_out;
        d.x_x0d = s.x_x0;
        d.x_x0 = (float)s.x_x0;
        double rad = s.kind == 0 ? s.sig_n : s.sig_3;
        double zz = s.kind == 0 ? s.sig_3 : s.sig_n;
        d.var_radd = rad * rad;
        d.var_rphid = s.sig_rphi * s.sig_rphi;
        d.var_zzd = zz * zz;
        d.var_rad = (float)d.var_radd;
        d.var_rphi = (float)d.var_rphid;
        d.var_zz = (float)d.var_zzd;
        d.dr = s.kind == 0 ? (float)s.dr : 0.f;
    }
    return KF_OK;
}

// scratch of at least `bytes` for work on stream `st` (grows; never shrinks)
int ws_get(kf_ctx *ctx, cudaStream_t st, size_t bytes, void **out)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    Buf &b = ctx->ws[st];
    if (b.n < bytes) {
        size_t want = bytes + bytes / 4;
        if (ctx->budget && ctx->used - b.n + want > ctx->budget)
            return fail(ctx, KF_ENOMEM, "workspace of %zu bytes exceeds the budget", want);
        if (b.p) {
            cudaStreamSynchronize(st);
            cudaFree(b.p);
            ctx->used -= b.n;
            b = Buf{};
            // graphs captured against the old workspace are stale
            if (ctx->gexec) {
                cudaGraphExecDestroy(ctx->gexec);
                ctx->gexec = nullptr;
                ctx->gkey.bytes.clear();
            }
        }
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, KF_ENOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
        }
        b.n = want;
        ctx->used += want;
    }
    *out = b.p;
    return KF_OK;
}

int check_fit_params(kf_ctx *ctx, const kf_fit_params *p, kf_fit_params &q)
{
    q.precision = KF_PREC_MIXED;
    q.n_fp64_updates = 3;
    q.seed_cov = 1e4;
    q.ms_on = 1;
    q.schedule = KF_SCHED_GRID;
    q.meas_model = KF_MEAS_LAYER;
    q.seed_update = KF_SEED_UD_DF;
    if (!p) return KF_OK;
    q = *p;
    if (q.precision != KF_PREC_MIXED && q.precision != KF_PREC_FP64)
        return fail(ctx, KF_EINVAL, "precision must be KF_PREC_MIXED or KF_PREC_FP64");
    if (q.n_fp64_updates < 0 || q.n_fp64_updates > 32) return fail(ctx, KF_EINVAL, "n_fp64_updates must be 0..32");
    if (!(q.seed_cov > 0)) return fail(ctx, KF_EINVAL, "seed_cov must be > 0");
    if (q.schedule != KF_SCHED_GRID && q.schedule != KF_SCHED_PERSISTENT)
        return fail(ctx, KF_EINVAL, "schedule must be KF_SCHED_GRID or KF_SCHED_PERSISTENT");
    if (q.meas_model != KF_MEAS_LAYER && q.meas_model != KF_MEAS_HIT_2D)
        return fail(ctx, KF_EINVAL, "meas_model must be KF_MEAS_LAYER or KF_MEAS_HIT_2D");
    if (q.seed_update != KF_SEED_UD_DF && q.seed_update != KF_SEED_JOSEPH_FP64)
        return fail(ctx, KF_EINVAL, "seed_update must be KF_SEED_UD_DF or KF_SEED_JOSEPH_FP64");
    if (q.meas_model == KF_MEAS_HIT_2D && q.schedule != KF_SCHED_GRID)
        return fail(ctx, KF_EINVAL, "meas_model KF_MEAS_HIT_2D runs on the grid schedule");
    return KF_OK;
}

int set_dev(kf_ctx *ctx)
{
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return KF_OK;
}

int n_bucket(int n)
{
    int b = 0;
    while ((1 << b) < n && b < 30) ++b;
    return b;
}

template <class T>
void key_put(std::vector<uint8_t> &k, const T &v)
{
    const uint8_t *p = reinterpret_cast<const uint8_t *>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

}  // namespace

extern "C" {

const char *kf_version(void) { return "libkf 0.1 (sm_103a)"; }

int kf_ctx_create(kf_ctx **out, int cuda_device, size_t budget)
{
    if (!out) return KF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
        cudaGetLastError();
        return KF_EINVAL;
    }
    kf_ctx *c = new kf_ctx();
    c->device = cuda_device;
    c->budget = budget;
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return KF_ECUDA;
    }
    *out = c;
    return KF_OK;
}

void kf_ctx_destroy(kf_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (auto &kv : c->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->host_ws.p) cudaFree(c->host_ws.p);
    for (int i = 0; i < 3; ++i)
        if (c->hs[i]) cudaStreamDestroy(c->hs[i]);
    for (auto &t : c->tev)
        for (cudaEvent_t ev : t)
            if (ev) cudaEventDestroy(ev);
    delete c;
}

int kf_fit_timing(kf_ctx *ctx, int enable)
{
    if (!ctx) return KF_EINVAL;
    int rc = set_dev(ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (enable && ctx->tev.empty()) {
        ctx->tev.resize(kf_ctx::TRING, std::array<cudaEvent_t, 3>{nullptr, nullptr, nullptr});
        for (auto &t : ctx->tev)
            for (cudaEvent_t &ev : t)
                if (cudaEventCreate(&ev) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, KF_ECUDA, "cudaEventCreate");
                }
    }
    ctx->timing = enable != 0;
    ctx->tcalls = 0;
    return KF_OK;
}

int kf_fit_phase_times(kf_ctx *ctx, int32_t *n_calls, double *ms_phase1, double *ms_phase2)
{
    if (!ctx || !n_calls || !ms_phase1 || !ms_phase2) return KF_EINVAL;
    int rc = set_dev(ctx);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const int m = std::min(ctx->tcalls, kf_ctx::TRING);
    if (m == 0) return fail(ctx, KF_EINVAL, "no timed kf_fit since kf_fit_timing(ctx, 1)");
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < m; ++i) {
        const auto &t = ctx->tev[(ctx->tcalls - 1 - i) % kf_ctx::TRING];
        float a = 0.f, b = 0.f;
        cudaError_t e = cudaEventSynchronize(t[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, t[0], t[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, t[1], t[2]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kf_fit_phase_times");
        s1 += a;
        s2 += b;
    }
    *n_calls = m;
    *ms_phase1 = s1 / m;
    *ms_phase2 = s2 / m;
    return KF_OK;
}

const char *kf_ctx_last_error(const kf_ctx *c) { return c ? c->err.c_str() : "null context"; }

int kf_make_seeds(kf_ctx *ctx, const kf_geometry *geom, int32_t n, const kf_track_hits *hits, float *state_out,
                  int8_t *q_out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (n < 0 || !hits) return fail(ctx, KF_EINVAL, "n must be >= 0 and hits given");
    Geom G;
    int rc = to_geom(ctx, geom, G);
    if (rc) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if (n == 0) return KF_OK;
    NEED_DEV(hits->offsets, "hits.offsets");
    NEED_DEV(hits->x, "hits.x");
    NEED_DEV(hits->y, "hits.y");
    NEED_DEV(hits->z, "hits.z");
    NEED_DEV(state_out, "state_out");
    NEED_DEV(q_out, "q_out");
    cudaError_t e = launch_seeds(G, n, n, 0, hits->offsets, hits->x, hits->y, hits->z, state_out, q_out,
                                 (cudaStream_t)stream);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "seed kernel");
}

static int fit_impl(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                    const kf_seeds *seeds, const kf_track_hits *hits, const kf_tracks_out *out, void *stream,
                    const Tuned *force, const double *p0 = nullptr, double p0_scale = 1.0)
{
    if (!ctx) return KF_EINVAL;
    if (n < 0 || !seeds || !hits || !out) return fail(ctx, KF_EINVAL, "n >= 0, seeds, hits and out are required");
    kf_fit_params P;
    int rc = check_fit_params(ctx, params, P);
    if (rc) return rc;
    Geom G;
    if ((rc = to_geom(ctx, geom, G))) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if (n == 0) return KF_OK;
    NEED_DEV(seeds->state, "seeds.state");
    NEED_DEV(seeds->q, "seeds.q");
    NEED_DEV(hits->offsets, "hits.offsets");
    NEED_DEV(hits->layer, "hits.layer");
    NEED_DEV(hits->x, "hits.x");
    NEED_DEV(hits->y, "hits.y");
    NEED_DEV(hits->z, "hits.z");
    OPT_DEV(out->state, "out.state");
    OPT_DEV(out->cov, "out.cov");
    OPT_DEV(out->cov_f32, "out.cov_f32");
    OPT_DEV(out->chi2, "out.chi2");
    OPT_DEV(out->ndof, "out.ndof");
    OPT_DEV(out->status, "out.status");
    cudaStream_t st = (cudaStream_t)stream;
    FitArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.t_begin = 0;
    a.count = n;
    a.n64 = P.n_fp64_updates;
    a.seed_df = P.seed_update == KF_SEED_UD_DF;
    a.seed_cov = P.seed_cov;
    a.ms_on = P.ms_on;
    a.meas_model = P.meas_model;
    a.seed_state = seeds->state;
    a.q = seeds->q;
    a.off = hits->offsets;
    a.layer = hits->layer;
    a.hx = hits->x;
    a.hy = hits->y;
    a.hz = hits->z;
    a.o_state = out->state;
    a.o_cov = out->cov;
    a.o_cov32 = out->cov_f32;
    a.o_chi2 = out->chi2;
    a.o_ndof = out->ndof;
    a.o_status = out->status;
    a.p0 = p0;
    a.p0_scale = p0_scale;
    const bool fp64 = P.precision == KF_PREC_FP64;
    // processing order (both schedules): tracks bucketed by hit count, seed phase and seed 1/pT
    const size_t nhist = order_scratch_ints();
    const size_t order_bytes = (((nhist + 64) * sizeof(int32_t) + (size_t)n * sizeof(int32_t)) + 255) & ~(size_t)255;
    const size_t need = order_bytes + (fp64 ? 0 : fit_carry_bytes(n)) + 256;
    void *wsp = nullptr;
    if ((rc = ws_get(ctx, st, need, &wsp))) return rc;
    int32_t *hist = reinterpret_cast<int32_t *>(wsp);
    int32_t *queue = hist + nhist;
    int32_t *order = queue + 64;
    a.order = order;
    const int nseed = std::max(3, P.n_fp64_updates);  // hits whose surfaces set the order's disk bit
    // the mixed fit hands each track from its phase-1 kernel to its phase-2 kernel here
    if (!fp64 && !p0) fit_carve_carry(a.carry, static_cast<char *>(wsp) + order_bytes, n);
    if (P.schedule == KF_SCHED_GRID && !force) {
        if (ctx->timing) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            a.timing_events = ctx->tev[ctx->tcalls % kf_ctx::TRING].data();
            ++ctx->tcalls;
        }
        cudaError_t e = launch_order(n, hits->offsets, seeds->state + 3 * (size_t)n, seeds->state + 5 * (size_t)n,
                                     hits->layer, &G, nseed, hist, order, st);
        if (e == cudaSuccess) e = launch_fit(G, a, fp64, 128, st);
        return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "fit kernel");
    }
    // persistent: order by hit count + work queue, captured once as a CUDA graph
    Tuned tu;
    if (force) {
        tu = *force;
    } else {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->tuned.find({fp64 ? 1 : 0, n_bucket(n)});
        if (it != ctx->tuned.end()) tu = it->second;
    }
    if (tu.grid <= 0) tu.grid = ctx->sm_count * std::max(1, persistent_blocks_per_sm(fp64, tu.block));
    a.queue = queue;
    a.chunk = tu.chunk;
    if (force) {
        cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
        if (e == cudaSuccess)
            e = launch_order(n, hits->offsets, seeds->state + 3 * (size_t)n, seeds->state + 5 * (size_t)n,
                             hits->layer, &G, nseed, hist, order, st);
        if (e == cudaSuccess) e = launch_fit_persistent(G, a, fp64, tu.block, tu.grid, st);
        return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "persistent fit");
    }
    GraphKey key;
    key_put(key.bytes, a);
    key_put(key.bytes, fp64);
    key_put(key.bytes, tu);
    key_put(key.bytes, G);
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->gexec || !(key == ctx->gkey)) {
        if (ctx->gexec) {
            cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = ctx->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
        cudaError_t e1 = cudaMemsetAsync(queue, 0, sizeof(int32_t), cs);
        if (e1 == cudaSuccess)
            e1 = launch_order(n, hits->offsets, seeds->state + 3 * (size_t)n, seeds->state + 5 * (size_t)n,
                              hits->layer, &G, nseed, hist, order, cs);
        if (e1 == cudaSuccess) e1 = launch_fit_persistent(G, a, fp64, tu.block, tu.grid, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e1 != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ctx, e1 != cudaSuccess ? e1 : e, "capturing the persistent fit");
        }
        e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->gexec = nullptr;
            return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
        ctx->gkey = key;
    }
    cudaError_t e = cudaGraphLaunch(ctx->gexec, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "cudaGraphLaunch");
}

int kf_fit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n, const kf_seeds *seeds,
           const kf_track_hits *hits, const kf_tracks_out *out, void *stream)
{
    return fit_impl(ctx, geom, params, n, seeds, hits, out, stream, nullptr);
}

int kf_refit_inward(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                    const kf_track_hits *hits, const double *fwd_state, const double *fwd_cov, const int8_t *q,
                    const int32_t *fwd_ndof, double cov_scale, const kf_tracks_out *out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (n < 0 || !hits || !out) return fail(ctx, KF_EINVAL, "n >= 0, hits and out are required");
    kf_fit_params P;
    int rc = check_fit_params(ctx, params, P);
    if (rc) return rc;
    P.schedule = KF_SCHED_GRID;  // the refit's fit runs on the grid schedule
    Geom G;
    if ((rc = to_geom(ctx, geom, G))) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if (n == 0) return KF_OK;
    NEED_DEV(hits->offsets, "hits.offsets");
    NEED_DEV(hits->layer, "hits.layer");
    NEED_DEV(hits->x, "hits.x");
    NEED_DEV(hits->y, "hits.y");
    NEED_DEV(hits->z, "hits.z");
    NEED_DEV(fwd_state, "fwd_state");
    NEED_DEV(q, "q");
    NEED_DEV(fwd_ndof, "fwd_ndof");
    NEED_DEV(fwd_cov, "fwd_cov");
    if (!(cov_scale > 0)) return fail(ctx, KF_EINVAL, "cov_scale must be > 0");
    OPT_DEV(out->state, "out.state");
    OPT_DEV(out->cov, "out.cov");
    OPT_DEV(out->cov_f32, "out.cov_f32");
    OPT_DEV(out->chi2, "out.chi2");
    OPT_DEV(out->ndof, "out.ndof");
    OPT_DEV(out->status, "out.status");
    int32_t nh = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&nh, hits->offsets + n, sizeof nh, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading offsets[n]");
    if (nh < 0) return fail(ctx, KF_EINVAL, "offsets[n] < 0");
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_l = 0, o_x = o_l + al((size_t)nh), o_y = o_x + al(4 * (size_t)nh), o_z = o_y + al(4 * (size_t)nh),
                 o_s = o_z + al(4 * (size_t)nh), o_q = o_s + al(24 * (size_t)n), o_c = o_q + al((size_t)n),
                 o_r = o_c + al(4 * (size_t)n), o_b = o_r + al(4 * ((size_t)n + 1)),
                 o_v = o_b + al(4 * ((size_t)n / 1024 + 2)), total = o_v + al(168 * (size_t)n);
    // the reversed copies sit in a scratch buffer of their own: kf_fit takes the
    // stream's workspace for its order pass
    void *buf = nullptr;
    if (cudaMallocAsync(&buf, total, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KF_ENOMEM, "refit scratch of %zu bytes", total);
    }
    char *b = static_cast<char *>(buf);
    uint8_t *rl = reinterpret_cast<uint8_t *>(b + o_l);
    float *rx = reinterpret_cast<float *>(b + o_x), *ry = reinterpret_cast<float *>(b + o_y),
          *rz = reinterpret_cast<float *>(b + o_z), *seed = reinterpret_cast<float *>(b + o_s);
    int8_t *rq = reinterpret_cast<int8_t *>(b + o_q);
    int32_t *cnt = reinterpret_cast<int32_t *>(b + o_c), *roff = reinterpret_cast<int32_t *>(b + o_r),
            *bsum = reinterpret_cast<int32_t *>(b + o_b);
    double *rcov = reinterpret_cast<double *>(b + o_v);
    e = launch_used_counts(n, hits->offsets, fwd_ndof, cnt, st);
    if (e == cudaSuccess) e = launch_scan_counts(n, cnt, roff, bsum, st);
    if (e == cudaSuccess)
        e = launch_reverse(n, hits->offsets, roff, hits->layer, hits->x, hits->y, hits->z, fwd_state, fwd_cov, q, rl,
                           rx, ry, rz, seed, rcov, rq, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return cuda_fail(ctx, e, "reversing the tracks");
    }
    const kf_seeds S{seed, rq};
    const kf_track_hits H{roff, rl, rx, ry, rz};
    rc = fit_impl(ctx, geom, &P, n, &S, &H, out, stream, nullptr, rcov, cov_scale);
    if (rc == KF_OK) {
        e = launch_unreverse(n, out->state, out->cov, out->cov_f32, st);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "turning the results back");
    }
    cudaFreeAsync(buf, st);
    return rc;
}

static bool is_host_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown to CUDA: pageable host memory
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

int kf_fit_host(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                const kf_track_hits *hits, const kf_tracks_out *out, int32_t n_chunks)
{
    if (!ctx) return KF_EINVAL;
    if (n < 0 || !hits || !out) return fail(ctx, KF_EINVAL, "n >= 0, hits and out are required");
    kf_fit_params P;
    int rc = check_fit_params(ctx, params, P);
    if (rc) return rc;
    Geom G;
    if ((rc = to_geom(ctx, geom, G))) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if (n == 0) return KF_OK;
    if (!is_host_ptr(hits->offsets) || !is_host_ptr(hits->layer) || !is_host_ptr(hits->x) ||
        !is_host_ptr(hits->y) || !is_host_ptr(hits->z))
        return fail(ctx, KF_EINVAL, "kf_fit_host: hits must be host memory");
    const void *outs[6] = {out->state, out->cov, out->chi2, out->ndof, out->status, out->cov_f32};
    for (const void *o : outs)
        if (o && !is_host_ptr(o)) return fail(ctx, KF_EINVAL, "kf_fit_host: outputs must be host memory");
    if (n_chunks < 0 || n_chunks > 64) return fail(ctx, KF_EINVAL, "n_chunks must be 0..64");
    if (hits->offsets[0] != 0) return fail(ctx, KF_EINVAL, "offsets[0] must be 0");
    const int64_t nh = hits->offsets[n];
    if (nh < 0) return fail(ctx, KF_EINVAL, "offsets[n] < 0");
    int C = n_chunks ? n_chunks : (n >= 65536 ? 8 : 1);
    if (C > n) C = n;
    // concurrent calls on one context share host_ws and hs: one at a time
    std::lock_guard<std::mutex> hold(ctx->host_mu);
    // device layout
    const size_t nhist = order_scratch_ints();
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // Three streams in turn, so that one chunk's copy in, another's fit and a
    // third's copy out overlap; the first and last chunks are half as large as the
    // others, since their copy in (resp. out) has nothing to overlap with.
    const int64_t wsum = 2 * (int64_t)C - 2;  // chunk weights 1, 2, ..., 2, 1
    auto bound = [&](int c) -> int {
        if (C == 1) return c == 0 ? 0 : n;
        const int64_t w = c == 0 ? 0 : (c == C ? wsum : 2 * (int64_t)c - 1);
        return (int)((int64_t)n * w / wsum);
    };
    int cmax = 0;  // the largest chunk: the size of each stream's phase-1 -> phase-2 carry
    for (int c = 0; c < C; ++c) cmax = std::max(cmax, bound(c + 1) - bound(c));
    const size_t carry_b = P.precision == KF_PREC_FP64 ? 0 : al(fit_carry_bytes(cmax));
    size_t o_off = 0, o_lay = o_off + al((size_t)(n + 1) * 4), o_x = o_lay + al((size_t)nh), o_y = o_x + al(nh * 4),
           o_z = o_y + al(nh * 4), o_seed = o_z + al(nh * 4), o_q = o_seed + al((size_t)6 * n * 4),
           o_st = o_q + al((size_t)n), o_cov = o_st + al((size_t)6 * n * 8), o_chi = o_cov + al((size_t)21 * n * 8),
           o_nd = o_chi + al((size_t)n * 8), o_sts = o_nd + al((size_t)n * 4), o_ord = o_sts + al((size_t)n * 4),
           o_carry = o_ord + 3 * al((nhist + (size_t)n) * 4), o_c32 = o_carry + 3 * carry_b,
           total = o_c32 + (out->cov_f32 ? al((size_t)21 * n * 4) : 0);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < 3; ++i)
            if (!ctx->hs[i] && cudaStreamCreateWithFlags(&ctx->hs[i], cudaStreamNonBlocking) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "stream create");
        Buf &b = ctx->host_ws;
        if (b.n < total) {
            if (ctx->budget && ctx->used - b.n + total > ctx->budget)
                return fail(ctx, KF_ENOMEM, "kf_fit_host buffers of %zu bytes exceed the budget", total);
            if (b.p) {
                cudaFree(b.p);
                ctx->used -= b.n;
                b = Buf{};
            }
            if (cudaMalloc(&b.p, total) != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, KF_ENOMEM, "cudaMalloc(%zu) for kf_fit_host", total);
            }
            b.n = total;
            ctx->used += total;
        }
    }
    char *base = static_cast<char *>(ctx->host_ws.p);
    int32_t *d_off = reinterpret_cast<int32_t *>(base + o_off);
    uint8_t *d_lay = reinterpret_cast<uint8_t *>(base + o_lay);
    float *d_x = reinterpret_cast<float *>(base + o_x);
    float *d_y = reinterpret_cast<float *>(base + o_y);
    float *d_z = reinterpret_cast<float *>(base + o_z);
    float *d_seed = reinterpret_cast<float *>(base + o_seed);
    int8_t *d_q = reinterpret_cast<int8_t *>(base + o_q);
    double *d_st = reinterpret_cast<double *>(base + o_st);
    double *d_cov = reinterpret_cast<double *>(base + o_cov);
    float *d_c32 = reinterpret_cast<float *>(base + o_c32);
    double *d_chi = reinterpret_cast<double *>(base + o_chi);
    int32_t *d_nd = reinterpret_cast<int32_t *>(base + o_nd);
    uint32_t *d_sts = reinterpret_cast<uint32_t *>(base + o_sts);
    const bool fp64 = P.precision == KF_PREC_FP64;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < C && e == cudaSuccess; ++c) {
        const int t0 = bound(c), t1 = bound(c + 1);
        const int cnt = t1 - t0;
        if (cnt <= 0) continue;
        cudaStream_t st = ctx->hs[c % 3];
        int32_t *hist = reinterpret_cast<int32_t *>(base + o_ord + (c % 3) * al((nhist + (size_t)n) * 4));
        int32_t *order = hist + nhist;
        const int64_t h0 = hits->offsets[t0], h1 = hits->offsets[t1];
        e = cudaMemcpyAsync(d_off + t0, hits->offsets + t0, (size_t)(cnt + 1) * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && h1 > h0) {
            e = cudaMemcpyAsync(d_lay + h0, hits->layer + h0, (size_t)(h1 - h0), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_x + h0, hits->x + h0, (size_t)(h1 - h0) * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_y + h0, hits->y + h0, (size_t)(h1 - h0) * 4, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_z + h0, hits->z + h0, (size_t)(h1 - h0) * 4, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = launch_seeds(G, cnt, n, t0, d_off, d_x, d_y, d_z, d_seed, d_q, st);
        if (e == cudaSuccess)
            e = launch_order(cnt, d_off + t0, d_seed + 3 * (size_t)n + t0, d_seed + 5 * (size_t)n + t0, d_lay, &G,
                             std::max(3, P.n_fp64_updates), hist, order, st);
        if (e == cudaSuccess) {
            FitArgs a;
            memset(&a, 0, sizeof a);
            a.n = n;
            a.t_begin = t0;
            a.count = cnt;
            a.n64 = P.n_fp64_updates;
            a.seed_df = P.seed_update == KF_SEED_UD_DF;
            a.seed_cov = P.seed_cov;
            a.ms_on = P.ms_on;
            a.meas_model = P.meas_model;
            a.seed_state = d_seed;
            a.q = d_q;
            a.off = d_off;
            a.layer = d_lay;
            a.hx = d_x;
            a.hy = d_y;
            a.hz = d_z;
            a.o_state = d_st;
            a.o_cov = out->cov ? d_cov : nullptr;
            a.o_cov32 = out->cov_f32 ? d_c32 : nullptr;
            a.o_chi2 = d_chi;
            a.o_ndof = d_nd;
            a.o_status = d_sts;
            a.order = order;
            if (!fp64) fit_carve_carry(a.carry, base + o_carry + (c % 3) * carry_b, cnt);
            e = launch_fit(G, a, fp64, 128, st);
        }
        // results of this range back to the host: the range of every state and
        // covariance plane as one strided copy each
        if (e == cudaSuccess && out->state)
            e = cudaMemcpy2DAsync(out->state + t0, (size_t)n * 8, d_st + t0, (size_t)n * 8, (size_t)cnt * 8, 6,
                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->cov)
            e = cudaMemcpy2DAsync(out->cov + t0, (size_t)n * 8, d_cov + t0, (size_t)n * 8, (size_t)cnt * 8, 21,
                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->cov_f32)
            e = cudaMemcpy2DAsync(out->cov_f32 + t0, (size_t)n * 4, d_c32 + t0, (size_t)n * 4, (size_t)cnt * 4, 21,
                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->chi2)
            e = cudaMemcpyAsync(out->chi2 + t0, d_chi + t0, (size_t)cnt * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->ndof)
            e = cudaMemcpyAsync(out->ndof + t0, d_nd + t0, (size_t)cnt * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->status)
            e = cudaMemcpyAsync(out->status + t0, d_sts + t0, (size_t)cnt * 4, cudaMemcpyDeviceToHost, st);
    }
    for (int i = 0; i < 3; ++i) {
        const cudaError_t es = cudaStreamSynchronize(ctx->hs[i]);
        if (e == cudaSuccess) e = es;
    }
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "kf_fit_host");
}

int kf_autotune_fit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                    const kf_seeds *seeds, const kf_track_hits *hits, const kf_tracks_out *out, void *stream,
                    char *report, size_t report_len)
{
    if (!ctx) return KF_EINVAL;
    kf_fit_params P;
    int rc = check_fit_params(ctx, params, P);
    if (rc) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if (n <= 0) return fail(ctx, KF_EINVAL, "autotune needs n > 0");
    if (P.meas_model != KF_MEAS_LAYER)
        return fail(ctx, KF_EINVAL, "the persistent schedule runs measurement model KF_MEAS_LAYER only");
    const bool fp64 = P.precision == KF_PREC_FP64;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Tuned best;
    best.ms = 1e30f;
    const int blocks[3] = {64, 128, 256};
    const int chunks[3] = {1, 2, 4};  // tracks per thread per grab
    for (int bi = 0; bi < 3; ++bi) {
        const int occ = persistent_blocks_per_sm(fp64, blocks[bi]);
        if (occ <= 0) continue;
        for (int ci = 0; ci < 3; ++ci) {
            Tuned c;
            c.block = blocks[bi];
            c.chunk = chunks[ci];
            c.grid = ctx->sm_count * occ;
            // warm-up, then the best of three timed runs
            rc = fit_impl(ctx, geom, &P, n, seeds, hits, out, stream, &c);
            if (rc) break;
            float bestc = 1e30f;
            for (int r = 0; r < 3 && !rc; ++r) {
                cudaEventRecord(e0, st);
                rc = fit_impl(ctx, geom, &P, n, seeds, hits, out, stream, &c);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < bestc) bestc = ms;
            }
            if (rc) break;
            c.ms = bestc;
            if (c.ms < best.ms) best = c;
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->tuned[{fp64 ? 1 : 0, n_bucket(n)}] = best;
    }
    if (report && report_len)
        snprintf(report, report_len, "%d,%d,%d,%.4f", best.block, best.chunk, best.grid, best.ms);
    return KF_OK;
}

int kf_layout_transport(kf_ctx *ctx, int32_t layout, int32_t n, const float *J, const float *P, float *P_out,
                        void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (layout != KF_LAYOUT_AOS && layout != KF_LAYOUT_SOA && layout != KF_LAYOUT_BLOCK)
        return fail(ctx, KF_EINVAL, "layout must be KF_LAYOUT_AOS, KF_LAYOUT_SOA or KF_LAYOUT_BLOCK");
    if (n < 0 || (layout == KF_LAYOUT_BLOCK && n % 32))
        return fail(ctx, KF_EINVAL, "n >= 0 (a multiple of 32 for KF_LAYOUT_BLOCK)");
    int rc = set_dev(ctx);
    if (rc) return rc;
    if (n == 0) return KF_OK;
    NEED_DEV(J, "J");
    NEED_DEV(P, "P");
    NEED_DEV(P_out, "P_out");
    cudaError_t e = launch_transport_layout(layout, n, J, P, P_out, (cudaStream_t)stream);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "layout transport kernel");
}

int kf_measure_peak(kf_ctx *ctx, int which, double *flops_per_s)
{
    if (!ctx) return KF_EINVAL;
    if ((which != 0 && which != 1) || !flops_per_s) return fail(ctx, KF_EINVAL, "which must be 0 or 1");
    int rc = set_dev(ctx);
    if (rc) return rc;
    void *wsp = nullptr;
    if ((rc = ws_get(ctx, nullptr, (size_t)ctx->sm_count * 8 * sizeof(double) + 256, &wsp))) return rc;
    cudaError_t e = measure_peak(which, ctx->sm_count, wsp, flops_per_s);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "peak kernel");
}

int kf_bin_hits(kf_ctx *ctx, int32_t n_hits, const float *x, const float *y, const float *z, double half_len,
                int32_t *perm_out, int32_t *offsets_out, float *packed_out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (n_hits < 0 || !(half_len > 0)) return fail(ctx, KF_EINVAL, "n_hits >= 0 and half_len > 0 required");
    int rc = set_dev(ctx);
    if (rc) return rc;
    NEED_DEV(offsets_out, "offsets_out");
    if (n_hits > 0) {
        NEED_DEV(x, "x");
        NEED_DEV(y, "y");
        NEED_DEV(z, "z");
        NEED_DEV(perm_out, "perm_out");
        OPT_DEV_AL(packed_out, "packed_out", 16);
    }
    cudaStream_t st = (cudaStream_t)stream;
    void *wsp = nullptr;
    if ((rc = ws_get(ctx, st, bin_scratch_bytes(n_hits), &wsp))) return rc;
    cudaError_t e = launch_bin(n_hits, x, y, z, half_len, perm_out, offsets_out, packed_out, wsp, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "binning kernels");
}

int kf_bin_hits_batched(kf_ctx *ctx, int32_t n_segments, const int32_t *segment_offsets, const double *half_len,
                        const float *x, const float *y, const float *z, int32_t *perm_out, int32_t *offsets_out,
                        float *packed_out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (n_segments <= 0 || !segment_offsets || !half_len)
        return fail(ctx, KF_EINVAL, "n_segments > 0, segment_offsets and half_len required");
    if (segment_offsets[0] != 0) return fail(ctx, KF_EINVAL, "segment_offsets[0] must be 0");
    for (int s = 0; s < n_segments; ++s) {
        if (segment_offsets[s + 1] < segment_offsets[s])
            return fail(ctx, KF_EINVAL, "segment_offsets must not decrease");
        if (!(half_len[s] > 0)) return fail(ctx, KF_EINVAL, "half_len[%d] must be > 0", s);
    }
    const int H = segment_offsets[n_segments];
    int rc = set_dev(ctx);
    if (rc) return rc;
    NEED_DEV(offsets_out, "offsets_out");
    if (H > 0) {
        NEED_DEV(x, "x");
        NEED_DEV(y, "y");
        NEED_DEV(z, "z");
        NEED_DEV(perm_out, "perm_out");
        OPT_DEV_AL(packed_out, "packed_out", 16);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t so = ((size_t)(n_segments + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
    const size_t hl = ((size_t)n_segments * sizeof(double) + 255) & ~(size_t)255;
    void *wsp = nullptr;
    if ((rc = ws_get(ctx, st, so + hl + bin_segments_scratch_bytes(H, n_segments), &wsp))) return rc;
    char *w = static_cast<char *>(wsp);
    // one copy from a pageable buffer of our own, staged by the runtime before the call returns
    std::vector<char> stage(so + (size_t)n_segments * sizeof(double));
    memcpy(stage.data(), segment_offsets, (size_t)(n_segments + 1) * sizeof(int32_t));
    memcpy(stage.data() + so, half_len, (size_t)n_segments * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(w, stage.data(), stage.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_bin_segments(n_segments, H, reinterpret_cast<const int32_t *>(w),
                                reinterpret_cast<const double *>(w + so), x, y, z, perm_out, offsets_out, packed_out,
                                w + so + hl, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "segmented binning kernels");
}

// device copy of the layer table and event offsets, in the stream's workspace after `skip` bytes
static int upload_layers(kf_ctx *ctx, cudaStream_t st, int n_events, int n_layers, const kf_binned_layer *layers,
                         const int32_t *event_offsets, size_t extra, void **ws_out, LayerDev **dl, int32_t **deoff,
                         bool need_xyz)
{
    const size_t nl = (size_t)n_events * n_layers;
    std::vector<LayerDev> host(nl);
    for (size_t i = 0; i < nl; ++i) {
        const kf_binned_layer &L = layers[i];
        if (L.n_hits < 0) return fail(ctx, KF_EINVAL, "layer %zu: n_hits < 0", i);
        host[i].packed = reinterpret_cast<const float4 *>(L.packed);
        host[i].offsets = L.offsets;
        host[i].x = L.x;
        host[i].y = L.y;
        host[i].z = L.z;
        host[i].n_hits = L.n_hits;
        host[i].surface = L.surface;
    }
    const size_t tbl = nl * sizeof(LayerDev), eo = (size_t)(n_events + 1) * sizeof(int32_t);
    const size_t tbl_al = (tbl + 255) & ~(size_t)255, eo_al = (eo + 255) & ~(size_t)255;
    void *wsp = nullptr;
    int rc = ws_get(ctx, st, tbl_al + eo_al + extra, &wsp);
    if (rc) return rc;
    // one copy from a pageable buffer of our own (the caller's arrays may be
    // page-locked): the runtime stages a pageable source before the call
    // returns, so the copy is ordered on the stream without waiting for it
    std::vector<char> stage(tbl_al + eo);
    memcpy(stage.data(), host.data(), tbl);
    memcpy(stage.data() + tbl_al, event_offsets, eo);
    cudaError_t e = cudaMemcpyAsync(wsp, stage.data(), stage.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "uploading the layer table");
    (void)need_xyz;
    *ws_out = (char *)wsp + tbl_al + eo_al;
    *dl = reinterpret_cast<LayerDev *>(wsp);
    *deoff = reinterpret_cast<int32_t *>((char *)wsp + tbl_al);
    return KF_OK;
}

static int check_events(kf_ctx *ctx, const kf_geometry *geom, int n_events, int n_layers,
                        const kf_binned_layer *layers, const int32_t *event_offsets, bool need_xyz)
{
    if (n_events <= 0 || n_layers < 3 || n_layers > KF_MAX_SURFACES || !layers || !event_offsets)
        return fail(ctx, KF_EINVAL, "need n_events > 0, 3 <= n_layers <= %d, layers and event_offsets",
                    KF_MAX_SURFACES);
    if (event_offsets[0] != 0) return fail(ctx, KF_EINVAL, "event_offsets[0] must be 0");
    for (int e = 0; e < n_events; ++e)
        if (event_offsets[e + 1] < event_offsets[e]) return fail(ctx, KF_EINVAL, "event_offsets must not decrease");
    for (int i = 0; i < n_events * n_layers; ++i) {
        const kf_binned_layer &L = layers[i];
        if (L.surface < 0 || L.surface >= geom->n_surfaces)
            return fail(ctx, KF_EINVAL, "layer %d: surface index out of range", i);
        if (geom->surfaces[L.surface].kind != 0) return fail(ctx, KF_EINVAL, "layer %d: building needs barrels", i);
        if (i % n_layers >= 3 && L.n_hits > 0) {
            if (!is_device_ptr_on(L.packed, ctx->device, 16) || !is_device_ptr_on(L.offsets, ctx->device, 4))
                return fail(ctx, KF_EINVAL, "layer %d: packed and offsets must be device memory (16- and 4-byte aligned)", i);
        } else if (i % n_layers >= 3 && !is_device_ptr_on(L.offsets, ctx->device, 4)) {
            return fail(ctx, KF_EINVAL, "layer %d: offsets must be device memory, 4-byte aligned", i);
        }
        if (need_xyz && i % n_layers >= 3 && L.n_hits > 0 &&
            (!is_device_ptr_on(L.x, ctx->device, 4) || !is_device_ptr_on(L.y, ctx->device, 4) ||
             !is_device_ptr_on(L.z, ctx->device, 4)))
            return fail(ctx, KF_EINVAL, "layer %d: x, y, z must be device memory, 4-byte aligned", i);
    }
    return KF_OK;
}

int kf_build_besthit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *fit, const kf_build_params *bp,
                     int32_t n_events, int32_t n_layers, const kf_binned_layer *layers, const int32_t *event_offsets,
                     const kf_seeds *seeds, const float *seed_hits, int32_t *hit_idx_out, const kf_tracks_out *out,
                     void *stream)
{
    if (!ctx) return KF_EINVAL;
    kf_fit_params P;
    int rc = check_fit_params(ctx, fit, P);
    if (rc) return rc;
    Geom G;
    if ((rc = to_geom(ctx, geom, G))) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if ((rc = check_events(ctx, geom, n_events, n_layers, layers, event_offsets, false))) return rc;
    kf_build_params B = {3.0, 30.0, 32, 0, nullptr};
    if (bp) B = *bp;
    if (!(B.nsigma > 0) || !(B.chi2_cut > 0) || B.max_cand < 1 || B.max_cand > 64)
        return fail(ctx, KF_EINVAL, "build params: nsigma > 0, chi2_cut > 0, 1 <= max_cand <= 64");
    const int n = event_offsets[n_events];
    if (n == 0) return KF_OK;
    if (!seeds || !out) return fail(ctx, KF_EINVAL, "seeds and out are required");
    NEED_DEV(seeds->state, "seeds.state");
    NEED_DEV(seeds->q, "seeds.q");
    NEED_DEV(seed_hits, "seed_hits");
    NEED_DEV(hit_idx_out, "hit_idx_out");
    OPT_DEV(out->state, "out.state");
    OPT_DEV(out->cov, "out.cov");
    OPT_DEV(out->cov_f32, "out.cov_f32");
    OPT_DEV(out->chi2, "out.chi2");
    OPT_DEV(out->ndof, "out.ndof");
    OPT_DEV(out->status, "out.status");
    OPT_DEV(B.debug_pred, "debug_pred");
    cudaStream_t st = (cudaStream_t)stream;
    void *rest = nullptr;
    LayerDev *dl = nullptr;
    int32_t *deoff = nullptr;
    const size_t nhist = order_scratch_ints();
    const size_t ord_bytes = ((nhist + (size_t)n) * sizeof(int32_t) + 255) & ~(size_t)255;
    if ((rc = upload_layers(ctx, st, n_events, n_layers, layers, event_offsets,
                            ord_bytes + build_seed_scratch_bytes(n), &rest, &dl, &deoff, false)))
        return rc;
    int32_t *hist = reinterpret_cast<int32_t *>(rest);
    int32_t *order = hist + nhist;
    cudaError_t eo =
        launch_order(n, nullptr, seeds->state + 3 * (size_t)n, nullptr, nullptr, &G, 0, hist, order, st);
    if (eo != cudaSuccess) return cuda_fail(ctx, eo, "build order");
    BuildArgs a;
    memset(&a, 0, sizeof a);
    a.seed_scratch = static_cast<char *>(rest) + ord_bytes;
    a.n = n;
    a.n_events = n_events;
    a.n_layers = n_layers;
    a.n64 = P.n_fp64_updates;
    a.seed_df = P.seed_update == KF_SEED_UD_DF;
    a.seed_cov = P.seed_cov;
    a.ms_on = P.ms_on;
    a.meas_model = P.meas_model;
    a.max_cand = B.max_cand;
    a.nsigma = (float)B.nsigma;
    a.chi2_cut = (float)B.chi2_cut;
    a.layers = dl;
    a.event_off = deoff;
    a.seed_state = seeds->state;
    a.q = seeds->q;
    a.seed_hits = seed_hits;
    a.hit_idx = hit_idx_out;
    a.order = order;
    a.o_state = out->state;
    a.o_cov = out->cov;
    a.o_cov32 = out->cov_f32;
    a.o_chi2 = out->chi2;
    a.o_ndof = out->ndof;
    a.o_status = out->status;
    a.dbg_pred = B.debug_pred;
    cudaError_t e = launch_build(G, a, P.precision == KF_PREC_FP64, B.warp_coop != 0, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "build kernel");
}

int kf_build_ckf(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *fit, const kf_build_params *bp,
                 int32_t n_slots, int32_t n_events, int32_t n_layers, const kf_binned_layer *layers,
                 const int32_t *event_offsets, const kf_seeds *seeds, const float *seed_hits, int32_t *hit_idx_out,
                 const kf_tracks_out *out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    kf_fit_params P;
    int rc = check_fit_params(ctx, fit, P);
    if (rc) return rc;
    if (P.precision != KF_PREC_MIXED)
        return fail(ctx, KF_EINVAL, "combinatorial building runs the mixed precision policy only");
    if (P.meas_model != KF_MEAS_LAYER)
        return fail(ctx, KF_EINVAL, "combinatorial building runs measurement model KF_MEAS_LAYER only");
    if (n_slots != 1 && n_slots != 2 && n_slots != 4 && n_slots != 8)
        return fail(ctx, KF_EINVAL, "n_slots must be 1, 2, 4 or 8");
    Geom G;
    if ((rc = to_geom(ctx, geom, G))) return rc;
    if ((rc = set_dev(ctx))) return rc;
    if ((rc = check_events(ctx, geom, n_events, n_layers, layers, event_offsets, false))) return rc;
    kf_build_params B = {3.0, 30.0, 32, 0, nullptr};
    if (bp) B = *bp;
    if (!(B.nsigma > 0) || !(B.chi2_cut > 0) || B.max_cand < 1 || B.max_cand > 64)
        return fail(ctx, KF_EINVAL, "build params: nsigma > 0, chi2_cut > 0, 1 <= max_cand <= 64");
    const int n = event_offsets[n_events];
    if (n == 0) return KF_OK;
    if (!seeds || !out) return fail(ctx, KF_EINVAL, "seeds and out are required");
    NEED_DEV(seeds->state, "seeds.state");
    NEED_DEV(seeds->q, "seeds.q");
    NEED_DEV(seed_hits, "seed_hits");
    NEED_DEV(hit_idx_out, "hit_idx_out");
    OPT_DEV(out->state, "out.state");
    OPT_DEV(out->cov, "out.cov");
    OPT_DEV(out->cov_f32, "out.cov_f32");
    OPT_DEV(out->chi2, "out.chi2");
    OPT_DEV(out->ndof, "out.ndof");
    OPT_DEV(out->status, "out.status");
    cudaStream_t st = (cudaStream_t)stream;
    void *rest = nullptr;
    LayerDev *dl = nullptr;
    int32_t *deoff = nullptr;
    const size_t nhist = order_scratch_ints();
    const size_t ord_bytes = ((nhist + (size_t)n) * sizeof(int32_t) + 255) & ~(size_t)255;
    if ((rc = upload_layers(ctx, st, n_events, n_layers, layers, event_offsets,
                            ord_bytes + ckf_scratch_bytes(n, n_layers, n_slots), &rest, &dl, &deoff, false)))
        return rc;
    int32_t *hist = reinterpret_cast<int32_t *>(rest);
    int32_t *order = hist + nhist;
    cudaError_t eo =
        launch_order(n, nullptr, seeds->state + 3 * (size_t)n, nullptr, nullptr, &G, 0, hist, order, st);
    if (eo != cudaSuccess) return cuda_fail(ctx, eo, "build order");
    CkfArgs c;
    memset(&c, 0, sizeof c);
    BuildArgs &a = c.b;
    a.n = n;
    a.n_events = n_events;
    a.n_layers = n_layers;
    a.n64 = P.n_fp64_updates;
    a.seed_df = P.seed_update == KF_SEED_UD_DF;
    a.seed_cov = P.seed_cov;
    a.ms_on = P.ms_on;
    a.meas_model = P.meas_model;
    a.max_cand = B.max_cand;
    a.nsigma = (float)B.nsigma;
    a.chi2_cut = (float)B.chi2_cut;
    a.layers = dl;
    a.event_off = deoff;
    a.seed_state = seeds->state;
    a.q = seeds->q;
    a.seed_hits = seed_hits;
    a.hit_idx = hit_idx_out;
    a.order = order;
    a.o_state = out->state;
    a.o_cov = out->cov;
    a.o_cov32 = out->cov_f32;
    a.o_chi2 = out->chi2;
    a.o_ndof = out->ndof;
    a.o_status = out->status;
    c.n_slots = n_slots;
    ckf_carve(c, static_cast<char *>(rest) + ord_bytes, n, n_layers, n_slots);
    cudaError_t e = launch_ckf(G, c, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "combinatorial build kernels");
}

int kf_gather_hits(kf_ctx *ctx, int32_t n_events, int32_t n_layers, const kf_binned_layer *layers,
                   const int32_t *event_offsets, const float *seed_hits, const int32_t *hit_idx, int32_t *offsets_out,
                   uint8_t *layer_out, float *x_out, float *y_out, float *z_out, void *stream)
{
    if (!ctx) return KF_EINVAL;
    int rc = set_dev(ctx);
    if (rc) return rc;
    if (n_events <= 0 || n_layers < 3 || n_layers > KF_MAX_SURFACES || !layers || !event_offsets)
        return fail(ctx, KF_EINVAL, "need n_events > 0, 3 <= n_layers <= %d, layers and event_offsets",
                    KF_MAX_SURFACES);
    for (int i = 0; i < n_events * n_layers; ++i)
        if (i % n_layers >= 3 && layers[i].n_hits > 0 &&
            (!is_device_ptr_on(layers[i].x, ctx->device, 4) || !is_device_ptr_on(layers[i].y, ctx->device, 4) ||
             !is_device_ptr_on(layers[i].z, ctx->device, 4)))
            return fail(ctx, KF_EINVAL, "layer %d: x, y, z must be device memory, 4-byte aligned", i);
    const int n = event_offsets[n_events];
    NEED_DEV(offsets_out, "offsets_out");
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(offsets_out, 0, sizeof(int32_t), (cudaStream_t)stream);
        return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "memset");
    }
    NEED_DEV(seed_hits, "seed_hits");
    NEED_DEV(hit_idx, "hit_idx");
    NEED_DEV(layer_out, "layer_out");
    NEED_DEV(x_out, "x_out");
    NEED_DEV(y_out, "y_out");
    NEED_DEV(z_out, "z_out");
    cudaStream_t st = (cudaStream_t)stream;
    void *rest = nullptr;
    LayerDev *dl = nullptr;
    int32_t *deoff = nullptr;
    if ((rc = upload_layers(ctx, st, n_events, n_layers, layers, event_offsets, gather_scratch_bytes(n), &rest, &dl,
                            &deoff, true)))
        return rc;
    cudaError_t e = launch_gather(n, n_events, n_layers, dl, deoff, seed_hits, hit_idx, offsets_out, layer_out, x_out,
                                  y_out, z_out, rest, st);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e, "gather kernels");
}

}  // extern "C"

// Context services for the serving runtime (kf_server.cu).
namespace kfd {
int ctx_geom(kf_ctx *ctx, const kf_geometry *g, Geom &G) { return to_geom(ctx, g, G); }
int ctx_fit_params(kf_ctx *ctx, const kf_fit_params *p, kf_fit_params &q) { return check_fit_params(ctx, p, q); }
int ctx_device(const kf_ctx *ctx) { return ctx->device; }
int ctx_fail(kf_ctx *ctx, int code, const char *msg) { return fail(ctx, code, "%s", msg); }
}  // namespace kfd
