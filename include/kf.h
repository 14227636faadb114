/*
 * kf.h -- C ABI of libkf.so: batched Kalman-filter track fitting and
 * best-hit track building on one GB300 (sm_103a).
 *
 * The method (arXiv:1711.06571): Kalman-filter tracking in three stages,
 * seeding, building and fitting (Sec. 2); state in hybrid coordinates, global
 * Cartesian position plus polar momentum, in a uniform longitudinal field
 * (Sec. 3); propagation to each detector layer and a KF update on the plane
 * tangent to the hit radius (Sec. 4.1); multiple scattering folded into the
 * trajectory estimate (Sec. 2); a binned hit structure for selecting hit
 * candidates (Sec. 3.1); one track per GPU thread over a structure-of-arrays
 * layout with coalesced loads, several events in flight (Sec. 4.2, 4.3).
 *
 * Conventions for every entry point
 *   - Return value: KF_OK (0) or a negative KF_E* code; the context keeps a
 *     message for the last error (kf_ctx_last_error).  Per-track problems never
 *     fail a call: they are reported in the per-track status word (KF_ST_*).
 *   - Arrays marked "device" must be device memory of the context's GPU
 *     (cudaMalloc / torch CUDA tensors), at an address that is a multiple of
 *     the element size (16 bytes for packed hits, read as 4-float vectors); a
 *     host pointer or a misaligned one is rejected with KF_EINVAL before
 *     anything is launched.  Arrays marked "host" are host memory.
 *   - The caller owns every array passed in or out.  The context owns its
 *     scratch (workspace, autotune results, CUDA graphs) and frees it in
 *     kf_ctx_destroy.
 *   - Work is enqueued on the given CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream) and returns before it completes;
 *     results are valid once the stream has been synchronised.
 *   - Structure-of-arrays layouts: "[k][n]" means k planes of n values, plane
 *     i at offset i*n.  Track state vectors are (x, y, z, 1/pT, phi, theta) in
 *     cm, GeV^-1 and rad; the charge q = +-1 is carried separately and 1/pT may
 *     change sign during a fit (the physical curvature is -q * kappa * Bz / pT).
 *     Covariances are packed lower triangles, row-major, i >= j:
 *     entry (i, j) at index i*(i+1)/2 + j, 21 values.
 *
 * Calls and the problem statement they follow
 *   kf_fit (seeds, hits, layer geometry -> fitted states, covariances, chi2)
 *   and kf_build_besthit (seeds, binned hits per layer -> hit indices per layer
 *   plus fitted states) are the two forms of the hot path.  Three choices of
 *   this interface differ from a one-call-per-concern layout:
 *   - the arithmetic precision is a field of kf_fit_params (precision,
 *     n_fp64_updates, seed_update), passed with every fit and build call,
 *     not a context-wide setter, so that calls of different precision can
 *     share a context and run concurrently;
 *   - serving statistics are read with kf_server_stats_get, which fills a
 *     caller-owned kf_server_stats structure (the structure takes the plain
 *     name);
 *   - kf_server_poll reports a finished event's latency and leaves the
 *     results in the caller's output arrays named at submission, instead of
 *     returning a result record that the library would own.
 */
#ifndef KF_H
#define KF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define KF_OK 0
#define KF_EINVAL (-1)   /* bad argument, size or pointer kind */
#define KF_ENOMEM (-2)   /* workspace allocation failed */
#define KF_ECUDA (-3)    /* a CUDA call or kernel launch failed */
#define KF_ETIMEOUT (-4) /* a device-side wait ran out (reported, never trapped) */
#define KF_EAGAIN (-5)   /* serving: result not ready yet */
#define KF_EBUSY (-6)    /* serving: request exceeds the memory budget */
#define KF_ESIZE (-7)    /* size beyond a fixed maximum (kf_bin_hits_static) */

/* per-track status bits */
#define KF_ST_NO_INTERSECT 1u /* helix never reaches the next surface; later hits unused */
#define KF_ST_CHOL_FAIL 2u    /* innovation covariance S not positive definite */
#define KF_ST_NONFINITE 4u    /* non-finite state */
#define KF_ST_CAND_CAPPED 8u  /* building: more window candidates than the cap */
#define KF_ST_GRAZING 16u     /* scattering thickness used the |cos(alpha)| >= 0.05 guard */
#define KF_ST_THETA_RANGE 32u /* an update carried theta out of (0, pi), through the pole of the
                                 (.., phi, theta) parametrisation where cot(theta) diverges: the
                                 next propagation is refused and the track ends there (set
                                 together with KF_ST_NO_INTERSECT) */
#define KF_ST_FP64_TRACK 64u  /* KF_PREC_MIXED: the track crosses one surface twice in a row (it
                                 turns back through a layer near its apex); it was fitted in
                                 FP64 throughout */

/* precision policies (kf_fit_params.precision) */
#define KF_PREC_MIXED 0 /* FP32 propagation/transport/update; FP64 for the 3x3 S
                           solve and for the first n_fp64_updates updates */
#define KF_PREC_FP64 1  /* every step in FP64 (the plain reference path) */

/* arithmetic of the first updates of a KF_PREC_MIXED fit, where the 1e4 seed
 * covariance cancels eight to ten digits (kf_fit_params.seed_update) */
#define KF_SEED_UD_DF 0       /* default: double-float arithmetic (an unevaluated sum of
                                 two floats, about 48 bits) on the FP32 pipe, the
                                 covariance update in Bierman's U-D factored form
                                 (P = U D U^T, one scalar measurement at a time), the
                                 update at the seed hit in closed form */
#define KF_SEED_JOSEPH_FP64 1 /* FP64 covariance, Joseph-form updates */

/* scheduling of kf_fit (kf_fit_params.schedule) */
#define KF_SCHED_GRID 0       /* one thread per track, one launch */
#define KF_SCHED_PERSISTENT 1 /* tracks bucketed by hit count, persistent kernel
                                 with an atomic work queue, replayed as a CUDA graph */

/* measurement model (kf_fit_params.meas_model), Sec. 4.1 */
#define KF_MEAS_LAYER 0  /* the hit lies on its layer's surface: 3-D update there */
#define KF_MEAS_HIT_2D 1 /* non-ideal barrel: a barrel hit lies on the cylinder through
                            it (its module sits up to dr off the layer radius); the
                            track is carried to that cylinder and updated with the
                            two coordinates measured on the plane tangent to it at the
                            hit (r-phi and z; disk hits keep KF_MEAS_LAYER).  The first
                            hit of a fit, where the state starts, keeps the 3-D update.  Best-hit
                            building takes two steps per layer: to the layer's average
                            cylinder (scattering noise and the window, widened by dr,
                            there), then to each candidate's cylinder to score it.
                            Grid schedule and per-thread scoring only; the persistent
                            schedule, the autotuner and kf_build_ckf refuse it. */

#define KF_MAX_SURFACES 64
#define KF_NPHI 1024
#define KF_NZ 64
#define KF_NBINS (KF_NPHI * KF_NZ)

typedef struct kf_ctx kf_ctx;

/* One detector surface (Sec. 3: ideal barrel layers; Sec. 4.1: barrel closed by end-cap disks).
 * kind 0: barrel cylinder r = pos, |z| <= half_or_rin.
 * kind 1: disk z = pos, half_or_rin <= r <= r_out.
 * x_x0: thickness in radiation lengths at normal incidence.
 * sig_n: hit resolution along the surface normal; sig_rphi: along phi-hat;
 * sig_3: along z (barrel) or r (disk), all in cm.
 * dr: barrel, radial half-extent of the layer's modules (a non-ideal layer whose
 * hits lie within pos +- dr, Sec. 4.1); 0 for an ideal cylinder.  Read by the
 * building window under KF_MEAS_HIT_2D. */
typedef struct {
    int32_t kind;
    int32_t pad_;
    double pos;
    double half_or_rin;
    double r_out;
    double x_x0;
    double sig_n;
    double sig_rphi;
    double sig_3;
    double dr;
} kf_surface;

/* Detector and field.  surfaces: host array of n_surfaces (<= KF_MAX_SURFACES). */
typedef struct {
    double bz;   /* T, uniform along z (Sec. 3) */
    double mass; /* GeV, particle mass for the velocity in the scattering angle */
    int32_t n_surfaces;
    int32_t pad_;
    const kf_surface *surfaces;
} kf_geometry;

typedef struct {
    int32_t precision;      /* KF_PREC_MIXED | KF_PREC_FP64 */
    int32_t n_fp64_updates; /* MIXED: updates (from the seed) kept in FP64, 0..32; default 3 */
    double seed_cov;        /* seed covariance = seed_cov * I6, default 1e4 */
    int32_t ms_on;          /* 1: add multiple-scattering noise at every surface */
    int32_t schedule;       /* KF_SCHED_GRID | KF_SCHED_PERSISTENT */
    int32_t meas_model;     /* KF_MEAS_LAYER (default) | KF_MEAS_HIT_2D */
    int32_t seed_update;    /* MIXED: KF_SEED_UD_DF (default) | KF_SEED_JOSEPH_FP64, for the
                               first n_fp64_updates updates (the name predates the
                               double-float form: these are the extended-precision updates) */
} kf_fit_params;

/* Seeds: device SoA. state [6][n] FP32 (x, y, z, 1/pT, phi, theta at the
 * track's first hit); q [n] int8 (+1 / -1). */
typedef struct {
    const float *state;
    const int8_t *q;
} kf_seeds;

/* Hits of n tracks in path order, device CSR: track t owns hits
 * offsets[t] .. offsets[t+1]-1; layer[] is the surface index of each hit. */
typedef struct {
    const int32_t *offsets; /* [n+1], offsets[0] == 0, non-decreasing */
    const uint8_t *layer;   /* [offsets[n]] */
    const float *x;
    const float *y;
    const float *z;
} kf_track_hits;

/* Fitted tracks, device outputs.  state [6][n] and cov [21][n] in FP64 storage
 * whatever the compute precision (the mixed path keeps the position and phi in
 * float-float, which FP32 storage would round away); chi2 [n]; ndof [n] =
 * 2 * (hits used) - 5; status [n] KF_ST_* bits.  cov_f32 [21][n]: the same
 * covariance in FP32 storage, beside or instead of cov -- the mixed path
 * carries the covariance in FP32, so rounding it there loses nothing when the
 * last update ran in the FP32 layer loop, and it halves the covariance's bytes
 * (84 instead of 168 per track; the all-FP64 path rounds its covariance).  Any
 * pointer may be NULL. */
typedef struct {
    double *state;
    double *cov;
    double *chi2;
    int32_t *ndof;
    uint32_t *status;
    float *cov_f32;
} kf_tracks_out;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device cuda_device.  device_mem_budget_bytes caps
 * the context's own workspace (0 = no cap).  *out receives the context. */
int kf_ctx_create(kf_ctx **out, int cuda_device, size_t device_mem_budget_bytes);
/* Free the context and everything it owns.  NULL is accepted. */
void kf_ctx_destroy(kf_ctx *ctx);
/* Message for the last error of this context (owned by the context). */
const char *kf_ctx_last_error(const kf_ctx *ctx);
/* Library version string (static). */
const char *kf_version(void);

/* ---------------------------------------------------------------- seeding */

/* Seed estimate (Sec. 2: seeding gives first track parameters from a handful
 * of hits on the innermost layers; the estimate itself is a reading): for
 * each track, hit 0 and the next two hits at least 2 cm apart in x-y (hits
 * 0, 1, 2 on a barrel); signed curvature of the circle through them, 1/pT =
 * |k| / (kappa |Bz|), q = -sign(k), phi = tangent at hit 0, theta from the
 * arc length, position = hit 0.  FP32.  Tracks with fewer than 3 hits get a
 * zero state and q = +1.
 * hits: device CSR (n tracks); state_out: device [6][n]; q_out: device [n]. */
int kf_make_seeds(kf_ctx *ctx, const kf_geometry *geom, int32_t n, const kf_track_hits *hits, float *state_out,
                  int8_t *q_out, void *stream);

/* ---------------------------------------------------------------- fitting */

/* Kalman-filter fit of n tracks (Sec. 2: with the hit collection known, the
 * KF is applied over it without branching; Sec. 4.1: propagate to each layer,
 * update on the tangent plane).  For each hit in path order: propagate the
 * state along the helix to the hit's surface with the surface-constrained
 * 6x6 Jacobian (no propagation for hit 0, where the seed sits), transport
 * P <- J P J^T, add Highland scattering noise to the phi and theta variances,
 * then the 3-D update: r = m - x, S = H P H^T + R, chi2 = r^T S^-1 r via an
 * LDL^T (square-root-free Cholesky) factorisation of S in FP64, K = P H^T S^-1,
 * x += K r, P updated (Joseph form on the FP64 updates).  The output state is
 * the one at the last used hit.
 * params: host struct (NULL = defaults); seeds, hits: device; out: device. */
int kf_fit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n, const kf_seeds *seeds,
           const kf_track_hits *hits, const kf_tracks_out *out, void *stream);

/* Outward-inward refit (the final fit of Sec. 2 run a second time, from the
 * last hit back to the first, so that the estimate at the first hit uses
 * every hit).  Each track is run backwards by reversing its direction of
 * motion -- phi -> phi + pi, theta -> pi - theta, q -> -q, the same helix
 * traversed the other way -- and the hits the forward fit used (the first
 * (ndof + 5) / 2 of the track), in reverse order, are fitted as by kf_fit
 * (FP64 for the first updates), starting at the last used hit from the forward
 * fit's state there with the forward covariance times cov_scale (100 is
 * usual: the forward information then counts once more with weight 1/100,
 * and the filter stays on the fitted trajectory near a track's apex, where a
 * fresh 1e4 covariance makes the result depend on rounding); the result at the
 * first hit is turned back to the forward direction.
 *   hits: device CSR as for kf_fit (forward path order).
 *   fwd_state, fwd_cov: device [6][n] and [21][n] FP64, the forward fit's state
 *     and covariance at each track's last used hit (kf_fit's out.state and
 *     out.cov); q: device [n], the charges used by that fit; fwd_ndof: device
 *     [n], its ndof.  cov_scale > 0.
 *   out: device, state and covariance at the first hit (forward direction),
 *     chi2 and ndof of the backward pass, status.
 * Blocks until offsets[n] is read; the rest runs on the stream (precision and
 * measurement model from params; always the grid schedule). */
int kf_refit_inward(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                    const kf_track_hits *hits, const double *fwd_state, const double *fwd_cov, const int8_t *q,
                    const int32_t *fwd_ndof, double cov_scale, const kf_tracks_out *out, void *stream);

/* End-to-end fit from host memory: copies the hits to the device, estimates
 * the seeds (kf_make_seeds), fits (kf_fit) and copies the results back.  The
 * tracks are split into n_chunks ranges processed in turn on three internal
 * streams, so that one range's copy in, another's kernels and a third's copy
 * out overlap (Sec. 4.3: copies overlapped with processing); the first and last
 * ranges are half the size of the others.  Blocks until the results are in
 * host memory.  hits: host CSR as in kf_track_hits; out: host arrays with the
 * layouts of kf_tracks_out (any may be NULL).  Page-locked host memory makes
 * the copies asynchronous; pageable memory works but serialises them.
 * n_chunks: 1..64, 0 = automatic.  Device buffers are owned by the context and
 * kept for later calls of the same or smaller size.  Calls on one context from
 * several host threads run one at a time (they share those buffers and the
 * internal streams). */
int kf_fit_host(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                const kf_track_hits *hits, const kf_tracks_out *out, int32_t n_chunks);

/* Timing of kf_fit's kernels (no counterpart in the paper; it gives the roofline
 * of each phase).  enable != 0: every later grid-schedule kf_fit on this context
 * records CUDA events on its stream around its two phases -- on the mixed path
 * phase 1 is the kernel that runs the first updates from the seed (extended
 * precision) and phase 2 the kernel of the FP32 layer loop; the all-FP64 path
 * runs one kernel, timed as phase 1.  enable == 0 stops recording; enabling
 * again starts a new count.  kf_fit_phase_times waits for the timed calls and
 * returns their number (the last 1024 at most) and the mean durations of the
 * two phases in ms; KF_EINVAL if there is none.  Recording adds three event
 * records to each call and no synchronisation. */
int kf_fit_timing(kf_ctx *ctx, int enable);
int kf_fit_phase_times(kf_ctx *ctx, int32_t *n_calls, double *ms_phase1, double *ms_phase2);

/* Choose block size and tracks per thread (per work-queue grab) of the persistent
 * fit for this (n, hit count) by timing candidates on the given inputs (it
 * runs the fit several times and overwrites out).  The choice is cached in the
 * context and used by later kf_fit calls with schedule = KF_SCHED_PERSISTENT.
 * report (host, may be NULL) receives "block,tracks_per_thread,grid,ms" of the
 * winner. */
int kf_autotune_fit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *params, int32_t n,
                    const kf_seeds *seeds, const kf_track_hits *hits, const kf_tracks_out *out, void *stream,
                    char *report, size_t report_len);

/* ---------------------------------------------------------------- binning */

/* Bin one layer's hits into the (phi, z) grid used to select hit candidates
 * (Sec. 3.1), in FP64 from the FP32 coordinates:
 *   phi_bin = clamp(floor(((atan2(y, x) + pi) * 1024) / (2 pi)), 0, 1023)
 *   z_bin   = clamp(floor(((z + half_len) * 64) / (2 half_len)), 0, 63)
 *   key     = z_bin * 1024 + phi_bin
 * then a stable counting sort by key (ties keep the original order).
 * x, y, z: device [n_hits].  perm_out: device [n_hits], original index of the
 * i-th hit in binned order.  offsets_out: device [KF_NBINS + 1], hits of key k
 * are binned positions offsets[k] .. offsets[k+1]-1.  packed_out: device
 * [n_hits][4] floats (x, y, z, original index as int32 bits) in binned order,
 * or NULL.  half_len > 0.  n_hits == 0 is allowed (offsets all zero). */
int kf_bin_hits(kf_ctx *ctx, int32_t n_hits, const float *x, const float *y, const float *z, double half_len,
                int32_t *perm_out, int32_t *offsets_out, float *packed_out, void *stream);

/* The binning of kf_bin_hits for many layers at once (several layers of
 * several events, Sec. 4.2), in one pass of five kernels instead of five per
 * layer.  Segment s holds hits segment_offsets[s] .. segment_offsets[s+1]-1 of
 * the concatenated x, y, z and is binned with its own half_len[s]; its results
 * are exactly those of kf_bin_hits on that segment alone:
 *   perm_out: device [H] (H = segment_offsets[n_segments]), at the segment's
 *     positions, indices local to the segment;
 *   offsets_out: device [n_segments][KF_NBINS + 1], segment s's CSR offsets
 *     (local) at s * (KF_NBINS + 1);
 *   packed_out: device [H][4] or NULL, at the segment's positions, index bits
 *     local to the segment.
 * segment_offsets: host [n_segments + 1], starting at 0, non-decreasing
 * (empty segments are allowed); half_len: host [n_segments], each > 0.  Both
 * are copied before the call returns. */
int kf_bin_hits_batched(kf_ctx *ctx, int32_t n_segments, const int32_t *segment_offsets, const double *half_len,
                        const float *x, const float *y, const float *z, int32_t *perm_out, int32_t *offsets_out,
                        float *packed_out, void *stream);

/* Binning without any allocation.  The paper has no counterpart: this is the
 * binning of kf_bin_hits for callers that cannot call cudaMalloc, such as a
 * host framework that owns all device memory and hands it out itself, or a
 * real-time (trigger) process whose memory footprint is fixed at start-up.
 * It needs no context: its scratch is a fixed array in device memory,
 * 4 * (5 * KF_STATIC_MAX_HITS + KF_NBINS) bytes (about 5.5 MB), which every
 * GPU that loads the library holds until the process exits.
 *   - Arguments, layouts and results are those of kf_bin_hits; n_hits may be
 *     at most KF_STATIC_MAX_HITS, larger sizes return KF_ESIZE and do nothing.
 *     Host pointers, memory of a GPU other than the current one, or a bad
 *     half_len return KF_EINVAL.
 *   - Each call looks up the array's device address (cudaGetSymbolAddress)
 *     with the caller's current device, so a cudaDeviceReset between calls is
 *     harmless; the first call on a device also loads the library's code
 *     there, so make that first call before any stream capture.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents (each call clears the one counter it starts from and writes
 *     every other scratch word before reading it).  Calls whose work overlaps
 *     on the GPU, from different streams or threads, race on it; serialise them.
 *   - It calls no allocation routine of any kind. */
#define KF_STATIC_MAX_HITS 262144
int kf_bin_hits_static(int32_t n_hits, const float *x, const float *y, const float *z, double half_len,
                       int32_t *perm_out, int32_t *offsets_out, float *packed_out, void *stream);

/* ---------------------------------------------------------------- building */

/* One binned layer of one event (device arrays made by kf_bin_hits). */
typedef struct {
    int32_t n_hits;
    int32_t surface;         /* index into the geometry (a barrel) */
    const float *packed;     /* [n_hits][4]: x, y, z, original index bits, binned order */
    const int32_t *offsets;  /* [KF_NBINS + 1] */
    const float *x;          /* [n_hits] original order (read by kf_gather_hits only; may be NULL otherwise) */
    const float *y;
    const float *z;
} kf_binned_layer;

typedef struct {
    double nsigma;    /* window half width in sigmas (3) */
    double chi2_cut;  /* accept the best hit only if chi2 < cut (30) */
    int32_t max_cand; /* candidates scored per step, in enumeration order (32), 1..64 */
    int32_t warp_coop;/* 1: score window candidates across the warp with a
                         shuffle min-reduction; 0: one thread per track
                         (KF_MEAS_HIT_2D always scores one thread per track) */
    double *debug_pred; /* diagnostics, NULL in normal use; kf_build_besthit only: device
                           [n_layers][27][n] FP64, for every build layer L >= 3 a track
                           reaches, its predicted state (6) and packed covariance (21)
                           after propagation and scattering noise, before its hit is
                           chosen (what its window and candidate scores were computed
                           from); entries of layers a track does not reach are left
                           as they are.  Lets a test replay one build decision. */
} kf_build_params;

/* Best-hit track building (Sec. 2: project the candidate outwards, use the KF
 * to pick the most likely continuation on each layer; here one candidate per
 * seed keeps the minimum-chi2 hit).  Tracks of several events run in one
 * launch (Sec. 4.2: several events processed together).  Per track: KF fit over its
 * three seed hits (layers 0..2 of the event), then for every later layer:
 * propagate, add scattering noise, open a window of +- nsigma in phi
 * (position and hit resolution) and z, enumerate the window's bins (z
 * ascending, phi ascending with wrap, binned order; at most max_cand hits),
 * chi2 of each candidate with the FP64 S solve, keep the smallest below
 * chi2_cut (ties: lower original index), update with it.
 *   n_events, n_layers: events and layers per event (all events share the
 *     layer list; n_layers <= KF_MAX_SURFACES).
 *   layers: host [n_events * n_layers] descriptors, event-major.
 *   event_offsets: host [n_events + 1], tracks of event e are
 *     event_offsets[e] .. event_offsets[e+1]-1 of the n = event_offsets[n_events]
 *     tracks.
 *   seeds: device, from kf_make_seeds over the three seed hits.
 *   seed_hits: device [9][n] FP32: x0, y0, z0, x1, y1, z1, x2, y2, z2.
 *   hit_idx_out: device [n_layers][n] int32: chosen original hit index per
 *     layer, -1 for none; the seed layers get -1 (the caller knows them).
 *   out: device fitted tracks after the last layer.
 * fit: host (precision, n_fp64_updates, seed_cov, ms_on are used). */
int kf_build_besthit(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *fit, const kf_build_params *bp,
                     int32_t n_events, int32_t n_layers, const kf_binned_layer *layers, const int32_t *event_offsets,
                     const kf_seeds *seeds, const float *seed_hits, int32_t *hit_idx_out, const kf_tracks_out *out,
                     void *stream);

/* Combinatorial track building (Sec. 2: building branches to explore several
 * candidates per seed; Sec. 4.3: a fixed number of candidate slots per seed,
 * the best candidates kept).  Each seed keeps at most n_slots candidates
 * (1, 2, 4 or 8), ranked.  After the seed fit, on every later layer each
 * candidate is propagated and scattered and its window searched as in
 * kf_build_besthit; its children are the candidate updated with each window
 * hit whose chi2 is below chi2_cut, and the candidate without a hit on this
 * layer (a candidate that cannot reach the layer stops and is carried
 * unchanged).  All children of a seed are ranked -- more hits first, then
 * smaller total chi2, then the lower rank of the parent, then the lower hit
 * index, a child without a hit after its parent's hits -- and the first
 * n_slots are kept.  After the last layer the first candidate is the track:
 * its hit per layer goes to hit_idx_out and its state to out.  With
 * n_slots = 1 this is best-hit building.  Mixed precision only
 * (fit->precision = KF_PREC_MIXED); other arguments as kf_build_besthit.
 * Scratch: about (140 + 5 * n_layers * n_slots) bytes per seed, in the
 * context's workspace. */
int kf_build_ckf(kf_ctx *ctx, const kf_geometry *geom, const kf_fit_params *fit, const kf_build_params *bp,
                 int32_t n_slots, int32_t n_events, int32_t n_layers, const kf_binned_layer *layers,
                 const int32_t *event_offsets, const kf_seeds *seeds, const float *seed_hits, int32_t *hit_idx_out,
                 const kf_tracks_out *out, void *stream);

/* Gather the hits a build chose into fit input (for the final fit, Sec. 2):
 * for each track, its three seed hits then every layer with hit_idx >= 0, in
 * layer order.  offsets_out: device [n+1]; layer_out, x_out, y_out, z_out:
 * device, capacity n * n_layers.  Arguments as in kf_build_besthit. */
int kf_gather_hits(kf_ctx *ctx, int32_t n_events, int32_t n_layers, const kf_binned_layer *layers,
                   const int32_t *event_offsets, const float *seed_hits, const int32_t *hit_idx, int32_t *offsets_out,
                   uint8_t *layer_out, float *x_out, float *y_out, float *z_out, void *stream);

/* ---------------------------------------------------------------- serving */

/* A serving loop over whole events (Sec. 4.2: several events in flight at a
 * time; Sec. 4.3: copies overlapped with processing).  Callers submit events
 * from host memory as they arrive; a dispatcher thread inside the library
 * admits queued events while the device memory of the batches in flight stays
 * under a budget, merges the admitted events (up to max_batch_events, arrival
 * order) into one batch and runs each batch on its own stream: copy in, bin
 * every build layer of every event in one segmented pass, seed, best-hit
 * build, gather, final fit, copy out.  Batches overlap one another on the
 * device.  Every track's arithmetic is that of kf_make_seeds, kf_bin_hits,
 * kf_build_besthit, kf_gather_hits and kf_fit (grid schedule), so an event's
 * results are bit-identical whatever it was batched with.
 * The server owns its threads, streams, a device memory pool and a
 * page-locked host staging arena; the context must outlive it. */
typedef struct kf_server kf_server;

typedef struct {
    size_t mem_budget_bytes;   /* device bytes the batches in flight may hold; 0 = 40 GiB */
    size_t host_staging_bytes; /* page-locked staging arena; 0 = 1 GiB */
    int32_t max_batches;       /* batches in flight (one stream each), 1..16; 0 = 4 */
    int32_t max_batch_events;  /* events merged into one batch, 1..64; 0 = 16 */
    kf_fit_params fit;         /* seed_cov == 0 selects the kf_fit defaults; schedule is ignored */
    kf_build_params build;     /* nsigma == 0 selects the kf_build_besthit defaults */
    double batch_window_ms;    /* a free stream waits until the oldest queued event is this
                                  old (or max_batch_events are queued) before it starts a
                                  batch: larger batches for some latency; 0 = start at once */
} kf_server_params;

/* One event, all host memory.
 *   n_tracks > 0 seeds; n_layers 4..KF_MAX_SURFACES, all barrels; the first
 *   three layers are the seed layers.
 *   surface [n_layers]: geometry index of each layer.
 *   n_hits [n_layers]: hits of each layer (layers 0..2 are not read).
 *   x, y, z [n_layers]: per layer, a host array of n_hits[l] FP32 coordinates
 *     (layers 0..2 are not read and may be NULL).
 *   seed_hits [n_tracks][3][3]: hit k of track t, (x, y, z) at 9t + 3k.
 *   flags: 0 = the coordinate and seed-hit arrays are copied into the staging
 *     arena before kf_server_submit returns; KF_EVENT_ZERO_COPY = the caller
 *     keeps them unchanged until the ticket completes and the kernels read them
 *     in place (any host memory on a GPU that reads pageable memory, such as a
 *     Grace-Blackwell board; elsewhere page-locked memory, else they are copied;
 *     an array not at a multiple of 4 bytes is copied as well).
 * The small arrays (surface, n_hits and the x, y, z pointer arrays) are read
 * during the call only. */
#define KF_EVENT_ZERO_COPY 1
typedef struct {
    int32_t n_tracks;
    int32_t n_layers;
    const int32_t *surface;
    const int32_t *n_hits;
    const float *const *x;
    const float *const *y;
    const float *const *z;
    const float *seed_hits;
    int32_t flags;
    int32_t pad_;
} kf_event;

/* Where an event's results go: host arrays the caller keeps alive until the
 * ticket has completed.  A kernel writes them in place when all of them are
 * page-locked and each sits at a multiple of its element size (4 bytes for
 * the int32 arrays, 8 for the doubles); otherwise the dispatcher thread copies
 * them from the server's staging (a GPU write into pageable memory pulls every
 * fresh page through the host, and a misaligned store would fault).  Any may
 * be NULL.
 *   hit_idx [n_layers][n_tracks]: as kf_build_besthit's hit_idx_out.
 *   state [6][n_tracks], cov [21][n_tracks], chi2, ndof: final fit over the
 *     seed hits and the chosen hits, as kf_fit.
 *   status [n_tracks]: build status | final-fit status (KF_ST_* bits). */
typedef struct {
    int32_t *hit_idx;
    double *state;
    double *cov;
    double *chi2;
    int32_t *ndof;
    uint32_t *status;
} kf_event_result;

typedef struct {
    uint64_t submitted, completed, rejected, batches;
    int32_t queued;             /* events waiting for admission */
    int32_t in_flight_events;
    int32_t in_flight_batches;
    int32_t pad_;
    size_t bytes_in_use;        /* device bytes reserved by the batches in flight */
    size_t peak_bytes_in_use;   /* maximum of bytes_in_use (never above the budget) */
    double mean_batch_events;
    double p50_ms, p99_ms, max_ms, mean_ms; /* submit -> results in the caller's arrays */
    double events_per_s, tracks_per_s;      /* completed since the last reset */
    double batch_device_ms;    /* mean time of a batch on its stream, first copy in to last copy out */
    double copy_out_ms;        /* mean host time per batch copying results into callers' arrays */
    double stage_ms;           /* mean host time per event staging its hits in kf_server_submit */
} kf_server_stats;

/* Start a server on the context's device.  params: host, NULL = defaults.
 * Returns KF_EINVAL (bad geometry or parameters), KF_ENOMEM (pool or staging
 * arena), KF_ECUDA. */
int kf_server_create(kf_ctx *ctx, const kf_geometry *geom, const kf_server_params *params, kf_server **out);

/* Queue one event; *ticket receives its id.  Thread-safe.  Returns KF_EBUSY
 * (and counts a rejection) when the event alone needs more device memory than
 * the budget or more staging than the whole arena, KF_EAGAIN when the staging
 * arena is full for now (retry after earlier events complete), KF_EINVAL for
 * a malformed event. */
int kf_server_submit(kf_server *s, const kf_event *ev, const kf_event_result *res, uint64_t *ticket);

/* KF_EAGAIN while the ticket is queued or in flight; then, once, its result
 * code (KF_OK, or KF_ENOMEM / KF_ECUDA if it could not run) with the latency in
 * *latency_ms (may be NULL); KF_EINVAL for an unknown or already reported ticket. */
int kf_server_poll(kf_server *s, uint64_t ticket, double *latency_ms);

/* kf_server_poll that blocks up to timeout_ms; KF_ETIMEOUT when it runs out. */
int kf_server_wait(kf_server *s, uint64_t ticket, double timeout_ms, double *latency_ms);

/* Counters and latency percentiles of the events completed since the last
 * reset; reset != 0 starts a new window.  Returns KF_ECUDA if a CUDA error
 * has been seen (the counters are still filled). */
int kf_server_stats_get(kf_server *s, kf_server_stats *out, int reset);

/* Finish the batches in flight, drop queued events, free everything.  NULL is
 * accepted. */
void kf_server_destroy(kf_server *s);

/* ---------------------------------------------------------------- measurement */

/* Layout study (Sec. 4.3: the paper timed batched 6x6 products on a GPU for
 * several memory layouts).  One launch of the covariance transport
 * P' = J P J^T for n matrices, one per thread, operands in registers, FP32,
 * with J (36 entries, row-major), P and P' (21 packed lower-triangle entries)
 * stored in the given layout:
 *   KF_LAYOUT_AOS    element k of matrix t at t * K + k;
 *   KF_LAYOUT_SOA    at k * n + t (the layout of this library's kernels);
 *   KF_LAYOUT_BLOCK  Matriplex-like blocks of 32: ((t / 32) * K + k) * 32 + t % 32
 *                    (n a multiple of 32).
 * J, P, P_out: device arrays of n * 36, n * 21, n * 21 floats.  Asynchronous
 * on the stream; time it with events around the call. */
#define KF_LAYOUT_AOS 0
#define KF_LAYOUT_SOA 1
#define KF_LAYOUT_BLOCK 2
int kf_layout_transport(kf_ctx *ctx, int32_t layout, int32_t n, const float *J, const float *P, float *P_out,
                        void *stream);

/* Peak arithmetic rate of this GPU, measured (no counterpart in the paper; it
 * gives the roofline denominators of the fit): a grid of several blocks per SM
 * runs eight independent fused multiply-add chains per thread in FP64
 * (which = 0) or FP32 (which = 1); *flops_per_s receives 2 * FMAs / elapsed.
 * Synchronous; uses the context's device and a scratch buffer of the context. */
int kf_measure_peak(kf_ctx *ctx, int which, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* KF_H */
