// kf_internal.h -- host-side declarations shared by the translation units of libkf.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kf_common.cuh"

namespace kfd {

// A track handed from phase 1 of the mixed fit to phase 2, at its processing
// position i ([k][m] planes): state as float-float (x, y, z, phi, theta; hi then
// lo) and 1/pT, the FP32 covariance, chi2, the next hit k (-1: finished in
// phase 1), hits used, status.
struct FitCarry {
    float *st;       // [11][m]
    float *cov;      // [21][m]
    double *chi2;    // [m]
    int32_t *k;      // [m]
    int32_t *used;   // [m]
    uint32_t *status;
    int m;
    int pad_;
};
size_t fit_carry_bytes(int m);
void fit_carve_carry(FitCarry &c, void *p, int m);

struct FitArgs {
    int n;            // plane stride of seeds and outputs ([k][n] arrays)
    int t_begin;      // first track of this launch
    int count;        // tracks in this launch (t_begin .. t_begin + count - 1)
    int n64;          // updates carried in FP64 (Joseph form) from the seed
    double seed_cov;
    int ms_on;
    int seed_df;      // mixed path: the first n64 updates in double-float, U-D form (else FP64 Joseph)
    const float *seed_state;  // [6][n]
    const int8_t *q;          // [n]
    const int32_t *off;       // [n+1]
    const uint8_t *layer;
    const float *hx, *hy, *hz;
    double *o_state;   // [6][n]
    double *o_cov;     // [21][n]
    float *o_cov32;    // [21][n] FP32 copy of the covariance, or null
    double *o_chi2;
    int32_t *o_ndof;
    uint32_t *o_status;
    // persistent schedule
    const int32_t *order;  // processing order (tracks sorted by hit count), or null
    int32_t *queue;        // work counter, zeroed before the launch
    int chunk;             // tracks per thread per queue grab (a block takes blockDim * chunk)
    int meas_model;        // 0: 3-D hit on the layer; 1: barrel hits on their own cylinder, 2-D (grid schedule)
    // initial covariance: p0_scale * p0 ([21][n] FP64) instead of seed_cov * I when p0 is set
    const double *p0;
    double p0_scale;
    // the mixed fit (not the refit): phase 1 -> phase 2 hand-over, m >= count
    FitCarry carry;
    // host side only: null, or three cudaEvent_t recorded before phase 1, between the
    // phases and after phase 2 (launch_fit; the one-kernel forms record the second
    // and third together)
    void *timing_events;
};

// kf_fit.cu
cudaError_t launch_seeds(const Geom &g, int count, int stride, int t_begin, const int32_t *off, const float *hx,
                         const float *hy, const float *hz, float *state, int8_t *q, cudaStream_t st);
cudaError_t launch_fit(const Geom &g, const FitArgs &a, bool fp64, int block, cudaStream_t st);
cudaError_t launch_fit_persistent(const Geom &g, const FitArgs &a, bool fp64, int block, int grid, cudaStream_t st);
int persistent_blocks_per_sm(bool fp64, int block);
size_t order_scratch_ints();
// processing order: tracks bucketed by (hit count, a disk among the first nseed
// hits' surfaces -- needs off, layer and g --, seed 1/pT, and for geometries with
// disks the seed theta of the stiff tracks); off null: by 1/pT alone
cudaError_t launch_order(int n, const int32_t *off, const float *seed_ip, const float *seed_th, const uint8_t *layer,
                         const Geom *g, int nseed, int32_t *hist, int32_t *order, cudaStream_t st);

// outward-inward refit (kf_fit.cu): cnt[t] = hits the forward fit used, then
// (after an exclusive scan of cnt into roff) those hits reversed into roff's CSR
cudaError_t launch_used_counts(int n, const int32_t *off, const int32_t *fwd_ndof, int32_t *cnt, cudaStream_t st);
cudaError_t launch_reverse(int n, const int32_t *off, const int32_t *roff, const uint8_t *layer, const float *x,
                           const float *y, const float *z, const double *fwd, const double *fwd_cov, const int8_t *q,
                           uint8_t *rl, float *rx, float *ry, float *rz, float *seed, double *rcov, int8_t *rq,
                           cudaStream_t st);
// exclusive scan of n counts into off_out[0..n] (kf_build.cu); bsum: n / 1024 + 2 ints
cudaError_t launch_scan_counts(int n, const int32_t *cnt, int32_t *off_out, int32_t *bsum, cudaStream_t st);
cudaError_t launch_unreverse(int n, double *state, double *cov, float *cov32, cudaStream_t st);

// kf_bin.cu
size_t bin_scratch_bytes(int n_hits);
cudaError_t launch_bin(int n_hits, const float *x, const float *y, const float *z, double half_len, int32_t *perm,
                       int32_t *offsets, float *packed, void *scratch, cudaStream_t st);

size_t bin_segments_scratch_bytes(int H, int nseg);
cudaError_t launch_bin_segments(int nseg, int H, const int32_t *seg_off, const double *half, const float *x,
                                const float *y, const float *z, int32_t *perm, int32_t *offsets, float *packed,
                                void *scratch, cudaStream_t st);

// kf_build.cu
struct LayerDev {
    const float4 *packed;
    const int32_t *offsets;
    const float *x, *y, *z;  // original order
    int n_hits;
    int surface;
};
struct BuildArgs {
    int n;
    int n_events;
    int n_layers;
    int n64;
    double seed_cov;
    int ms_on;
    int max_cand;
    float nsigma;
    float chi2_cut;
    const LayerDev *layers;       // device [n_events][n_layers]
    const int32_t *event_off;     // device [n_events + 1]
    const float *seed_state;      // [6][n]
    const int8_t *q;
    const float *seed_hits;       // [9][n]
    int32_t *hit_idx;             // [n_layers][n]
    const int32_t *order;         // processing order (by seed 1/pT), or null
    double *o_state, *o_cov, *o_chi2;
    float *o_cov32;  // [21][n] FP32 copy of the covariance, or null
    int32_t *o_ndof;
    uint32_t *o_status;
    int meas_model;  // as FitArgs::meas_model (per-thread scoring only)
    int seed_df;     // as FitArgs::seed_df
    // mixed path: device scratch of build_seed_scratch_bytes(n) bytes, where a
    // pre-pass kernel leaves each track's seed fit for the layer kernel
    void *seed_scratch;
    // diagnostics (kf_build_params.debug_pred): [n_layers][27][n] predicted
    // state and covariance per build step, or null
    double *dbg_pred;
};
size_t build_seed_scratch_bytes(int n);
cudaError_t launch_build(const Geom &g, const BuildArgs &a, bool fp64, bool warp_coop, cudaStream_t st);

// Combinatorial building: n_slots candidates per seed (mixed precision).  The
// seed fit runs first, one thread per seed, into the seed_* arrays; then
// n_slots lanes of a warp carry one seed's candidates through the layers,
// leaving back pointers (parent slot, hit) per layer and slot.
struct CkfArgs {
    BuildArgs b;
    int n_slots;
    int pad_;
    float *seed_st;        // [11][n]: x, y, z, phi, theta as float-float (hi, lo), then 1/pT
    float *seed_cov;       // [21][n]
    double *seed_chi2;     // [n]
    int32_t *seed_used;    // [n]
    uint32_t *seed_status; // [n]
    int8_t *seed_alive;    // [n]
    int8_t *bp_parent;     // [n_layers][n * n_slots]
    int32_t *bp_hit;       // [n_layers][n * n_slots]
};
size_t ckf_scratch_bytes(int n, int n_layers, int n_slots);
void ckf_carve(CkfArgs &c, void *scratch, int n, int n_layers, int n_slots);
cudaError_t launch_ckf(const Geom &g, const CkfArgs &c, cudaStream_t st);
size_t gather_scratch_bytes(int n);
cudaError_t launch_gather(int n, int n_events, int n_layers, const LayerDev *layers, const int32_t *event_off,
                          const float *seed_hits, const int32_t *hit_idx, int32_t *off_out, uint8_t *layer_out,
                          float *x_out, float *y_out, float *z_out, void *scratch, cudaStream_t st);

// kf_layout.cu
cudaError_t launch_transport_layout(int layout, int n, const float *J, const float *P, float *Po, cudaStream_t st);

// kf_peak.cu
cudaError_t measure_peak(int which, int sm_count, void *scratch, double *flops_per_s);

// kf_api.cu: context services used by the serving runtime
int ctx_geom(kf_ctx *ctx, const kf_geometry *g, Geom &G);
int ctx_fit_params(kf_ctx *ctx, const kf_fit_params *p, kf_fit_params &q);
int ctx_device(const kf_ctx *ctx);
int ctx_fail(kf_ctx *ctx, int code, const char *msg);

}  // namespace kfd
