// kf_build.cu -- best-hit track building (Sec. 2: track building projects the
// candidate outwards and uses the KF to pick the most likely continuation on
// each layer; this variant keeps one candidate per seed, the minimum-chi2 hit).
//
// Tracks of several events run in one launch (Sec. 4.2: several events at a
// time fill the machine).  Per track: KF fit over its three seed hits (FP64,
// Joseph form), then for every later layer propagate, add scattering noise,
// open a +-nsigma window in (phi, z), score the window's hits, update with
// the best one.  A window row (one z bin, a run of phi bins) is one or two
// contiguous ranges of the layer's binned hits, read as 16-byte (x, y, z,
// index) records.
//
// Two scoring schemes:
//   per-thread: each thread walks its own window;
//   warp-cooperative: the 32 tracks of a warp pool their candidates; every lane
//     scores one (track, candidate) pair per round and a shuffle reduction
//     picks each track's minimum, so a warp costs ceil(total/32) rounds
//     instead of max-over-lanes candidates.
#include "kf_internal.h"
#include "kf_df.cuh"
#include "kf_track.cuh"

namespace kfd {

__device__ __forceinline__ int find_event(const int32_t *__restrict__ eoff, int n_events, int t)
{
    int lo = 0, hi = n_events - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Window of a predicted state on a barrel layer (a reading: +- nsigma in the
// azimuth of the predicted position, with its variance from P and the hit
// resolution, and in z).
struct Window {
    int phi_lo;  // first phi bin, in [0, 1024)
    int nphi;    // number of phi bins, <= 1024
    int z_lo, z_hi;
};

//
// dr > 0 (model 1, hits within +-dr of the layer radius): the window widens by
// the azimuth and z the track sweeps over dr, dr tan(a) / R and dr |cot theta| /
// cos(a) with a the angle between the track and the radial direction; the whole
// layer when the track runs nearly along the layer (cos(a) <= 1e-3).
template <class T, class P>
__device__ __forceinline__ Window make_window(const Track<T, P> &st, const float p[21], const Surf &sf, float nsig,
                                              float dr = 0.f)
{
    const float X = (float)lead(st.x), Y = (float)lead(st.y), Z = (float)lead(st.z);
    const float r2 = X * X + Y * Y;
    const float phip = atan2f(Y, X);
    const float sphi2 = (Y * Y * p[pk(0, 0)] + X * X * p[pk(1, 1)] - 2.f * X * Y * p[pk(1, 0)]) / (r2 * r2);
    const float R = sf.pos;
    float dphi = nsig * sqrtf(fmaxf(sphi2, 0.f) + sf.var_rphi / (R * R));
    float dz = nsig * sqrtf(fmaxf(p[pk(2, 2)], 0.f) + sf.var_zz);
    if (dr > 0.f) {
        float sd, cd, sth, cth;
        sincosf((float)lead(st.phi) - phip, &sd, &cd);
        sincosf((float)lead(st.th), &sth, &cth);
        const float ca = fabsf(cd), sa = fabsf(sd);
        if (ca > 1e-3f) {
            dphi += dr * sa / (ca * R);
            dz += dr * fabsf(cth / sth) / ca;
        } else {
            dphi = PI_F;
            dz = 2.f * sf.half;
        }
    }
    const float kphi = 1024.f / (2.f * PI_F);
    Window w;
    if (!(dphi < PI_F) || !(fabsf(phip) <= 2.f * PI_F)) {
        // the whole ring (also for a non-finite prediction)
        w.nphi = KF_NPHI;
        w.phi_lo = 0;
    } else {
        const int lo = (int)floorf((phip - dphi + PI_F) * kphi);  // within [-1024, 2048]
        const int hi = (int)floorf((phip + dphi + PI_F) * kphi);
        w.nphi = max(0, min(hi - lo + 1, KF_NPHI));
        w.phi_lo = ((lo % KF_NPHI) + KF_NPHI) % KF_NPHI;
    }
    const float L = sf.half;
    const float kz = 64.f / (2.f * L);
    const float zl = fminf(fmaxf(floorf((Z - dz + L) * kz), 0.f), (float)(KF_NZ - 1));
    const float zh = fminf(fmaxf(floorf((Z + dz + L) * kz), 0.f), (float)(KF_NZ - 1));
    w.z_lo = zl == zl ? (int)zl : 0;  // NaN -> 0
    w.z_hi = zh == zh ? (int)zh : KF_NZ - 1;
    return w;
}

// chi2 of one candidate against the predicted state; S shared (f) when the hit
// covariance does not depend on the hit azimuth, else built for this hit.
template <class T, class P>
__device__ __forceinline__ double cand_chi2(const Track<T, P> &st, const float p[21], const Surf &sf, bool shared,
                                            const Ldl3 &f, float4 h)
{
    const auto r0 = resid(h.x, st.x), r1 = resid(h.y, st.y), r2 = resid(h.z, st.z);
    if (shared) return ldl3_chi2(f, wide(r0), wide(r1), wide(r2));
    float rxx, rxy, ryy, rzz;
    meas_cov<float>(sf, h.x, h.y, rxx, rxy, ryy, rzz);
    Ldl3 g;
    if (!ldl3<false>(wide(p[pk(0, 0)] + rxx), wide(p[pk(1, 0)] + rxy), wide(p[pk(1, 1)] + ryy), wide(p[pk(2, 0)]),
              wide(p[pk(2, 1)]), wide(p[pk(2, 2)] + rzz), g))
        return -1.0;
    return ldl3_chi2(g, wide(r0), wide(r1), wide(r2));
}

// chi2 of one candidate under model 1: the predicted state (on the layer's
// average cylinder) carried on to the cylinder through the hit, with the
// position block of its covariance, and the 2-D chi2 there; -1 when the hit's
// cylinder is out of reach or S is not positive definite.
template <class T, class P, class C>
__device__ __forceinline__ double cand_chi2_m1(const Track<T, P> &st, const Dir<T> &dir, const C pc[21],
                                               const Surf &sf, T alpha, float4 h)
{
    const Surf hs = hit_surface(sf, h.x, h.y);
    Track<T, P> s2 = st;
    Jac<T> J;
    if (!propagate_from(s2, alpha, hs, J, dir)) return -1.0;
    C q[6];
    transport_pos<C>(pc, JacAs<C>::get(J), q);
    return kf_chi2_2d(s2, q, h.x, h.y, h.z, hs);
}

template <bool FP64> struct sel_t;
template <> struct sel_t<true> { using T = double; using P = double; };
template <> struct sel_t<false> { using T = float; using P = ff; };

// Result of one layer step of one track.
struct StepOut {
    int chosen;     // original hit index or -1
    bool capped;
};

// Per-thread scoring: walk the window's rows (z ascending, phi from the low edge
// with wrap, binned order), at most max_cand candidates.
// M1: each candidate scored by cand_chi2_m1 (pc, alpha) instead of cand_chi2.
template <bool M1, class T, class P, class C>
__device__ __forceinline__ void score_own(const Track<T, P> &st, const float pw[21], const C pc[21], T alpha,
                                          const Surf &sf, const LayerDev &ly, const Window &w, bool shared,
                                          const Ldl3 &fs, int max_cand, int &best, double &bchi, float4 &bhit,
                                          bool &capped)
{
    int ncand = 0;
    Dir<T> dir;
    if constexpr (M1) dir = direction(st);  // shared by the candidates' second steps
    // A screen in FP32 before each candidate's FP64 chi2 (mixed path, shared S):
    // the same forward substitution with the factor rounded to FP32.  A candidate
    // whose FP32 chi2 exceeds the best FP64 chi2 so far by more than 1% cannot
    // become the best (the FP32 value is within ~1e-6 relative of the FP64 one),
    // so its FP64 chi2 is not needed; every decision is still taken on FP64
    // values, and the choice is the one the full FP64 scan makes.
    constexpr bool SCREEN = !M1 && sizeof(T) == 4;
    float sl21 = 0.f, sl31 = 0.f, sl32 = 0.f, si1 = 0.f, si2 = 0.f, si3 = 0.f;
    if constexpr (SCREEN) {
        if (shared) {
            sl21 = d2f(fs.l21);
            sl31 = d2f(fs.l31);
            sl32 = d2f(fs.l32);
            si1 = d2f(fs.i1);
            si2 = d2f(fs.i2);
            si3 = d2f(fs.i3);
        }
    }
    for (int zb = w.z_lo; zb <= w.z_hi && !capped; ++zb) {
        const int row = zb * KF_NPHI;
        const int first = w.phi_lo, last = w.phi_lo + w.nphi - 1;
        for (int part = 0; part < 2 && !capped; ++part) {
            int b0, b1;  // bin range [b0, b1] in this row
            if (part == 0) {
                b0 = first;
                b1 = min(last, KF_NPHI - 1);
            } else {
                if (last < KF_NPHI) break;
                b0 = 0;
                b1 = last - KF_NPHI;
            }
            const int j0 = max(ly.offsets[row + b0], 0), j1 = min(ly.offsets[row + b1 + 1], ly.n_hits);
            for (int j = j0; j < j1; ++j) {
                if (ncand >= max_cand) {
                    capped = true;
                    break;
                }
                ++ncand;
                const float4 h = ly.packed[j];
                if constexpr (SCREEN) {
                    if (shared && best >= 0) {
                        const float r0 = resid(h.x, st.x), r1 = resid(h.y, st.y), r2 = resid(h.z, st.z);
                        const float z2 = fmaf(-sl21, r0, r1), z3 = fmaf(-sl32, z2, fmaf(-sl31, r0, r2));
                        const float c32 = fmaf(z3 * si3, z3, fmaf(z2 * si2, z2, r0 * si1 * r0));
                        if (c32 > (float)bchi * 1.01f + 1e-4f) continue;
                    }
                }
                double c2;
                if constexpr (M1) c2 = cand_chi2_m1(st, dir, pc, sf, alpha, h);
                else c2 = cand_chi2(st, pw, sf, shared, fs, h);
                const int hi = __float_as_int(h.w);
                if (c2 >= 0.0 && (best < 0 || c2 < bchi || (c2 == bchi && hi < best))) {
                    best = hi;
                    bchi = c2;
                    bhit = h;
                }
            }
        }
    }
}

// shared S factor (hit covariance independent of the hit azimuth)
template <class C>
__device__ __forceinline__ bool shared_factor(const C pc[21], const Surf &sf, Ldl3 &fs)
{
    const C vr = sizeof(C) == 8 ? (C)sf.var_radd : (C)sf.var_rad;
    const C vz = sizeof(C) == 8 ? (C)sf.var_zzd : (C)sf.var_zz;
    // float -> double by bit operations (wide): a conversion instruction would take an FP64 issue slot
    return ldl3<sizeof(C) == 8>(wide(C(pc[pk(0, 0)] + vr)), wide(pc[pk(1, 0)]), wide(C(pc[pk(1, 1)] + vr)), wide(pc[pk(2, 0)]),
                wide(pc[pk(2, 1)]), wide(C(pc[pk(2, 2)] + vz)), fs);
}

// The build parameters a layer step reads.
struct StepKnobs {
    int ms_on;
    int max_cand;
    float nsigma;
    float chi2_cut;
    double *dbg;     // diagnostics: this (layer, track)'s predicted state and covariance, or null
    int dbg_stride;  // planes of dbg are dbg_stride doubles apart
};

// the predicted state (6) and covariance (21) of a build step, before the hit is
// chosen (kf_build_params.debug_pred)
template <class T, class P, class C>
__device__ __forceinline__ void debug_pred_put(const StepKnobs &a, const Track<T, P> &st, const C pc[21])
{
    if (!a.dbg) return;
    const double sv[6] = {to_d(st.x), to_d(st.y), to_d(st.z), (double)st.ip, to_d(st.phi), to_d(st.th)};
    for (int i = 0; i < 6; ++i) a.dbg[(size_t)i * a.dbg_stride] = sv[i];
    for (int i = 0; i < 21; ++i) a.dbg[(size_t)(6 + i) * a.dbg_stride] = (double)pc[i];
}

// One build layer for one track with per-thread scoring: propagate, transport,
// scattering noise, window, candidates, update.  JOSEPH selects the covariance
// update form (the FP64 steps).
//
// M1 (measurement model 1, Sec. 4.1, barrel layers): two propagation steps, to
// the layer's average cylinder (scattering noise and the window, widened by
// the layer's dr, there), then from there to each candidate's own cylinder,
// where it is scored in 2-D; the chosen hit is reached the same way and the
// 2-D update made on its cylinder.
template <bool JOSEPH, bool M1, class T, class P, class C>
__device__ __forceinline__ StepOut layer_step_thread(Track<T, P> &st, C pc[21], T alpha, T mass2, const StepKnobs &a,
                                                     const Surf &sf, const LayerDev &ly, double &chi2,
                                                     unsigned &status, bool &alive)
{
    StepOut o{-1, false};
    Jac<T> J;
    if (!propagate(st, alpha, sf, J)) {
        status |= reach_bits(st);
        alive = false;
        return o;
    }
    transport<C>(pc, JacAs<C>::get(J));
    if (a.ms_on) status |= ms_noise<T, C>(st, sf, J.cphi1, J.sphi1, mass2, pc);
    debug_pred_put(a, st, pc);
    float pw[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pw[i] = (float)pc[i];
    int best = -1;
    double bchi = 0.0;
    float4 bhit = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (M1) {
        if (sf.kind == 0) {
            const Window w = make_window(st, pw, sf, a.nsigma, sf.dr);
            const Ldl3 none{0, 0, 0, 0, 0, 0};
            score_own<true>(st, pw, pc, alpha, sf, ly, w, false, none, a.max_cand, best, bchi, bhit, o.capped);
            if (best >= 0 && bchi < (double)a.chi2_cut) {
                const Surf hs = hit_surface(sf, bhit.x, bhit.y);
                Jac<T> J;
                bool ok = propagate(st, alpha, hs, J);
                if (ok) {
                    transport<C>(pc, JacAs<C>::get(J));
                    if constexpr (JOSEPH) ok = kf_update2d<true>(st, pc, bhit.x, bhit.y, bhit.z, hs, chi2);
                    else ok = kf_update2d_mixed(st, pc, bhit.x, bhit.y, bhit.z, hs, chi2);
                }
                if (ok) {
                    o.chosen = best;
                } else {
                    status |= KF_ST_CHOL_FAIL;
                    alive = false;
                }
            }
            return o;
        }
    }
    const Window w = make_window(st, pw, sf, a.nsigma);
    const bool shared = sf.var_rad == sf.var_rphi;
    Ldl3 fs{0, 0, 0, 0, 0, 0};
    if (shared && !shared_factor(pc, sf, fs)) {
        status |= KF_ST_CHOL_FAIL;
        alive = false;
        return o;
    }
    score_own<false>(st, pw, pc, alpha, sf, ly, w, shared, fs, a.max_cand, best, bchi, bhit, o.capped);
    if (best >= 0 && bchi < (double)a.chi2_cut) {
        bool ok;
        if constexpr (JOSEPH) {
            ok = kf_update<true>(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2);
        } else if constexpr (sizeof(C) == 4) {  // mixed path: reuse the window's S factor
            ok = shared ? kf_update_mixed_factored(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2, fs, bchi)
                        : kf_update_mixed(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2);
        } else {
            ok = kf_update_mixed(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2);
        }
        if (ok) {
            o.chosen = best;
        } else {
            status |= KF_ST_CHOL_FAIL;
            alive = false;
        }
    }
    return o;
}

// FP64 layer step for a mixed-path track at a near-tangent crossing
template <bool M1>
__device__ __forceinline__ StepOut layer_step_fp64(Track<float, ff> &st, float pc[21], double alpha, double mass2,
                                                   const StepKnobs &a, const Surf &sf, const LayerDev &ly,
                                                   double &chi2, unsigned &status, bool &alive)
{
    Track<double, double> sd;
    sd.x = to_d(st.x);
    sd.y = to_d(st.y);
    sd.z = to_d(st.z);
    sd.phi = to_d(st.phi);
    sd.th = to_d(st.th);
    sd.ip = st.ip;
    double pd[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pd[i] = pc[i];
    const StepOut o = layer_step_thread<true, M1>(sd, pd, alpha, mass2, a, sf, ly, chi2, status, alive);
    if (alive) {
        auto f = [](double d) {
            float h = (float)d;
            return ff{h, (float)(d - (double)h)};
        };
        st.x = f(sd.x);
        st.y = f(sd.y);
        st.z = f(sd.z);
        st.phi = f(sd.phi);
        st.th = f(sd.th);
        st.ip = (float)sd.ip;
#pragma unroll
        for (int i = 0; i < 21; ++i) pc[i] = (float)pd[i];
    }
    return o;
}

// layer_step_fp64 out of line, so that the FP32 layer loop stays compact in
// the instruction cache (about 2% of the steps are near-tangent)
struct Fp64LayerIO {
    MixedIO m;
    StepOut o;
    int alive;
};
template <bool M1>
static __device__ __noinline__ Fp64LayerIO layer_step_fp64_out_of_line(Fp64LayerIO io, double alpha, double mass2,
                                                                       StepKnobs kn, const Surf *sf, LayerDev ly)
{
    bool alive = io.alive != 0;
    io.o = layer_step_fp64<M1>(io.m.st, io.m.p, alpha, mass2, kn, *sf, ly, io.m.chi2, io.m.status, alive);
    io.alive = alive;
    return io;
}

// A near-tangent layer step of the mixed build under measurement model 0: FP32
// propagation; the transport and the scattering noise in double-float (the
// Jacobian grows like 1 / cos(alpha) and FP32 arithmetic cannot carry the
// transport); window and candidate scores from that covariance rounded to FP32,
// as in layer_step_thread; the update with the chosen hit in double-float U-D
// form (kf_df.cuh).
__device__ __forceinline__ StepOut layer_step_df(Track<float, ff> &st, float pc[21], float alpha, float mass2,
                                                 const StepKnobs &a, const Surf &sf, const LayerDev &ly,
                                                 double &chi2, unsigned &status, bool &alive)
{
    StepOut o{-1, false};
    Jac<float> J;
    if (!propagate(st, alpha, sf, J)) {
        status |= reach_bits(st);
        alive = false;
        return o;
    }
    df p[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) p[i] = df(pc[i]);
    transport<df>(p, J);
    if (a.ms_on) status |= ms_noise<float, df>(st, sf, J.cphi1, J.sphi1, mass2, p);
    float pw[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pw[i] = p[i].hi;
    debug_pred_put(a, st, pw);
    const Window w = make_window(st, pw, sf, a.nsigma);
    const bool shared = sf.var_rad == sf.var_rphi;
    Ldl3 fs{0, 0, 0, 0, 0, 0};
    if (shared && !shared_factor(pw, sf, fs)) {
        status |= KF_ST_CHOL_FAIL;
        alive = false;
        return o;
    }
    int best = -1;
    double bchi = 0.0;
    float4 bhit = make_float4(0.f, 0.f, 0.f, 0.f);
    score_own<false>(st, pw, pw, alpha, sf, ly, w, shared, fs, a.max_cand, best, bchi, bhit, o.capped);
    if (best >= 0 && bchi < (double)a.chi2_cut) {
        df c2 = df(0.f);
        if (ud_update3(st, p, bhit.x, bhit.y, bhit.z, sf, c2)) {
            chi2 += df_to_d(c2);
            o.chosen = best;
        } else {
            status |= KF_ST_CHOL_FAIL;
            alive = false;
        }
    }
#pragma unroll
    for (int i = 0; i < 21; ++i) pc[i] = p[i].hi;
    return o;
}
static __device__ __noinline__ Fp64LayerIO layer_step_df_out_of_line(Fp64LayerIO io, float alpha, float mass2,
                                                                     StepKnobs kn, const Surf *sf, LayerDev ly)
{
    bool alive = io.alive != 0;
    io.o = layer_step_df(io.m.st, io.m.p, alpha, mass2, kn, *sf, ly, io.m.chi2, io.m.status, alive);
    io.alive = alive;
    return io;
}

// Warp-cooperative scoring of one layer: every lane of the warp calls it; lanes
// with do_step == false contribute no candidates.  Lanes list their window's
// candidates as consecutive items of one warp-wide list; each round every lane
// scores one item for the item's owner (predicted position and S factor come by
// shuffle) and each owner folds its items' chi2 into its best by shuffles.
template <class T, class P>
__device__ __forceinline__ void score_coop(const Track<T, P> &st, bool do_step, const Window &w, const Ldl3 &fs,
                                           const LayerDev &ly, int max_cand, int &best, double &bchi, float4 &bhit,
                                           bool &capped)
{
    const int lane = threadIdx.x & 31;
    int my_total = 0;
    if (do_step) {
        for (int zb = w.z_lo; zb <= w.z_hi; ++zb) {
            const int row = zb * KF_NPHI;
            const int first = w.phi_lo, last = w.phi_lo + w.nphi - 1;
            my_total += ly.offsets[row + min(last, KF_NPHI - 1) + 1] - ly.offsets[row + first];
            if (last >= KF_NPHI) my_total += ly.offsets[row + (last - KF_NPHI) + 1] - ly.offsets[row];
        }
        my_total = max(my_total, 0);
        if (my_total > max_cand) {
            capped = true;
            my_total = max_cand;
        }
    }
    int pre = my_total;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, pre, d);
        if (lane >= d) pre += o;
    }
    const int warp_total = __shfl_sync(0xffffffffu, pre, 31);
    pre -= my_total;
    const float Xh = (float)lead(st.x), Yh = (float)lead(st.y), Zh = (float)lead(st.z);
    const float Xl = (float)lo_part(st.x), Yl = (float)lo_part(st.y), Zl = (float)lo_part(st.z);
    for (int r0 = 0; r0 < warp_total; r0 += 32) {
        const int item = r0 + lane;
        // owner: the last lane whose first item is <= item
        int owner = 0;
#pragma unroll
        for (int d = 0; d < 32; ++d) {
            const int pd_ = __shfl_sync(0xffffffffu, pre, d);
            if (pd_ <= item) owner = d;
        }
        const int opre = __shfl_sync(0xffffffffu, pre, owner);
        const int ozlo = __shfl_sync(0xffffffffu, w.z_lo, owner);
        const int ozhi = __shfl_sync(0xffffffffu, w.z_hi, owner);
        const int oplo = __shfl_sync(0xffffffffu, w.phi_lo, owner);
        const int onph = __shfl_sync(0xffffffffu, w.nphi, owner);
        // the owner's layer: lanes of one warp can belong to different events
        const int32_t *ooff = reinterpret_cast<const int32_t *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(ly.offsets), owner));
        const float4 *opk = reinterpret_cast<const float4 *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(ly.packed), owner));
        const int onh = __shfl_sync(0xffffffffu, ly.n_hits, owner);
        const float oXh = __shfl_sync(0xffffffffu, Xh, owner), oYh = __shfl_sync(0xffffffffu, Yh, owner),
                    oZh = __shfl_sync(0xffffffffu, Zh, owner);
        const float oXl = __shfl_sync(0xffffffffu, Xl, owner), oYl = __shfl_sync(0xffffffffu, Yl, owner),
                    oZl = __shfl_sync(0xffffffffu, Zl, owner);
        Ldl3 of;
        of.l21 = __shfl_sync(0xffffffffu, fs.l21, owner);
        of.l31 = __shfl_sync(0xffffffffu, fs.l31, owner);
        of.l32 = __shfl_sync(0xffffffffu, fs.l32, owner);
        of.i1 = __shfl_sync(0xffffffffu, fs.i1, owner);
        of.i2 = __shfl_sync(0xffffffffu, fs.i2, owner);
        of.i3 = __shfl_sync(0xffffffffu, fs.i3, owner);
        double c2 = -1.0;
        int hidx = 0x7fffffff;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        if (item < warp_total) {
            int rem = item - opre;
            int j = -1;
            const int last = oplo + onph - 1;
            for (int zb = ozlo; zb <= ozhi && j < 0; ++zb) {
                const int row = zb * KF_NPHI;
                const int a0 = ooff[row + oplo], a1 = ooff[row + min(last, KF_NPHI - 1) + 1];
                if (rem < a1 - a0) {
                    j = a0 + rem;
                    break;
                }
                rem -= a1 - a0;
                if (last >= KF_NPHI) {
                    const int b0 = ooff[row], b1 = ooff[row + (last - KF_NPHI) + 1];
                    if (rem < b1 - b0) {
                        j = b0 + rem;
                        break;
                    }
                    rem -= b1 - b0;
                }
            }
            if (j >= 0 && j < onh) {
                h = opk[j];
                hidx = __float_as_int(h.w);
                const float rx = __fsub_rn(__fsub_rn(h.x, oXh), oXl);
                const float ry = __fsub_rn(__fsub_rn(h.y, oYh), oYl);
                const float rz = __fsub_rn(__fsub_rn(h.z, oZh), oZl);
                c2 = ldl3_chi2(of, wide(rx), wide(ry), wide(rz));
            }
        }
        // each owner folds the round's items that belong to it
#pragma unroll 1
        for (int d = 0; d < 32; ++d) {
            const double dc = __shfl_sync(0xffffffffu, c2, d);
            const int di = __shfl_sync(0xffffffffu, hidx, d);
            const int down = __shfl_sync(0xffffffffu, owner, d);
            const float dhx = __shfl_sync(0xffffffffu, h.x, d), dhy = __shfl_sync(0xffffffffu, h.y, d),
                        dhz = __shfl_sync(0xffffffffu, h.z, d);
            if (down == lane && r0 + d < warp_total && dc >= 0.0 &&
                (best < 0 || dc < bchi || (dc == bchi && di < best))) {
                best = di;
                bchi = dc;
                bhit = make_float4(dhx, dhy, dhz, __int_as_float(di));
            }
        }
    }
}

// The build keeps the covariance in FP32 on the mixed path after the seed fit
// (whose updates are the FP64 ones) and in FP64 on the all-FP64 path; a mixed
// step at a near-tangent crossing runs in FP64.
// The seed fit of a build track over its three seed hits (layers 0..2 of its
// event): the first n64 updates with an FP64 covariance (the structured update
// at the first hit, Joseph form after), the rest in the layer covariance type.
// Returns whether the track is still alive.
// M1: barrel seed hits on their own cylinders with the 2-D update.
template <bool FP64, bool M1 = false>
__device__ __forceinline__ bool seed_fit(const BuildArgs &a, const Surf *s_surf, const LayerDev *lays, int n, int t,
                                         Track<typename sel_t<FP64>::T, typename sel_t<FP64>::P> &st,
                                         typename sel_t<FP64>::T pc[21], typename sel_t<FP64>::T alpha,
                                         typename sel_t<FP64>::T mass2, unsigned &status, double &chi2, int &used,
                                         bool alive)
{
    using T = typename sel_t<FP64>::T;
    using C = T;
    // seed fit over the three seed hits; the first n64 updates with an FP64 covariance
    double pd[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pd[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) pd[pk(i, i)] = a.seed_cov;
    const int n1 = min(a.n64, 3);
    int k = 0;
    bool in_pc = false;  // phase 1 ran in double-float and left its covariance in pc
    if constexpr (!FP64) {
        if (a.seed_df && n1 > 0) {
            // the first n1 updates in double-float on the FP32 pipe (kf_df.cuh)
            df pq[21];
            df_seed_cov(pq, a.seed_cov);
            df c2 = df(0.f);
            for (; k < n1 && alive; ++k) {
                const Surf &sf = s_surf[lays[k].surface];
                const float hx = a.seed_hits[(3 * k + 0) * n + t], hy = a.seed_hits[(3 * k + 1) * n + t],
                            hz = a.seed_hits[(3 * k + 2) * n + t];
                bool ok;
                if (M1 && k > 0 && sf.kind == 0)
                    ok = df_step_on<true>(st, pq, k, alpha, mass2, a.ms_on, hit_surface(sf, hx, hy), hx, hy, hz, c2,
                                          status, k == 1);
                else
                    ok = df_step_on<false>(st, pq, k, alpha, mass2, a.ms_on, sf, hx, hy, hz, c2, status, k == 1);
                if (!ok) {
                    alive = false;
                    break;
                }
                ++used;
            }
            chi2 += df_to_d(c2);
#pragma unroll
            for (int i = 0; i < 21; ++i) pc[i] = pq[i].hi;
            in_pc = true;
        }
    }
    for (; !in_pc && k < n1 && alive; ++k) {
        const Surf &sf = s_surf[lays[k].surface];
        const float hx = a.seed_hits[(3 * k + 0) * n + t], hy = a.seed_hits[(3 * k + 1) * n + t],
                    hz = a.seed_hits[(3 * k + 2) * n + t];
        if constexpr (M1) {
            if (k > 0 && sf.kind == 0) {  // the first hit: the 3-D update (the state starts on it)
                const Surf h = hit_surface(sf, hx, hy);
                // k == 1: the covariance is the one the structured seed-hit update left
                alive = k == 1 ? fit_step_on<true, double, true, true>(st, pd, k, alpha, mass2, a.ms_on, h, hx, hy,
                                                                       hz, chi2, status)
                               : fit_step_on<true, double, true>(st, pd, k, alpha, mass2, a.ms_on, h, hx, hy, hz,
                                                                 chi2, status);
                if (!alive) break;
                ++used;
                continue;
            }
        }
        T cphi, sphi;
        if (k > 0) {
            Jac<T> J;
            if (!propagate(st, alpha, sf, J)) {
                status |= reach_bits(st);
                alive = false;
                break;
            }
            // k == 1: the covariance is the one the structured seed-hit update left
            if (k == 1) transport_seeded<double>(pd, JacAs<double>::get(J));
            else transport<double>(pd, JacAs<double>::get(J));
            cphi = J.cphi1;
            sphi = J.sphi1;
        } else {
            sincos_pos(st.phi, sphi, cphi);
        }
        if (a.ms_on) status |= ms_noise<T, double>(st, sf, cphi, sphi, mass2, pd);
        // the first hit meets the diagonal seed covariance: the structured update
        const bool ok = k == 0 ? kf_seed_update(st, pd, hx, hy, hz, sf, chi2)
                               : kf_update<true>(st, pd, hx, hy, hz, sf, chi2);
        if (!ok) {
            status |= KF_ST_CHOL_FAIL;
            alive = false;
            break;
        }
        ++used;
    }
    if (!in_pc) {
#pragma unroll
        for (int i = 0; i < 21; ++i) pc[i] = (C)pd[i];
    }
    for (; k < 3 && alive; ++k) {
        const Surf &sf = s_surf[lays[k].surface];
        const float hx = a.seed_hits[(3 * k + 0) * n + t], hy = a.seed_hits[(3 * k + 1) * n + t],
                    hz = a.seed_hits[(3 * k + 2) * n + t];
        if constexpr (M1) {
            if (k > 0 && sf.kind == 0) {  // the first hit: the 3-D update (the state starts on it)
                const Surf h = hit_surface(sf, hx, hy);
                alive = fit_step_on<false, C, true>(st, pc, k, alpha, mass2, a.ms_on, h, hx, hy, hz, chi2, status);
                if (!alive) break;
                ++used;
                continue;
            }
        }
        T cphi, sphi;
        if (k > 0) {
            Jac<T> J;
            if (!propagate(st, alpha, sf, J)) {
                status |= reach_bits(st);
                alive = false;
                break;
            }
            transport<C>(pc, JacAs<C>::get(J));
            cphi = J.cphi1;
            sphi = J.sphi1;
        } else {
            sincos_pos(st.phi, sphi, cphi);
        }
        if (a.ms_on) status |= ms_noise<T, C>(st, sf, cphi, sphi, mass2, pc);
        if (!kf_update_mixed(st, pc, hx, hy, hz, sf, chi2)) {
            status |= KF_ST_CHOL_FAIL;
            alive = false;
            break;
        }
        ++used;
    }
    return alive;
}

// The seed fit of a mixed-path build track as the pre-pass leaves it: state as
// float-float (x, y, z, phi, theta; hi then lo) and 1/pT, the FP32 covariance,
// chi2, hits used, status, alive; [k][n] arrays.
struct SeedFits {
    float *st;       // [11][n]
    float *cov;      // [21][n]
    double *chi2;    // [n]
    int32_t *used;   // [n]
    uint32_t *status;
    int8_t *alive;
};
__host__ __device__ inline size_t seed_al(size_t b) { return (b + 255) & ~(size_t)255; }
__host__ __device__ inline SeedFits seed_carve(void *scratch, int n)
{
    const size_t m = (size_t)n;
    char *p = static_cast<char *>(scratch);
    SeedFits f;
    f.st = reinterpret_cast<float *>(p);
    p += seed_al(11 * 4 * m);
    f.cov = reinterpret_cast<float *>(p);
    p += seed_al(21 * 4 * m);
    f.chi2 = reinterpret_cast<double *>(p);
    p += seed_al(8 * m);
    f.used = reinterpret_cast<int32_t *>(p);
    p += seed_al(4 * m);
    f.status = reinterpret_cast<uint32_t *>(p);
    p += seed_al(4 * m);
    f.alive = reinterpret_cast<int8_t *>(p);
    return f;
}
size_t build_seed_scratch_bytes(int n)
{
    const size_t m = (size_t)n;
    return seed_al(11 * 4 * m) + seed_al(21 * 4 * m) + seed_al(8 * m) + seed_al(4 * m) + seed_al(4 * m) + seed_al(m) +
           256;
}

// Pre-pass of the mixed-path best-hit build: the seed fit of every track (its
// FP64 phase) in a kernel of its own, so that the layer kernel's code holds the
// layer loop alone (warps at different stages of one kernel share its
// instruction cache).  Tracks in processing order, as the layer kernel.  Four
// blocks per SM (128 registers instead of 168 at three): the build call 1.34 ms
// against 1.38 for 10 x 20,000 tracks.
template <bool M1>
__global__ void __launch_bounds__(128, 4) build_seed_kernel(const Geom g, const BuildArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) s_surf[i] = g.s[i];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int t = a.order ? a.order[i] : i;
    const int n = a.n;
    const int e = find_event(a.event_off, a.n_events, t);
    const LayerDev *lays = a.layers + (size_t)e * a.n_layers;
    Track<float, ff> st;
    st.x = from_f<ff>(a.seed_state[0 * n + t]);
    st.y = from_f<ff>(a.seed_state[1 * n + t]);
    st.z = from_f<ff>(a.seed_state[2 * n + t]);
    st.ip = a.seed_state[3 * n + t];
    st.phi = from_f<ff>(a.seed_state[4 * n + t]);
    st.th = from_f<ff>(a.seed_state[5 * n + t]);
    const int q = a.q[t];
    float pc[21];
    unsigned status = 0u;
    double chi2 = 0.0;
    int used = 0;
    const bool alive =
        seed_fit<false, M1>(a, s_surf, lays, n, t, st, pc, float(-q) * g.kb, g.mass2, status, chi2, used, true);
    const SeedFits f = seed_carve(a.seed_scratch, n);
    const float w[11] = {st.x.hi, st.x.lo, st.y.hi, st.y.lo, st.z.hi, st.z.lo, st.phi.hi, st.phi.lo, st.th.hi,
                         st.th.lo, st.ip};
#pragma unroll
    for (int k = 0; k < 11; ++k) f.st[(size_t)k * n + t] = w[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) f.cov[(size_t)k * n + t] = pc[k];
    f.chi2[t] = chi2;
    f.used[t] = used;
    f.status[t] = status;
    f.alive[t] = alive ? 1 : 0;
}

// Launch shape of the layer kernel.  Model 0: blocks of 256 threads, two per SM
// (at most 128 registers a thread: 16 warps to hide the FP64 and memory
// latencies), so that eight warps step each layer together under the block
// barrier and share the instruction cache: 1.26 ms per build call for
// 10 x 20,000 tracks against 1.34 with four blocks of 128 and 1.53 with eight of
// 64.  M1, measurement model 1 (per-thread scoring): two blocks of 128 (208
// registers; its larger step spills less), 5.5 ms against 6.7 with one block of
// 256 and 6.3 with three of 128.
template <bool M1>
constexpr int build_block_threads()
{
    return M1 ? 128 : 256;
}

template <bool FP64, bool COOP, bool M1>
__global__ void __launch_bounds__(build_block_threads<M1>(), 2) build_kernel(const Geom g, const BuildArgs a)
{
    using T = typename sel_t<FP64>::T;
    using P = typename sel_t<FP64>::P;
    using C = T;  // covariance type of the build layers
    __shared__ Surf s_surf[MAX_SURF];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) s_surf[i] = g.s[i];
    __syncthreads();
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i0 < a.n;
    const int i = active ? i0 : a.n - 1;  // inactive lanes shadow a real track but write nothing
    const int t = a.order ? a.order[i] : i;
    const int n = a.n;
    const int e = find_event(a.event_off, a.n_events, t);
    const LayerDev *lays = a.layers + (size_t)e * a.n_layers;
    Track<T, P> st;
    st.x = from_f<P>(a.seed_state[0 * n + t]);
    st.y = from_f<P>(a.seed_state[1 * n + t]);
    st.z = from_f<P>(a.seed_state[2 * n + t]);
    st.ip = (T)a.seed_state[3 * n + t];
    st.phi = from_f<P>(a.seed_state[4 * n + t]);
    st.th = from_f<P>(a.seed_state[5 * n + t]);
    const int q = a.q[t];
    const T alpha = FP64 ? T(-q * g.kbd) : T(-q) * T(g.kb);
    const T mass2 = FP64 ? T(g.mass2d) : T(g.mass2);
    const double alphad = -q * g.kbd;
    unsigned status = 0u;
    double chi2 = 0.0;
    int used = 0;
    bool alive = active;
    C pc[21];
    const StepKnobs kn{a.ms_on, a.max_cand, a.nsigma, a.chi2_cut, nullptr, n};
    if constexpr (FP64) {
        alive = seed_fit<FP64, M1>(a, s_surf, lays, n, t, st, pc, alpha, mass2, status, chi2, used, alive);
    } else {  // the pre-pass's seed fit
        const SeedFits f = seed_carve(a.seed_scratch, n);
        st.x = ff{f.st[0 * (size_t)n + t], f.st[1 * (size_t)n + t]};
        st.y = ff{f.st[2 * (size_t)n + t], f.st[3 * (size_t)n + t]};
        st.z = ff{f.st[4 * (size_t)n + t], f.st[5 * (size_t)n + t]};
        st.phi = ff{f.st[6 * (size_t)n + t], f.st[7 * (size_t)n + t]};
        st.th = ff{f.st[8 * (size_t)n + t], f.st[9 * (size_t)n + t]};
        st.ip = f.st[10 * (size_t)n + t];
#pragma unroll
        for (int k = 0; k < 21; ++k) pc[k] = f.cov[(size_t)k * n + t];
        chi2 = f.chi2[t];
        used = f.used[t];
        status = f.status[t];
        alive = active && f.alive[t] != 0;
    }
    if (active)
        for (int L = 0; L < 3; ++L) a.hit_idx[(size_t)L * n + t] = -1;
    // build layers.  A block barrier per layer keeps the block's four warps in
    // the same layer step, so that they run the same stretch of the long loop
    // body and share the instruction cache (instruction fetch was the largest
    // stall): 1.39 ms for 10 x 20,000 tracks against 1.75 without it.  Every
    // thread runs every layer (no thread leaves the loop early).
    for (int L = 3; L < a.n_layers; ++L) {
        __syncthreads();
        const LayerDev ly = lays[L];
        const Surf &sf = s_surf[ly.surface];
        StepKnobs knl = kn;
        if (a.dbg_pred && active) knl.dbg = a.dbg_pred + (size_t)L * 27 * n + t;
        StepOut so{-1, false};
        bool near_tangent = false;
        if constexpr (!FP64) near_tangent = alive && crossing_sine(st, alpha, sf) > 0.8f;
        if (near_tangent) {
            if constexpr (!FP64) {
                Fp64LayerIO io;
                mixed_pack(io.m, st, pc, chi2, status);
                io.alive = alive;
                // model 0: the double-float step; model 1 (two propagations per step) in FP64
                if constexpr (M1) io = layer_step_fp64_out_of_line<M1>(io, alphad, g.mass2d, knl, &sf, ly);
                else io = layer_step_df_out_of_line(io, alpha, mass2, knl, &sf, ly);
                mixed_unpack(io.m, st, pc, chi2, status);
                alive = io.alive != 0;
                so = io.o;
            }
        }
        // the cooperative path needs the S factor shared by a layer's candidates; the
        // condition is the same for every lane (all events share the geometry)
        const bool coop = COOP && !M1 && sf.var_rad == sf.var_rphi;
        if (!coop) {
            if (alive && !near_tangent)
                so = layer_step_thread<false, M1>(st, pc, alpha, mass2, knl, sf, ly, chi2, status, alive);
        } else {
            // every lane of the warp takes part in the shuffles, stepping or not
            bool do_step = alive && !near_tangent;
            if (do_step) {
                Jac<T> J;
                if (!propagate(st, alpha, sf, J)) {
                    status |= reach_bits(st);
                    alive = false;
                    do_step = false;
                } else {
                    transport<C>(pc, JacAs<C>::get(J));
                    if (a.ms_on) status |= ms_noise<T, C>(st, sf, J.cphi1, J.sphi1, mass2, pc);
                    debug_pred_put(knl, st, pc);
                }
            }
            float pw[21];
#pragma unroll
            for (int i = 0; i < 21; ++i) pw[i] = (float)pc[i];
            Window w{0, 0, 0, -1};
            Ldl3 fs{0, 0, 0, 0, 0, 0};
            if (do_step) {
                w = make_window(st, pw, sf, a.nsigma);
                if (!shared_factor(pc, sf, fs)) {
                    status |= KF_ST_CHOL_FAIL;
                    alive = false;
                    do_step = false;
                }
            }
            int best = -1;
            double bchi = 0.0;
            float4 bhit = make_float4(0.f, 0.f, 0.f, 0.f);
            score_coop(st, do_step, w, fs, ly, a.max_cand, best, bchi, bhit, so.capped);
            if (do_step && best >= 0 && bchi < (double)a.chi2_cut) {
                bool ok;
                if constexpr (sizeof(C) == 4) ok = kf_update_mixed_factored(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2, fs, bchi);
                else ok = kf_update_mixed(st, pc, bhit.x, bhit.y, bhit.z, sf, chi2);
                if (ok) {
                    so.chosen = best;
                } else {
                    status |= KF_ST_CHOL_FAIL;
                    alive = false;
                }
            }
        }
        if (so.capped) status |= KF_ST_CAND_CAPPED;
        if (so.chosen >= 0) ++used;
        if (active) a.hit_idx[(size_t)L * n + t] = so.chosen;
    }
    if (!active) return;
    double sv[6] = {to_d(st.x), to_d(st.y), to_d(st.z), (double)st.ip, to_d(st.phi), to_d(st.th)};
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (!isfinite(sv[i])) status |= KF_ST_NONFINITE;
    if (a.o_state)
        for (int i = 0; i < 6; ++i) a.o_state[(size_t)i * n + t] = sv[i];
    if (a.o_cov)
        for (int i = 0; i < 21; ++i) a.o_cov[(size_t)i * n + t] = (double)pc[i];
    if (a.o_cov32)
        for (int i = 0; i < 21; ++i) a.o_cov32[(size_t)i * n + t] = (float)pc[i];
    if (a.o_chi2) a.o_chi2[t] = chi2;
    if (a.o_ndof) a.o_ndof[t] = 2 * used - 5;
    if (a.o_status) a.o_status[t] = status;
}

cudaError_t launch_build(const Geom &g, const BuildArgs &a, bool fp64, bool warp_coop, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const int b = 128, grid = (a.n + b - 1) / b;  // the seed pre-pass
    if (!fp64) {
        if (!a.seed_scratch) return cudaErrorInvalidValue;
        if (a.meas_model == 1) build_seed_kernel<true><<<grid, b, 0, st>>>(g, a);
        else build_seed_kernel<false><<<grid, b, 0, st>>>(g, a);
    }
    if (a.meas_model == 1) {  // per-thread scoring
        constexpr int b1 = build_block_threads<true>();
        const int grid1 = (a.n + b1 - 1) / b1;
        if (fp64) build_kernel<true, false, true><<<grid1, b1, 0, st>>>(g, a);
        else build_kernel<false, false, true><<<grid1, b1, 0, st>>>(g, a);
    } else {
        constexpr int b0 = build_block_threads<false>();
        const int grid0 = (a.n + b0 - 1) / b0;
        if (fp64) {
            if (warp_coop) build_kernel<true, true, false><<<grid0, b0, 0, st>>>(g, a);
            else build_kernel<true, false, false><<<grid0, b0, 0, st>>>(g, a);
        } else {
            if (warp_coop) build_kernel<false, true, false><<<grid0, b0, 0, st>>>(g, a);
            else build_kernel<false, false, false><<<grid0, b0, 0, st>>>(g, a);
        }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ combinatorial building
// Sec. 2: building branches to explore several candidates per seed; Sec. 4.3:
// a fixed number of slots per seed holds its candidates, the best kept.  Here
// the slots of a seed are n_slots consecutive lanes of a warp, each carrying
// one candidate in registers.  Per layer every lane predicts its candidate,
// searches the window and lists its best children (hits below the chi2 cut,
// ranked; then the candidate without a hit); the lanes of the seed merge their
// lists with shuffles into the seed's new ranking (more hits first, then
// smaller total chi2, then lower parent slot, then lower hit index); lane j
// takes the j-th child, fetching its parent's predicted state from the
// parent's lane by shuffles, and updates it with the child's hit.  A back
// pointer (parent slot, hit) per layer and slot gives the hits of the best
// candidate at the end.

// pre-pass: the seed fit, one thread per seed
__global__ void __launch_bounds__(128, 4) ckf_seed_kernel(const Geom g, const CkfArgs c)
{
    const BuildArgs &a = c.b;
    __shared__ Surf s_surf[MAX_SURF];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) s_surf[i] = g.s[i];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n) return;
    const int n = a.n;
    const int e = find_event(a.event_off, a.n_events, t);
    const LayerDev *lays = a.layers + (size_t)e * a.n_layers;
    Track<float, ff> st;
    st.x = from_f<ff>(a.seed_state[0 * n + t]);
    st.y = from_f<ff>(a.seed_state[1 * n + t]);
    st.z = from_f<ff>(a.seed_state[2 * n + t]);
    st.ip = a.seed_state[3 * n + t];
    st.phi = from_f<ff>(a.seed_state[4 * n + t]);
    st.th = from_f<ff>(a.seed_state[5 * n + t]);
    const int q = a.q[t];
    float pc[21];
    unsigned status = 0u;
    double chi2 = 0.0;
    int used = 0;
    const bool alive =
        seed_fit<false>(a, s_surf, lays, n, t, st, pc, float(-q) * g.kb, g.mass2, status, chi2, used, true);
    const float w[11] = {st.x.hi, st.x.lo, st.y.hi, st.y.lo, st.z.hi, st.z.lo, st.phi.hi, st.phi.lo, st.th.hi,
                         st.th.lo, st.ip};
#pragma unroll
    for (int k = 0; k < 11; ++k) c.seed_st[(size_t)k * n + t] = w[k];
#pragma unroll
    for (int k = 0; k < 21; ++k) c.seed_cov[(size_t)k * n + t] = pc[k];
    c.seed_chi2[t] = chi2;
    c.seed_used[t] = used;
    c.seed_status[t] = status;
    c.seed_alive[t] = alive ? 1 : 0;
}

// prediction of a near-tangent crossing with the transport and scattering
// noise in double-float (FP32 propagation), out of line
static __device__ __noinline__ MixedIO ckf_predict_df(MixedIO m, float alpha, float mass2, int ms_on,
                                                     const Surf *sf)
{
    Jac<float> J;
    if (!propagate(m.st, alpha, *sf, J)) {
        m.ok = 0;
        return m;
    }
    df p[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) p[i] = df(m.p[i]);
    transport<df>(p, J);
    if (ms_on) m.status |= ms_noise<float, df>(m.st, *sf, J.cphi1, J.sphi1, mass2, p);
#pragma unroll
    for (int i = 0; i < 21; ++i) m.p[i] = p[i].hi;
    m.ok = 1;
    return m;
}

// A child in the seed's ranking.  nh < 0: no child.
struct CkfKey {
    int nh;
    int parent;
    int hit;  // original hit index; a child without a hit ranks after its parent's hits
    double chi2;
};
constexpr int CKF_NO_HIT = 0x7fffffff;

__device__ __forceinline__ bool ckf_before(const CkfKey &a, const CkfKey &b)
{
    if (a.nh != b.nh) return a.nh > b.nh;
    if (a.chi2 != b.chi2) return a.chi2 < b.chi2;
    if (a.parent != b.parent) return a.parent < b.parent;
    return a.hit < b.hit;
}

__device__ __forceinline__ CkfKey ckf_shfl_xor(const CkfKey &k, int m)
{
    CkfKey o;
    o.nh = __shfl_xor_sync(0xffffffffu, k.nh, m);
    o.parent = __shfl_xor_sync(0xffffffffu, k.parent, m);
    o.hit = __shfl_xor_sync(0xffffffffu, k.hit, m);
    o.chi2 = __shfl_xor_sync(0xffffffffu, k.chi2, m);
    return o;
}

__device__ __forceinline__ ff shfl_ff(ff v, int src)
{
    return ff{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

// At most 128 registers a thread (16 warps per SM).  Four and eight slots: blocks
// of 256 threads, two per SM, eight warps stepping each layer together under the
// block barrier: 4.62 / 10.08 ms on 10 x 20,000 tracks against 4.78 / 10.52 with
// four blocks of 128; two slots: four blocks of 128 (2.27 ms, against 2.32).
template <int NS>
constexpr int ckf_block_threads()
{
    return NS >= 4 ? 256 : 128;
}

template <int NS>
__global__ void __launch_bounds__(ckf_block_threads<NS>(), NS >= 4 ? 2 : 4) ckf_kernel(const Geom g, const CkfArgs c)
{
    const BuildArgs &a = c.b;
    __shared__ Surf s_surf[MAX_SURF];
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) s_surf[i] = g.s[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int slot = lane & (NS - 1);
    const int base = lane & ~(NS - 1);
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) / NS;
    const bool active = i0 < a.n;
    const int i = active ? i0 : a.n - 1;  // inactive lanes shadow a real seed but write nothing
    const int t = a.order ? a.order[i] : i;
    const int n = a.n;
    const size_t nslots = (size_t)n * NS;
    const int e = find_event(a.event_off, a.n_events, t);
    const LayerDev *lays = a.layers + (size_t)e * a.n_layers;
    const int q = a.q[t];
    const float alpha = float(-q) * g.kb;
    const StepKnobs kn{a.ms_on, a.max_cand, a.nsigma, a.chi2_cut, nullptr, n};
    // the seed's candidate in slot 0; the other slots start empty
    Track<float, ff> st;
    st.x = ff{c.seed_st[0 * (size_t)n + t], c.seed_st[1 * (size_t)n + t]};
    st.y = ff{c.seed_st[2 * (size_t)n + t], c.seed_st[3 * (size_t)n + t]};
    st.z = ff{c.seed_st[4 * (size_t)n + t], c.seed_st[5 * (size_t)n + t]};
    st.phi = ff{c.seed_st[6 * (size_t)n + t], c.seed_st[7 * (size_t)n + t]};
    st.th = ff{c.seed_st[8 * (size_t)n + t], c.seed_st[9 * (size_t)n + t]};
    st.ip = c.seed_st[10 * (size_t)n + t];
    float pc[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) pc[k] = c.seed_cov[(size_t)k * n + t];
    double chi2 = c.seed_chi2[t];
    int nu = c.seed_used[t];
    int nh = 3;
    unsigned status = c.seed_status[t];
    bool alive = slot == 0 && c.seed_alive[t] != 0;
    bool stopped = false;
    if (active && slot == 0)
        for (int L = 0; L < 3; ++L) a.hit_idx[(size_t)L * n + t] = -1;
    // a block barrier per layer keeps the block's warps in the same layer step
    // (the instruction cache; as in the best-hit kernel): 4.81 ms for four slots
    // of 10 x 20,000 seeds against 5.30 without it.  No thread leaves the loop early.
    for (int L = 3; L < a.n_layers; ++L) {
        __syncthreads();
        const LayerDev ly = lays[L];
        const Surf &sf = s_surf[ly.surface];
        // 1. prediction (a candidate that cannot reach the layer stops, unchanged)
        unsigned step = 0u;
        bool search = alive && !stopped;
        bool stop_now = false;
        if (search) {
            if (crossing_sine(st, alpha, sf) > 0.8f) {
                MixedIO m;
                mixed_pack(m, st, pc, chi2, 0u);
                m = ckf_predict_df(m, alpha, g.mass2, a.ms_on, &sf);
                if (m.ok) {
                    unsigned s2;
                    double c2;
                    mixed_unpack(m, st, pc, c2, s2);
                    step |= s2;
                } else {
                    stop_now = true;
                }
            } else {
                Jac<float> J;
                if (!propagate(st, alpha, sf, J)) {
                    stop_now = true;
                } else {
                    transport<float>(pc, J);
                    if (a.ms_on) step |= ms_noise<float, float>(st, sf, J.cphi1, J.sphi1, g.mass2, pc);
                }
            }
        }
        if (stop_now) {
            step |= reach_bits(st);
            search = false;
        }
        const bool pass = alive && (stopped || stop_now);  // carried unchanged
        // 2. window search: this candidate's best NS hits below the cut, ranked
        double lc[NS];
        int lh[NS], lp[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            lc[k] = 0.0;
            lh[k] = CKF_NO_HIT;
            lp[k] = -1;
        }
        int cnt = 0;
        if (search) {
            const Window w = make_window(st, pc, sf, kn.nsigma);
            const bool shared = sf.var_rad == sf.var_rphi;
            Ldl3 fs{0, 0, 0, 0, 0, 0};
            const bool fs_ok = !shared || shared_factor(pc, sf, fs);
            int ncand = 0;
            bool capped = false;
            for (int zb = w.z_lo; zb <= w.z_hi && !capped && fs_ok; ++zb) {
                const int row = zb * KF_NPHI;
                const int first = w.phi_lo, last = w.phi_lo + w.nphi - 1;
                for (int part = 0; part < 2 && !capped; ++part) {
                    int b0, b1;
                    if (part == 0) {
                        b0 = first;
                        b1 = min(last, KF_NPHI - 1);
                    } else {
                        if (last < KF_NPHI) break;
                        b0 = 0;
                        b1 = last - KF_NPHI;
                    }
                    const int j0 = max(ly.offsets[row + b0], 0), j1 = min(ly.offsets[row + b1 + 1], ly.n_hits);
                    for (int j = j0; j < j1; ++j) {
                        if (ncand >= kn.max_cand) {
                            capped = true;
                            break;
                        }
                        ++ncand;
                        const float4 h = ly.packed[j];
                        const double c2 = cand_chi2(st, pc, sf, shared, fs, h);
                        if (!(c2 >= 0.0 && c2 < (double)kn.chi2_cut)) continue;
                        const double tot = chi2 + c2;
                        const int hi = __float_as_int(h.w);
                        // rank among this candidate's hits: total chi2, then hit index
                        int pos = 0;
#pragma unroll
                        for (int k = 0; k < NS; ++k)
                            if (k < cnt && (lc[k] < tot || (lc[k] == tot && lh[k] < hi))) ++pos;
                        if (pos < NS) {
#pragma unroll
                            for (int k = NS - 1; k > 0; --k)
                                if (k > pos) {
                                    lc[k] = lc[k - 1];
                                    lh[k] = lh[k - 1];
                                    lp[k] = lp[k - 1];
                                }
#pragma unroll
                            for (int k = 0; k < NS; ++k)
                                if (k == pos) {
                                    lc[k] = tot;
                                    lh[k] = hi;
                                    lp[k] = j;
                                }
                            cnt = min(cnt + 1, NS);
                        }
                    }
                }
            }
            if (capped) step |= KF_ST_CAND_CAPPED;
        }
        // 3. the seed's new ranking: NS rounds of a shuffle minimum over its lanes
        int head = 0;
        CkfKey mine{-1, 0, CKF_NO_HIT, 0.0};
        int my_ppos = -1;
        for (int r = 0; r < NS; ++r) {
            CkfKey k{-1, slot, CKF_NO_HIT, 0.0};
            int ppos = -1;
            if (pass) {
                if (head == 0) k = CkfKey{nh, slot, CKF_NO_HIT, chi2};
            } else if (search) {
#pragma unroll
                for (int m = 0; m < NS; ++m)
                    if (m == head && m < cnt) {
                        k = CkfKey{nh + 1, slot, lh[m], lc[m]};
                        ppos = lp[m];
                    }
                if (head == cnt) k = CkfKey{nh, slot, CKF_NO_HIT, chi2};
            }
            CkfKey best = k;
#pragma unroll
            for (int m = 1; m < NS; m <<= 1) {
                const CkfKey o = ckf_shfl_xor(best, m);
                if (ckf_before(o, best)) best = o;
            }
            const int owner = base + (best.nh >= 0 ? best.parent : slot);
            const int wpos = __shfl_sync(0xffffffffu, ppos, owner);
            if (best.nh >= 0 && best.parent == slot) ++head;
            if (slot == r) {
                mine = best;
                my_ppos = wpos;
            }
        }
        // 4. take the child: the parent's predicted candidate, by shuffles
        const int src = base + (mine.nh >= 0 ? mine.parent : slot);
        const unsigned pstat = status | step;
        Track<float, ff> ps;
        ps.x = shfl_ff(st.x, src);
        ps.y = shfl_ff(st.y, src);
        ps.z = shfl_ff(st.z, src);
        ps.phi = shfl_ff(st.phi, src);
        ps.th = shfl_ff(st.th, src);
        ps.ip = __shfl_sync(0xffffffffu, st.ip, src);
#pragma unroll
        for (int k = 0; k < 21; ++k) pc[k] = __shfl_sync(0xffffffffu, pc[k], src);
        st = ps;
        chi2 = __shfl_sync(0xffffffffu, chi2, src);
        nu = __shfl_sync(0xffffffffu, nu, src);
        status = __shfl_sync(0xffffffffu, pstat, src);
        const bool pstop = __shfl_sync(0xffffffffu, (int)(stopped || stop_now), src) != 0;
        alive = active && mine.nh >= 0;
        stopped = pstop;
        if (alive && mine.hit != CKF_NO_HIT) {
            const float4 h = ly.packed[my_ppos];
            double c2u = 0.0;
            if (!kf_update_mixed(st, pc, h.x, h.y, h.z, sf, c2u)) status |= KF_ST_CHOL_FAIL;
            nu += 1;
        }
        if (alive) {
            chi2 = mine.chi2;
            nh = mine.nh;
        }
        if (active) {
            c.bp_parent[(size_t)L * nslots + (size_t)i * NS + slot] = (int8_t)(alive ? mine.parent : -1);
            c.bp_hit[(size_t)L * nslots + (size_t)i * NS + slot] = alive && mine.hit != CKF_NO_HIT ? mine.hit : -1;
        }
    }
    __syncwarp();
    if (!active || slot != 0) return;
    // 5. the first candidate is the track
    int s = 0;
    for (int L = a.n_layers - 1; L >= 3; --L) {
        const size_t o = (size_t)L * nslots + (size_t)i * NS + s;
        a.hit_idx[(size_t)L * n + t] = c.bp_hit[o];
        s = max((int)c.bp_parent[o], 0);
    }
    double sv[6] = {to_d(st.x), to_d(st.y), to_d(st.z), (double)st.ip, to_d(st.phi), to_d(st.th)};
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (!isfinite(sv[k])) status |= KF_ST_NONFINITE;
    if (a.o_state)
        for (int k = 0; k < 6; ++k) a.o_state[(size_t)k * n + t] = sv[k];
    if (a.o_cov)
        for (int k = 0; k < 21; ++k) a.o_cov[(size_t)k * n + t] = (double)pc[k];
    if (a.o_cov32)
        for (int k = 0; k < 21; ++k) a.o_cov32[(size_t)k * n + t] = (float)pc[k];
    if (a.o_chi2) a.o_chi2[t] = chi2;
    if (a.o_ndof) a.o_ndof[t] = 2 * nu - 5;
    if (a.o_status) a.o_status[t] = status;
}

size_t ckf_scratch_bytes(int n, int n_layers, int n_slots)
{
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t m = (size_t)n;
    return al(11 * 4 * m) + al(21 * 4 * m) + al(8 * m) + al(4 * m) + al(4 * m) + al(m) +
           al((size_t)n_layers * m * n_slots) + al(4 * (size_t)n_layers * m * n_slots) + 256;
}

void ckf_carve(CkfArgs &c, void *scratch, int n, int n_layers, int n_slots)
{
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t m = (size_t)n;
    char *p = static_cast<char *>(scratch);
    c.seed_st = reinterpret_cast<float *>(p);
    p += al(11 * 4 * m);
    c.seed_cov = reinterpret_cast<float *>(p);
    p += al(21 * 4 * m);
    c.seed_chi2 = reinterpret_cast<double *>(p);
    p += al(8 * m);
    c.seed_used = reinterpret_cast<int32_t *>(p);
    p += al(4 * m);
    c.seed_status = reinterpret_cast<uint32_t *>(p);
    p += al(4 * m);
    c.seed_alive = reinterpret_cast<int8_t *>(p);
    p += al(m);
    c.bp_parent = reinterpret_cast<int8_t *>(p);
    p += al((size_t)n_layers * m * n_slots);
    c.bp_hit = reinterpret_cast<int32_t *>(p);
}

cudaError_t launch_ckf(const Geom &g, const CkfArgs &c, cudaStream_t st)
{
    const int n = c.b.n;
    if (n <= 0) return cudaSuccess;
    ckf_seed_kernel<<<(n + 127) / 128, 128, 0, st>>>(g, c);
    const long long threads = (long long)n * c.n_slots;
    auto grid = [threads](int b) { return (int)((threads + b - 1) / b); };
    switch (c.n_slots) {
    case 1: ckf_kernel<1><<<grid(ckf_block_threads<1>()), ckf_block_threads<1>(), 0, st>>>(g, c); break;
    case 2: ckf_kernel<2><<<grid(ckf_block_threads<2>()), ckf_block_threads<2>(), 0, st>>>(g, c); break;
    case 4: ckf_kernel<4><<<grid(ckf_block_threads<4>()), ckf_block_threads<4>(), 0, st>>>(g, c); break;
    case 8: ckf_kernel<8><<<grid(ckf_block_threads<8>()), ckf_block_threads<8>(), 0, st>>>(g, c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ gather for the final fit

__global__ void gather_count_kernel(int n, int n_layers, const int32_t *__restrict__ hit_idx, int32_t *cnt)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int c = 3;
    for (int L = 3; L < n_layers; ++L) c += hit_idx[(size_t)L * n + t] >= 0;
    cnt[t] = c;
}

// exclusive scan of n counts into off[0..n] (off[n] = total); one block per 1024 entries,
// then a single-block pass over block sums, then a fix-up (n <= 1024 * 1024 * 64)
__global__ void __launch_bounds__(1024) block_scan_kernel(int n, const int32_t *__restrict__ in,
                                                          int32_t *__restrict__ out, int32_t *__restrict__ bsum)
{
    __shared__ int32_t wt[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t v = i < n ? in[i] : 0, x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t y = wt[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t o = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += o;
        }
        wt[lane] = y;
    }
    __syncthreads();
    const int32_t incl = x + (wid > 0 ? wt[wid - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}
__global__ void bsum_scan_kernel(int nb, int32_t *bsum)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t acc = 0;
        for (int i = 0; i < nb; ++i) {
            int32_t v = bsum[i];
            bsum[i] = acc;
            acc += v;
        }
        bsum[nb] = acc;
    }
}
__global__ void add_bsum_kernel(int n, int32_t *out, const int32_t *__restrict__ bsum, int nb)
{
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
    if (i == 0) out[n] = bsum[nb];
}

__global__ void gather_fill_kernel(int n, int n_events, int n_layers, const LayerDev *__restrict__ layers,
                                   const int32_t *__restrict__ eoff, const float *__restrict__ seed_hits,
                                   const int32_t *__restrict__ hit_idx, const int32_t *__restrict__ off,
                                   uint8_t *lay_out, float *xo, float *yo, float *zo)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int e = find_event(eoff, n_events, t);
    const LayerDev *lays = layers + (size_t)e * n_layers;
    int o = off[t];
    for (int k = 0; k < 3; ++k) {
        lay_out[o] = (uint8_t)lays[k].surface;
        xo[o] = seed_hits[(3 * k + 0) * n + t];
        yo[o] = seed_hits[(3 * k + 1) * n + t];
        zo[o] = seed_hits[(3 * k + 2) * n + t];
        ++o;
    }
    for (int L = 3; L < n_layers; ++L) {
        const int h = hit_idx[(size_t)L * n + t];
        if (h < 0) continue;
        const LayerDev ly = lays[L];
        lay_out[o] = (uint8_t)ly.surface;
        xo[o] = ly.x[h];
        yo[o] = ly.y[h];
        zo[o] = ly.z[h];
        ++o;
    }
}

size_t gather_scratch_bytes(int n) { return ((size_t)n + (size_t)(n / 1024 + 2)) * sizeof(int32_t) + 256; }

cudaError_t launch_scan_counts(int n, const int32_t *cnt, int32_t *off_out, int32_t *bsum, cudaStream_t st)
{
    if (n <= 0) return cudaMemsetAsync(off_out, 0, sizeof(int32_t), st);
    const int nb = (n + 1023) / 1024;
    block_scan_kernel<<<nb, 1024, 0, st>>>(n, cnt, off_out, bsum);
    bsum_scan_kernel<<<1, 32, 0, st>>>(nb, bsum);
    add_bsum_kernel<<<nb, 1024, 0, st>>>(n, off_out, bsum, nb);
    return cudaGetLastError();
}

cudaError_t launch_gather(int n, int n_events, int n_layers, const LayerDev *layers, const int32_t *event_off,
                          const float *seed_hits, const int32_t *hit_idx, int32_t *off_out, uint8_t *layer_out,
                          float *x_out, float *y_out, float *z_out, void *scratch, cudaStream_t st)
{
    if (n <= 0) return cudaMemsetAsync(off_out, 0, sizeof(int32_t), st);
    int32_t *cnt = reinterpret_cast<int32_t *>(scratch);
    const int nb = (n + 1023) / 1024;
    int32_t *bsum = cnt + n;
    gather_count_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, n_layers, hit_idx, cnt);
    block_scan_kernel<<<nb, 1024, 0, st>>>(n, cnt, off_out, bsum);
    bsum_scan_kernel<<<1, 32, 0, st>>>(nb, bsum);
    add_bsum_kernel<<<nb, 1024, 0, st>>>(n, off_out, bsum, nb);
    gather_fill_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, n_events, n_layers, layers, event_off, seed_hits,
                                                        hit_idx, off_out, layer_out, x_out, y_out, z_out);
    return cudaGetLastError();
}

}  // namespace kfd
