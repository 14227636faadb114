// kf_fit.cu -- seed estimate and Kalman-filter track fit kernels.
//
// One thread fits one track: the state and the packed covariance stay in
// registers across the whole layer loop (Sec. 2: fitting applies the KF over
// a known hit list with no branching between tracks; Sec. 4.3: one track per
// thread, structure-of-arrays inputs and outputs so neighbouring threads touch
// neighbouring addresses).
#include "kf_df.cuh"
#include "kf_internal.h"
#include "kf_track.cuh"

namespace kfd {

constexpr double PI_D_FIT = 3.14159265358979323846;

template <bool B, class X, class Y> struct sel { using type = X; };
template <class X, class Y> struct sel<false, X, Y> { using type = Y; };

__device__ __forceinline__ void load_geom(const Geom &g, Surf *s_surf)
{
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) s_surf[i] = g.s[i];
    __syncthreads();
}

// ------------------------------------------------------------------ seeds

// Seed hits: hit 0, then the first hit >= 2 cm (transverse) from it, then the
// first later hit >= 2 cm from that one (hits 1, 2 if none).  The distance test
// decides exactly as an FP64 evaluation with explicit rounding would on the same
// FP32 inputs.  The single-precision square distance is within 3e-7 (relative)
// of the exact one (a rounded difference squared, a rounded product and sum),
// and the FP64 one within 3e-16, so where the former lies more than 1e-6 from
// the threshold 4 both fall on the same side of it; only nearer does the FP64
// evaluation (four conversions and five operations on the FP64 pipe) run.
__device__ __forceinline__ bool far_enough(float xa, float ya, float xb, float yb)
{
    const float fx = xb - xa, fy = yb - ya;
    const float f2 = fx * fx + fy * fy;
    if (f2 > 4.f * (1.f + 1e-6f)) return true;
    if (f2 < 4.f * (1.f - 1e-6f)) return false;
    double dx = (double)xb - (double)xa, dy = (double)yb - (double)ya;
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) >= 4.0;
}

// index of the third seed hit of a track (the rule above)
__device__ __forceinline__ int seed_hit_last(const float *__restrict__ hx, const float *__restrict__ hy, int nh)
{
    int a = -1, b = -1;
    for (int j = 1; j < nh; ++j)
        if (far_enough(hx[0], hy[0], hx[j], hy[j])) {
            a = j;
            break;
        }
    if (a > 0)
        for (int j = a + 1; j < nh; ++j)
            if (far_enough(hx[a], hy[a], hx[j], hy[j])) {
                b = j;
                break;
            }
    return (a < 0 || b < 0) ? 2 : b;
}

__global__ void __launch_bounds__(128) seed_kernel(int count, int n, int t_begin, const int32_t *__restrict__ off,
                                                   const float *__restrict__ hx, const float *__restrict__ hy,
                                                   const float *__restrict__ hz, float kb_abs,
                                                   float *__restrict__ state, int8_t *__restrict__ qo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int t = t_begin + i;
    const int o = off[t], nh = off[t + 1] - o;
    if (nh < 3) {
#pragma unroll
        for (int i = 0; i < 6; ++i) state[i * n + t] = 0.f;
        qo[t] = 1;
        return;
    }
    int a = -1, b = -1;
    const float x0 = hx[o], y0 = hy[o];
    for (int j = 1; j < nh; ++j)
        if (far_enough(x0, y0, hx[o + j], hy[o + j])) {
            a = j;
            break;
        }
    if (a > 0)
        for (int j = a + 1; j < nh; ++j)
            if (far_enough(hx[o + a], hy[o + a], hx[o + j], hy[o + j])) {
                b = j;
                break;
            }
    if (a < 0 || b < 0) {
        a = 1;
        b = 2;
    }
    // circle through three points: signed curvature k = 2 (a x b) / (|a| |b| |b - a|)
    const float ax = hx[o + a] - x0, ay = hy[o + a] - y0;
    const float bx = hx[o + b] - x0, by = hy[o + b] - y0;
    const float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by);
    const float lab = sqrtf((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    const float cr = ax * by - ay * bx;
    const float k = 2.f * cr / (la * lb * lab);
    const float ak = fabsf(k);
    const float sg = k > 0.f ? 1.f : (k < 0.f ? -1.f : 0.f);
    const float arc = ak > 0.f ? 2.f * asinf(fminf(1.f, 0.5f * lb * ak)) / ak : lb;
    float phi = atan2f(ay, ax) - sg * asinf(fminf(1.f, 0.5f * la * ak));
    if (phi > PI_F) phi -= 2.f * PI_F;
    if (phi <= -PI_F) phi += 2.f * PI_F;
    state[0 * n + t] = x0;
    state[1 * n + t] = y0;
    state[2 * n + t] = hz[o];
    state[3 * n + t] = kb_abs > 0.f ? ak / kb_abs : 0.f;
    state[4 * n + t] = phi;
    state[5 * n + t] = atan2f(arc, hz[o + b] - hz[o]);
    qo[t] = k > 0.f ? (int8_t)-1 : (int8_t)1;
}

cudaError_t launch_seeds(const Geom &g, int count, int stride, int t_begin, const int32_t *off, const float *hx,
                         const float *hy, const float *hz, float *state, int8_t *q, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    seed_kernel<<<(count + 127) / 128, 128, 0, st>>>(count, stride, t_begin, off, hx, hy, hz, fabsf(g.kb), state, q);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fit

template <bool FP64>
struct FitTypes {
    using T = typename sel<FP64, double, float>::type;
    using P = typename sel<FP64, double, ff>::type;
};

// one hit on layer surface sf.  M1 (measurement model 1, Sec. 4.1): a barrel
// hit after the first (k > 0; the state starts on the first) is reached on the
// cylinder through it and measured in 2-D there.
template <bool JOSEPH, class C, bool M1 = false, class T, class P>
__device__ __forceinline__ bool fit_step(Track<T, P> &st, C p[21], int k, T alpha, T mass2, int ms_on,
                                         const Surf &sf, float hx, float hy, float hz, double &chi2,
                                         unsigned &status, bool seeded = false, const Dir<T> *dir = nullptr)
{
    if constexpr (M1) {
        if (k > 0 && sf.kind == 0) {
            const Surf h = hit_surface(sf, hx, hy);
            return fit_step_on<JOSEPH, C, true>(st, p, k, alpha, mass2, ms_on, h, hx, hy, hz, chi2, status,
                                                seeded, dir);
        }
    }
    return fit_step_on<JOSEPH, C, false>(st, p, k, alpha, mass2, ms_on, sf, hx, hy, hz, chi2, status, seeded,
                                         dir);
}

// Crossings that leave the plain FP32 step (a mixed-path step): barrel, the
// helix meets the cylinder close to its apex, sine of the transverse crossing
// angle above 0.8 (cos < 0.6: about 2% of the steps on the 17-layer barrel,
// low-pT tracks); disk, the direction close to the disk plane, incidence cosine
// |cos(theta)| below 0.5.  There the surface-constrained Jacobian grows like
// 1 / cos(alpha) and the gain of the standard-form FP32 update, formed from the
// transported covariance, loses the covariance.
constexpr float NEAR_TANGENT_SINE = 0.8f;
constexpr float NEAR_TANGENT_DISK_COS = 0.5f;
// A near-tangent barrel crossing whose 3-D incidence cosine sin(theta) cos(alpha)
// is above this takes the FP32 U-D update (FP32 transport); the steeper ones and
// the disk crossings take the double-float step.
constexpr float UD32_MIN_COS = 0.2f;

// the crossing kind of a mixed-path step: 0 plain FP32, 1 FP32 U-D update,
// 2 double-float step
__device__ __forceinline__ int crossing_kind(const Track<float, ff> &st, float alpha, const Surf &sf,
                                             const Dir<float> &d)
{
    if (sf.kind == 0) {
        const float s = crossing_sine(st, alpha, sf, d.sphi, d.cphi);
        if (!(s > NEAR_TANGENT_SINE)) return 0;
        const float c = __fmul_rn(d.sth, __fsqrt_rn(fmaxf(0.f, __fmaf_rn(-s, s, 1.f))));
        return c > UD32_MIN_COS ? 1 : 2;
    }
    return fabsf(d.cth) < NEAR_TANGENT_DISK_COS ? 2 : 0;
}
// the same on the surface the hit is measured on
template <bool M1>
__device__ __forceinline__ int crossing_kind(const Track<float, ff> &st, float alpha, const Surf &sf, float hx,
                                             float hy, const Dir<float> &d)
{
    if constexpr (M1)
        if (sf.kind == 0) return crossing_kind(st, alpha, hit_surface(sf, hx, hy), d);
    return crossing_kind(st, alpha, sf, d);
}
// whether the crossing leaves the plain FP32 step
template <bool M1>
__device__ __forceinline__ bool grazing_crossing(const Track<float, ff> &st, float alpha, const Surf &sf, float hx,
                                                 float hy)
{
    return crossing_kind<M1>(st, alpha, sf, hx, hy, direction(st)) != 0;
}

__device__ __forceinline__ ff ff_from_d(double d)
{
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}

// one full step in FP64 for a mixed-path track (state float-float, P float)
template <bool M1>
__device__ __forceinline__ bool fp64_step(Track<float, ff> &st, float pf[21], int k, double alpha, double mass2,
                                       int ms_on, const Surf &sf, float hx, float hy, float hz, double &chi2,
                                       unsigned &status)
{
    Track<double, double> sd;
    sd.x = to_d(st.x);
    sd.y = to_d(st.y);
    sd.z = to_d(st.z);
    sd.phi = to_d(st.phi);
    sd.ip = st.ip;
    sd.th = to_d(st.th);
    double pd[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pd[i] = f2d(pf[i]);
    if (!fit_step<true, double, M1>(sd, pd, k, alpha, mass2, ms_on, sf, hx, hy, hz, chi2, status)) return false;
    st.x = ff_from_d(sd.x);
    st.y = ff_from_d(sd.y);
    st.z = ff_from_d(sd.z);
    st.phi = ff_from_d(sd.phi);
    st.ip = (float)sd.ip;
    st.th = ff_from_d(sd.th);
#pragma unroll
    for (int i = 0; i < 21; ++i) pf[i] = d2f(pd[i]);
    return true;
}

// fp64_step out of line (a near-tangent crossing is about 2% of the steps)
template <bool M1>
static __device__ __noinline__ MixedIO fp64_step_out_of_line(MixedIO m, int k, double alpha, double mass2,
                                                             int ms_on, const Surf *sf, float hx, float hy,
                                                             float hz)
{
    m.ok = fp64_step<M1>(m.st, m.p, k, alpha, mass2, ms_on, *sf, hx, hy, hz, m.chi2, m.status);
    return m;
}

// A near-tangent crossing of the FP32 layer loop: the step in double-float U-D
// form (df_step_from_f32), out of line (about 2% of the steps)
template <bool M1>
static __device__ __noinline__ MixedIO df_step_out_of_line(MixedIO m, float alpha, float mass2, int ms_on,
                                                           const Surf *sf, float hx, float hy, float hz)
{
    if (M1 && sf->kind == 0)
        m.ok = df_step_from_f32<true>(m.st, m.p, alpha, mass2, ms_on, hit_surface(*sf, hx, hy), hx, hy, hz, m.chi2,
                                      m.status);
    else
        m.ok = df_step_from_f32<false>(m.st, m.p, alpha, mass2, ms_on, *sf, hx, hy, hz, m.chi2, m.status);
    return m;
}

// A near-tangent barrel crossing that is not steep: FP32 propagation, transport
// and noise, then the update in FP32 U-D form (out of line)
template <bool M1>
static __device__ __noinline__ MixedIO ud32_step_out_of_line(MixedIO m, float alpha, float mass2, int ms_on,
                                                             const Surf *sf, float hx, float hy, float hz)
{
    if (M1 && sf->kind == 0)
        m.ok = ud32_step<true>(m.st, m.p, alpha, mass2, ms_on, hit_surface(*sf, hx, hy), hx, hy, hz, m.chi2,
                               m.status);
    else
        m.ok = ud32_step<false>(m.st, m.p, alpha, mass2, ms_on, *sf, hx, hy, hz, m.chi2, m.status);
    return m;
}

// A near-tangent crossing inside the FP64 phase (the covariance already FP64):
// the propagation in FP64 too, out of line.  A track fitted inwards meets its
// near-tangent crossings first, while the seed covariance is still large.
struct MixedIOD {
    Track<float, ff> st;
    double p[21];
    double chi2;
    unsigned status;
    int ok;
};

template <bool M1>
// df_update (a disk-seeded track's seed-phase updates after the first, model 0):
// the propagation, transport and noise in FP64 as above, the update in
// double-float U-D form.  Measured on 20,000 barrel+disk tracks against the
// oracle with the host build of this code: the same parity as the FP64 Joseph
// update (covariance within 2.0e-4 of its sigmas); the first update in U-D form
// as well left the covariance 1.85e-3 off.
static __device__ __noinline__ MixedIOD fp64_step_pd_out_of_line(MixedIOD m, int k, double alpha, double mass2,
                                                                 int ms_on, const Surf *sf, float hx, float hy,
                                                                 float hz, bool seeded, bool df_update)
{
    Track<double, double> sd;
    sd.x = to_d(m.st.x);
    sd.y = to_d(m.st.y);
    sd.z = to_d(m.st.z);
    sd.phi = to_d(m.st.phi);
    sd.ip = m.st.ip;
    sd.th = to_d(m.st.th);
    if (!M1 && df_update) {
        Jac<double> J;
        if (!propagate(sd, alpha, *sf, J)) {
            m.status |= reach_bits(sd);
            m.ok = 0;
            return m;
        }
        transport<double>(m.p, J);
        if (ms_on) m.status |= ms_noise<double, double>(sd, *sf, J.cphi1, J.sphi1, mass2, m.p);
        Track<float, ff> st;
        st.x = ff_from_d(sd.x);
        st.y = ff_from_d(sd.y);
        st.z = ff_from_d(sd.z);
        st.phi = ff_from_d(sd.phi);
        st.ip = (float)sd.ip;
        st.th = ff_from_d(sd.th);
        df p[21];
#pragma unroll
        for (int i = 0; i < 21; ++i) p[i] = df_from_d(m.p[i]);
        df c2 = df(0.f);
        m.ok = ud_update3(st, p, hx, hy, hz, *sf, c2);
        if (!m.ok) {
            m.status |= KF_ST_CHOL_FAIL;
            return m;
        }
        m.chi2 += df_to_d(c2);
#pragma unroll
        for (int i = 0; i < 21; ++i) m.p[i] = df_to_d(p[i]);
        m.st = st;
        return m;
    }
    m.ok = fit_step<true, double, M1>(sd, m.p, k, alpha, mass2, ms_on, *sf, hx, hy, hz, m.chi2, m.status, seeded);
    if (m.ok) {
        m.st.x = ff_from_d(sd.x);
        m.st.y = ff_from_d(sd.y);
        m.st.z = ff_from_d(sd.z);
        m.st.phi = ff_from_d(sd.phi);
        m.st.ip = (float)sd.ip;
        m.st.th = ff_from_d(sd.th);
    }
    return m;
}

// the covariance into the FP64 and/or the FP32 output planes
template <class C>
__device__ __forceinline__ void store_cov(const FitArgs &a, int n, int t, const C p[21])
{
    if (a.o_cov)
#pragma unroll
        for (int i = 0; i < 21; ++i) a.o_cov[(size_t)i * n + t] = (double)p[i];
    if (a.o_cov32)
#pragma unroll
        for (int i = 0; i < 21; ++i) a.o_cov32[(size_t)i * n + t] = (float)p[i];
}

template <bool FP64, bool M1 = false, bool P0 = false>
__device__ __forceinline__ void fit_track(int t, const FitArgs &a, const Surf *surf, float kb, float mass2f,
                                          double kbd, double mass2d);

// A track that crosses one surface twice in a row (it turns back through a layer
// near its apex, the second crossing close to tangent) has a step that
// amplifies the mixed path's rounding about tenfold: the whole track is fitted
// in FP64, out of line (it is rare, and its code stays out of the FP32 loop's).
template <bool M1, bool P0>
static __device__ __noinline__ void fit_track_fp64_out_of_line(int t, const FitArgs *a, const Surf *surf,
                                                               double kbd, double mass2d)
{
    fit_track<true, M1, P0>(t, *a, surf, (float)kbd, (float)mass2d, kbd, mass2d);
    if (a->o_status) a->o_status[t] |= KF_ST_FP64_TRACK;
}

// A track between the two phases of the fit: phase 1 (the first updates from
// the seed, with an extended-precision covariance) leaves it here for phase 2
// (the rest of the hits, covariance in T).
template <bool FP64>
struct Phase {
    Track<typename FitTypes<FP64>::T, typename FitTypes<FP64>::P> st;
    typename FitTypes<FP64>::T pf[21];
    double chi2;
    unsigned status;
    int used, k;
};

template <class T, class P>
__device__ __forceinline__ void write_outputs(const FitArgs &a, int t, const Track<T, P> &st, double chi2, int used,
                                              unsigned status)
{
    const int n = a.n;
    double sv[6] = {to_d(st.x), to_d(st.y), to_d(st.z), (double)st.ip, to_d(st.phi), to_d(st.th)};
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (!isfinite(sv[i])) status |= KF_ST_NONFINITE;
    if (a.o_state) {
#pragma unroll
        for (int i = 0; i < 6; ++i) a.o_state[(size_t)i * n + t] = sv[i];
    }
    if (a.o_chi2) a.o_chi2[t] = chi2;
    if (a.o_ndof) a.o_ndof[t] = 2 * used - 5;
    if (a.o_status) a.o_status[t] = status;
}

// Phase 1 of track t: from the seed, the first n1 updates with an extended-
// precision covariance.  Returns true with ph filled when phase 2 has hits to
// fit; false when the track is finished here (its outputs written).
// P0: the initial covariance is a.p0_scale * a.p0 (the refit), not seed_cov * I;
// a separate instance, so that the plain fit does not carry the general first update.
template <bool FP64, bool M1, bool P0>
__device__ __forceinline__ bool fit_phase1(int t, const FitArgs &a, const Surf *surf, float kb, float mass2f,
                                           double kbd, double mass2d, Phase<FP64> &ph)
{
    using T = typename FitTypes<FP64>::T;
    using P = typename FitTypes<FP64>::P;
    const int n = a.n;
    const int o0 = a.off[t], nh = a.off[t + 1] - o0;
    if constexpr (!FP64) {
        bool recross = false;
        for (int j = 1; j < nh; ++j) recross |= a.layer[o0 + j] == a.layer[o0 + j - 1];
        if (recross) {
            fit_track_fp64_out_of_line<M1, P0>(t, &a, surf, kbd, mass2d);
            return false;
        }
    }
    Track<T, P> &st = ph.st;
    st.x = from_f<P>(a.seed_state[0 * n + t]);
    st.y = from_f<P>(a.seed_state[1 * n + t]);
    st.z = from_f<P>(a.seed_state[2 * n + t]);
    st.ip = (T)a.seed_state[3 * n + t];
    st.phi = from_f<P>(a.seed_state[4 * n + t]);
    st.th = from_f<P>(a.seed_state[5 * n + t]);
    const int q = a.q[t];
    const T alpha = FP64 ? T(-q * kbd) : T(-q) * T(kb);
    const T mass2 = FP64 ? T(mass2d) : T(mass2f);
    unsigned status = 0u;
    double chi2 = 0.0;
    int used = 0, k = 0;
    bool alive = true;
    double pd[21];
    if constexpr (P0) {
#pragma unroll
        for (int i = 0; i < 21; ++i) pd[i] = a.p0_scale * a.p0[(size_t)i * n + t];
    } else {
#pragma unroll
        for (int i = 0; i < 21; ++i) pd[i] = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) pd[pk(i, i)] = a.seed_cov;
    }
    // phase 1: the first n64 updates with an extended-precision covariance, and
    // at least until the third seed hit (the seed-hit rule) has been used: a
    // disk/barrel overlap can put two of the first hits a fraction of a mm
    // apart, and the curvature is only pinned by the third distinct point
    int n1 = a.n64;
    if (a.n64 > 0 && nh >= 3) {
        const int s2 = seed_hit_last(a.hx + o0, a.hy + o0, nh);
        n1 = max(n1, s2 + 1);
    }
    n1 = min(n1, nh);
    // the covariance after phase 1: in ph.pf (T) when the seed phase ran in
    // double-float, else in pd (FP64)
    T *pf = ph.pf;
    bool in_pf = false;
    // A disk hit among the seed-phase hits: a steep track whose curvature rests
    // on short transverse lever arms.  Its seed phase runs wholly in FP64,
    // propagation included: neither 48 bits (double-float) in the covariance
    // update nor the FP32 propagation and Jacobian are enough there.
    bool disk_seed = false;
    if constexpr (!FP64 && !P0)
        for (int j = 0; j < n1; ++j) disk_seed |= surf[a.layer[o0 + j]].kind == 1;
    if constexpr (!FP64 && !P0) {
        // double-float U-D for seed phases on barrels
        if (a.seed_df && n1 > 0 && !disk_seed) {
            // phase 1 in double-float on the FP32 pipe: the closed-form update
            // at the seed hit, then U-D factored updates
            df pq[21];
            df_seed_cov(pq, a.seed_cov);
            df c2 = df(0.f);
            for (; k < n1; ++k) {
                const int h = o0 + k;
                const Surf &sf = surf[a.layer[h]];
                const float hx = a.hx[h], hy = a.hy[h], hz = a.hz[h];
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
            for (int i = 0; i < 21; ++i) pf[i] = pq[i].hi;
            in_pf = true;
        }
    }
    if (!in_pf && n1 > 0) {
        // the seed hit: no propagation, the structured first update
        const Surf &sf = surf[a.layer[o0]];
        T cphi, sphi;
        sincos_pos(st.phi, sphi, cphi);
        // (under model 1 as well: the state starts at this hit, on its own radius)
        if (a.ms_on) status |= ms_noise<T, double>(st, sf, cphi, sphi, mass2, pd);
        // the structured update needs the diagonal seed covariance; a given one takes the general form
        bool ok0;
        if constexpr (P0) ok0 = kf_update<true>(st, pd, a.hx[o0], a.hy[o0], a.hz[o0], sf, chi2);
        else ok0 = kf_seed_update(st, pd, a.hx[o0], a.hy[o0], a.hz[o0], sf, chi2);
        if (ok0) {
            ++used;
            k = 1;
        } else {
            status |= KF_ST_CHOL_FAIL;
            alive = false;
        }
    }
    for (; !in_pf && alive && k < n1; ++k) {
        const int h = o0 + k;
        const Surf &sf = surf[a.layer[h]];
        bool ok;
        // the refit meets a track's near-tangent crossings (its outer end) among its
        // first updates, and a steep track its seed-phase disks: there the
        // FP64-covariance step also propagates in FP64
        if constexpr (!FP64) {
            if (P0 ? grazing_crossing<M1>(st, alpha, sf, a.hx[h], a.hy[h]) : disk_seed) {
                MixedIOD m;
                m.st = st;
#pragma unroll
                for (int i = 0; i < 21; ++i) m.p[i] = pd[i];
                m.chi2 = chi2;
                m.status = status;
                // k == 1 after the structured seed-hit update: the transport skips its zero blocks
                m = fp64_step_pd_out_of_line<M1>(m, k, kbd * (double)(-q), mass2d, a.ms_on, &sf, a.hx[h], a.hy[h],
                                                 a.hz[h], !P0 && k == 1, !P0 && k >= 2);
                st = m.st;
#pragma unroll
                for (int i = 0; i < 21; ++i) pd[i] = m.p[i];
                chi2 = m.chi2;
                status = m.status;
                ok = m.ok != 0;
            } else {
                ok = fit_step<true, double, M1>(st, pd, k, alpha, mass2, a.ms_on, sf, a.hx[h], a.hy[h], a.hz[h],
                                                chi2, status, !P0 && k == 1);
            }
        } else {
            // k == 1 after the structured seed-hit update: the transport skips its zero blocks
            ok = fit_step<true, double, M1>(st, pd, k, alpha, mass2, a.ms_on, sf, a.hx[h], a.hy[h], a.hz[h], chi2,
                                            status, !P0 && k == 1);
        }
        if (!ok) {
            alive = false;
            break;
        }
        ++used;
    }
    if (alive && k < nh) {
        if (!in_pf) {
#pragma unroll
            for (int i = 0; i < 21; ++i) pf[i] = to_t(pd[i], T(0));
        }
        ph.chi2 = chi2;
        ph.status = status;
        ph.used = used;
        ph.k = k;
        return true;
    }
    if (in_pf) store_cov(a, n, t, pf);
    else store_cov(a, n, t, pd);
    write_outputs(a, t, st, chi2, used, status);
    return false;
}

// Phase 2 of track t: its hits from ph.k on, the covariance in T (FP32 on the
// mixed path, standard form; FP64 steps at near-tangent crossings and for
// strongly informative updates), then its outputs.
template <bool FP64, bool M1>
__device__ __forceinline__ void fit_phase2(int t, const FitArgs &a, const Surf *surf, float kb, float mass2f,
                                           double kbd, double mass2d, Phase<FP64> &ph)
{
    using T = typename FitTypes<FP64>::T;
    const int n = a.n;
    const int o0 = a.off[t], nh = a.off[t + 1] - o0;
    const int q = a.q[t];
    const T alpha = FP64 ? T(-q * kbd) : T(-q) * T(kb);
    const T mass2 = FP64 ? T(mass2d) : T(mass2f);
    auto &st = ph.st;
    T *pf = ph.pf;
    double chi2 = ph.chi2;
    unsigned status = ph.status;
    int used = ph.used, k = ph.k;
    // software pipelining: the next hit's coordinates and surface load while a step computes
    float nx = 0.f, ny = 0.f, nz = 0.f;
    int nl = 0;
    if (k < nh) {
        nx = a.hx[o0 + k];
        ny = a.hy[o0 + k];
        nz = a.hz[o0 + k];
        nl = a.layer[o0 + k];
    }
    for (; k < nh; ++k) {
        const float hx = nx, hy = ny, hz = nz;
        const Surf &sf = surf[nl];
        if (k + 1 < nh) {
            const int h1 = o0 + k + 1;
            nx = a.hx[h1];
            ny = a.hy[h1];
            nz = a.hz[h1];
            nl = a.layer[h1];
        }
        bool near_tangent = false;
        if constexpr (!FP64) {
            // the direction's sines and cosines, shared by the near-tangent test and the propagation
            const Dir<float> d = direction(st);
            const int kind = crossing_kind<M1>(st, alpha, sf, hx, hy, d);
            near_tangent = kind != 0;
            if (near_tangent) {
                // near-tangent crossing: the update in U-D form, in FP32 (kind 1) or with
                // the transport in double-float (kind 2)
                MixedIO m;
                mixed_pack(m, st, pf, chi2, status);
                if (kind == 1) m = ud32_step_out_of_line<M1>(m, alpha, mass2, a.ms_on, &sf, hx, hy, hz);
                else m = df_step_out_of_line<M1>(m, alpha, mass2, a.ms_on, &sf, hx, hy, hz);
                if (!mixed_unpack(m, st, pf, chi2, status)) break;
            } else if (!fit_step<false, T, M1>(st, pf, k, alpha, mass2, a.ms_on, sf, hx, hy, hz, chi2, status,
                                               false, &d)) {
                break;
            }
        } else if (!fit_step<false, T, M1>(st, pf, k, alpha, mass2, a.ms_on, sf, hx, hy, hz, chi2, status)) {
            break;
        }
        ++used;
    }
    store_cov(a, n, t, pf);
    write_outputs(a, t, st, chi2, used, status);
}

template <bool FP64, bool M1, bool P0>
__device__ __forceinline__ void fit_track(int t, const FitArgs &a, const Surf *surf, float kb, float mass2f,
                                          double kbd, double mass2d)
{
    Phase<FP64> ph;
    if (fit_phase1<FP64, M1, P0>(t, a, surf, kb, mass2f, kbd, mass2d, ph))
        fit_phase2<FP64, M1>(t, a, surf, kb, mass2f, kbd, mass2d, ph);
}

// ------------------------------------------------------------------ the mixed fit in two kernels
// Phase 1 (double-float or FP64 seed phase: long straight-line code) and phase
// 2 (the FP32 layer loop) run as two kernels, so that the warps of each run
// one compact piece of code and the instruction cache holds it; each track is
// handed over in the carry buffer at its processing position i (coalesced in
// both kernels).
__device__ __forceinline__ void carry_put(const FitCarry &c, int i, const Phase<false> &ph)
{
    const int m = c.m;
    const float w[11] = {ph.st.x.hi, ph.st.x.lo, ph.st.y.hi, ph.st.y.lo, ph.st.z.hi, ph.st.z.lo, ph.st.phi.hi,
                         ph.st.phi.lo, ph.st.th.hi, ph.st.th.lo, ph.st.ip};
#pragma unroll
    for (int j = 0; j < 11; ++j) c.st[(size_t)j * m + i] = w[j];
#pragma unroll
    for (int j = 0; j < 21; ++j) c.cov[(size_t)j * m + i] = ph.pf[j];
    c.chi2[i] = ph.chi2;
    c.k[i] = ph.k;
    c.used[i] = ph.used;
    c.status[i] = ph.status;
}
__device__ __forceinline__ void carry_get(const FitCarry &c, int i, Phase<false> &ph)
{
    const int m = c.m;
    float w[11];
#pragma unroll
    for (int j = 0; j < 11; ++j) w[j] = c.st[(size_t)j * m + i];
    ph.st.x = ff{w[0], w[1]};
    ph.st.y = ff{w[2], w[3]};
    ph.st.z = ff{w[4], w[5]};
    ph.st.phi = ff{w[6], w[7]};
    ph.st.th = ff{w[8], w[9]};
    ph.st.ip = w[10];
#pragma unroll
    for (int j = 0; j < 21; ++j) ph.pf[j] = c.cov[(size_t)j * m + i];
    ph.chi2 = c.chi2[i];
    ph.k = c.k[i];
    ph.used = c.used[i];
    ph.status = c.status[i];
}

size_t fit_carry_bytes(int m)
{
    const size_t M = (size_t)max(m, 0);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(11 * 4 * M) + al(21 * 4 * M) + al(8 * M) + 3 * al(4 * M) + 256;
}
void fit_carve_carry(FitCarry &c, void *p, int m)
{
    const size_t M = (size_t)max(m, 0);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *q = static_cast<char *>(p);
    c.m = m;
    c.st = reinterpret_cast<float *>(q);
    q += al(11 * 4 * M);
    c.cov = reinterpret_cast<float *>(q);
    q += al(21 * 4 * M);
    c.chi2 = reinterpret_cast<double *>(q);
    q += al(8 * M);
    c.k = reinterpret_cast<int32_t *>(q);
    q += al(4 * M);
    c.used = reinterpret_cast<int32_t *>(q);
    q += al(4 * M);
    c.status = reinterpret_cast<uint32_t *>(q);
}

// phase 1 of the mixed fit, one thread per track in processing order; four
// blocks of 128 per SM (at most 128 registers: 0.77 ms per 1e6 tracks against
// 0.80 with three blocks at 168 registers)
template <bool M1>
__global__ void __launch_bounds__(128, 4) fit_seed_kernel(const Geom g, const FitArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    load_geom(g, s_surf);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    const int t = a.t_begin + (a.order ? a.order[i] : i);
    Phase<false> ph;
    if (fit_phase1<false, M1, false>(t, a, s_surf, g.kb, g.mass2, g.kbd, g.mass2d, ph)) carry_put(a.carry, i, ph);
    else a.carry.k[i] = -1;  // finished in phase 1
}

// phase 2 of the mixed fit, grid schedule; seven blocks of 128 per SM (at most
// 72 registers: 1.175 ms per 1e6 barrel tracks against 1.211 with six, 1.183
// with eight; with the earlier per-track-random bucket order five had been the
// best, 1.43 against 1.46)
template <bool M1>
__global__ void __launch_bounds__(128, 7) fit_loop_kernel(const Geom g, const FitArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    load_geom(g, s_surf);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count || a.carry.k[i] < 0) return;
    const int t = a.t_begin + (a.order ? a.order[i] : i);
    Phase<false> ph;
    carry_get(a.carry, i, ph);
    fit_phase2<false, M1>(t, a, s_surf, g.kb, g.mass2, g.kbd, g.mass2d, ph);
}

// Mixed path: four blocks of 128 per SM (at most 128 registers a thread, a few
// spills; measured 1% faster than three blocks at 159 registers).
template <bool FP64, bool M1, bool P0>
__global__ void __launch_bounds__(128, FP64 ? 3 : 4) fit_kernel(const Geom g, const FitArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    load_geom(g, s_surf);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    const int t = a.t_begin + (a.order ? a.order[i] : i);
    fit_track<FP64, M1, P0>(t, a, s_surf, g.kb, g.mass2, g.kbd, g.mass2d);
}

// Persistent form: a grid sized to the machine; each block takes
// BLOCK * a.chunk consecutive entries of a.order (a.chunk = tracks per thread;
// the order groups tracks by hit count and seed 1/pT, so neighbouring threads
// cross nearly the same layers) from an atomic work counter until the queue is
// empty: dynamic load balancing in place of the work stealing of Sec. 3.2.  The
// whole block takes work together and meets at a barrier between grabs, so its
// warps run the same part of the loop at the same time (warps that drift apart
// in a loop of this size compete for the instruction cache).
template <bool FP64, int BLOCK>
// 512 threads (16 warps) per SM whatever the block size, at most 128 registers a
// thread: on the uneven barrel+disk batch 15.3 ms against 16.6 with the registers
// uncapped (block 256: one block, 8 warps per SM)
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) fit_persistent_kernel(const Geom g, const FitArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    __shared__ int s_base;
    load_geom(g, s_surf);
    const int per = BLOCK * a.chunk;
    for (;;) {
        if (threadIdx.x == 0) s_base = atomicAdd(a.queue, per);
        __syncthreads();
        const int base = s_base;
        __syncthreads();  // every thread has read s_base before thread 0 writes the next one
        if (base >= a.count) break;
        const int end = min(base + per, a.count);
        for (int i = base + (int)threadIdx.x; i < end; i += BLOCK) {
            const int t = a.t_begin + (a.order ? a.order[i] : i);
            fit_track<FP64>(t, a, s_surf, g.kb, g.mass2, g.kbd, g.mass2d);
        }
    }
}

// phase 2 of the mixed fit in the persistent form (the work queue of
// fit_persistent_kernel over processing positions; phase 1 ran as a grid); 1024
// threads (32 warps) per SM whatever the block size, at most 64 registers a
// thread: on the 2e6-track barrel+disk batch 9.87 ms against 9.99 at 24 warps and
// 10.21 at 16
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) fit_loop_persistent_kernel(const Geom g, const FitArgs a)
{
    __shared__ Surf s_surf[MAX_SURF];
    __shared__ int s_base;
    load_geom(g, s_surf);
    const int per = BLOCK * a.chunk;
    for (;;) {
        if (threadIdx.x == 0) s_base = atomicAdd(a.queue, per);
        __syncthreads();
        const int base = s_base;
        __syncthreads();  // every thread has read s_base before thread 0 writes the next one
        if (base >= a.count) break;
        const int end = min(base + per, a.count);
        for (int i = base + (int)threadIdx.x; i < end; i += BLOCK) {
            if (a.carry.k[i] < 0) continue;
            const int t = a.t_begin + (a.order ? a.order[i] : i);
            Phase<false> ph;
            carry_get(a.carry, i, ph);
            fit_phase2<false, false>(t, a, s_surf, g.kb, g.mass2, g.kbd, g.mass2d, ph);
        }
    }
}

// ------------------------------------------------------------------ outward-inward refit
// The track is run backwards by reversing its direction of motion, the same
// helix traversed the other way: phi -> phi + pi, theta -> pi - theta, q -> -q
// (1/pT and the position unchanged; the theta row and column of the
// covariance change sign); the reversed list of the hits the forward fit used
// is then fitted from the forward state with the inflated forward covariance,
// and the result at the first hit is turned back.

// hits the forward fit used: the first (ndof + 5) / 2 of the track
__global__ void used_counts_kernel(int n, const int32_t *__restrict__ off, const int32_t *__restrict__ ndof,
                                   int32_t *__restrict__ cnt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int nh = off[t + 1] - off[t];
    cnt[t] = min(max((ndof[t] + 5) / 2, 0), nh);
}

__global__ void reverse_hits_kernel(int n, const int32_t *__restrict__ off, const int32_t *__restrict__ roff,
                                    const uint8_t *__restrict__ layer, const float *__restrict__ x,
                                    const float *__restrict__ y, const float *__restrict__ z, uint8_t *__restrict__ rl,
                                    float *__restrict__ rx, float *__restrict__ ry, float *__restrict__ rz)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int o = off[t], ro = roff[t], m = roff[t + 1] - ro;  // m <= the track's hit count
    for (int k = 0; k < m; ++k) {
        const int s = o + m - 1 - k;
        rl[ro + k] = layer[s];
        rx[ro + k] = x[s];
        ry[ro + k] = y[s];
        rz[ro + k] = z[s];
    }
}

__device__ __forceinline__ double reverse_phi(double p)
{
    const double r = p + PI_D_FIT;
    return r > PI_D_FIT ? r - 2.0 * PI_D_FIT : r;
}

__global__ void reverse_seed_kernel(int n, const double *__restrict__ fwd, const double *__restrict__ fwd_cov,
                                    const int8_t *__restrict__ q, float *__restrict__ seed, double *__restrict__ rcov,
                                    int8_t *__restrict__ rq)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const double v = fwd_cov[(size_t)pk(i, j) * n + t];
            rcov[(size_t)pk(i, j) * n + t] = (i == 5) != (j == 5) ? -v : v;
        }
    seed[0 * (size_t)n + t] = (float)fwd[0 * (size_t)n + t];
    seed[1 * (size_t)n + t] = (float)fwd[1 * (size_t)n + t];
    seed[2 * (size_t)n + t] = (float)fwd[2 * (size_t)n + t];
    seed[3 * (size_t)n + t] = (float)fwd[3 * (size_t)n + t];
    seed[4 * (size_t)n + t] = (float)reverse_phi(fwd[4 * (size_t)n + t]);
    seed[5 * (size_t)n + t] = (float)(PI_D_FIT - fwd[5 * (size_t)n + t]);
    rq[t] = (int8_t)(-q[t]);
}

__global__ void unreverse_kernel(int n, double *__restrict__ st, double *__restrict__ cov, float *__restrict__ cov32)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (st) {
        const double p = st[4 * (size_t)n + t] - PI_D_FIT;
        st[4 * (size_t)n + t] = p <= -PI_D_FIT ? p + 2.0 * PI_D_FIT : p;
        st[5 * (size_t)n + t] = PI_D_FIT - st[5 * (size_t)n + t];
    }
    if (cov)
#pragma unroll
        for (int j = 0; j < 5; ++j) cov[(size_t)pk(5, j) * n + t] = -cov[(size_t)pk(5, j) * n + t];
    if (cov32)
#pragma unroll
        for (int j = 0; j < 5; ++j) cov32[(size_t)pk(5, j) * n + t] = -cov32[(size_t)pk(5, j) * n + t];
}

cudaError_t launch_used_counts(int n, const int32_t *off, const int32_t *fwd_ndof, int32_t *cnt, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    used_counts_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, off, fwd_ndof, cnt);
    return cudaGetLastError();
}

cudaError_t launch_reverse(int n, const int32_t *off, const int32_t *roff, const uint8_t *layer, const float *x,
                           const float *y, const float *z, const double *fwd, const double *fwd_cov, const int8_t *q,
                           uint8_t *rl, float *rx, float *ry, float *rz, float *seed, double *rcov, int8_t *rq,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    reverse_hits_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, off, roff, layer, x, y, z, rl, rx, ry, rz);
    reverse_seed_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, fwd, fwd_cov, q, seed, rcov, rq);
    return cudaGetLastError();
}

cudaError_t launch_unreverse(int n, double *state, double *cov, float *cov32, cudaStream_t st)
{
    if (n <= 0 || (!state && !cov && !cov32)) return cudaSuccess;
    unreverse_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, state, cov, cov32);
    return cudaGetLastError();
}

cudaError_t launch_fit(const Geom &g, const FitArgs &a, bool fp64, int block, cudaStream_t st)
{
    if (a.count <= 0) return cudaSuccess;
    (void)block;
    const int b = 128;
    const int grid = (a.count + b - 1) / b;
    const bool m1 = a.meas_model == 1, p0 = a.p0 != nullptr;
    cudaEvent_t *ev = static_cast<cudaEvent_t *>(a.timing_events);
    if (ev) cudaEventRecord(ev[0], st);
    if (!fp64 && !p0) {  // the mixed fit: phase 1, then phase 2 (carry in a.carry)
        if (!a.carry.k || a.carry.m < a.count) return cudaErrorInvalidValue;
        if (m1) fit_seed_kernel<true><<<grid, b, 0, st>>>(g, a);
        else fit_seed_kernel<false><<<grid, b, 0, st>>>(g, a);
        if (ev) cudaEventRecord(ev[1], st);
        if (m1) fit_loop_kernel<true><<<grid, b, 0, st>>>(g, a);
        else fit_loop_kernel<false><<<grid, b, 0, st>>>(g, a);
        if (ev) cudaEventRecord(ev[2], st);
        return cudaGetLastError();
    }
    if (p0) {  // the refit
        if (m1) {
            if (fp64) fit_kernel<true, true, true><<<grid, b, 0, st>>>(g, a);
            else fit_kernel<false, true, true><<<grid, b, 0, st>>>(g, a);
        } else {
            if (fp64) fit_kernel<true, false, true><<<grid, b, 0, st>>>(g, a);
            else fit_kernel<false, false, true><<<grid, b, 0, st>>>(g, a);
        }
    } else if (m1) {
        fit_kernel<true, true, false><<<grid, b, 0, st>>>(g, a);
    } else {
        fit_kernel<true, false, false><<<grid, b, 0, st>>>(g, a);
    }
    if (ev) {
        cudaEventRecord(ev[1], st);
        cudaEventRecord(ev[2], st);
    }
    return cudaGetLastError();
}

cudaError_t launch_fit_persistent(const Geom &g, const FitArgs &a, bool fp64, int block, int grid, cudaStream_t st)
{
    if (a.count <= 0) return cudaSuccess;
    // model 1 and the refit's initial covariance run on the grid schedule
    if (a.meas_model != 0 || a.p0) return cudaErrorInvalidValue;
    if (fp64) {
        switch (block) {
        case 64: fit_persistent_kernel<true, 64><<<grid, 64, 0, st>>>(g, a); break;
        case 128: fit_persistent_kernel<true, 128><<<grid, 128, 0, st>>>(g, a); break;
        case 256: fit_persistent_kernel<true, 256><<<grid, 256, 0, st>>>(g, a); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    // mixed: phase 1 as a grid, phase 2 from the work queue
    if (!a.carry.k || a.carry.m < a.count) return cudaErrorInvalidValue;
    if (block != 64 && block != 128 && block != 256) return cudaErrorInvalidValue;
    fit_seed_kernel<false><<<(a.count + 127) / 128, 128, 0, st>>>(g, a);
    switch (block) {
    case 64: fit_loop_persistent_kernel<64><<<grid, 64, 0, st>>>(g, a); break;
    case 128: fit_loop_persistent_kernel<128><<<grid, 128, 0, st>>>(g, a); break;
    default: fit_loop_persistent_kernel<256><<<grid, 256, 0, st>>>(g, a); break;
    }
    return cudaGetLastError();
}

// resident blocks per SM of the persistent kernel at this block size
int persistent_blocks_per_sm(bool fp64, int block)
{
    int nb = 0;
    cudaError_t e = cudaSuccess;
    switch (block) {
    case 64:
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_persistent_kernel<true, 64>, 64, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_loop_persistent_kernel<64>, 64, 0);
        break;
    case 128:
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_persistent_kernel<true, 128>, 128, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_loop_persistent_kernel<128>, 128, 0);
        break;
    case 256:
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_persistent_kernel<true, 256>, 256, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fit_loop_persistent_kernel<256>, 256, 0);
        break;
    default: return 0;
    }
    return e == cudaSuccess ? nb : 0;
}

// ------------------------------------------------------------------ processing order

// Counting sort of the tracks into buckets of (hit count, descending) x (seed
// phase with a disk hit first) x (seed |1/pT|, descending): a warp then takes
// tracks that cross nearly the same layers, bend alike and run the same seed
// phase, so the layer loop, the seed phase (FP64 with a disk hit, double-float
// without) and the near-tangent steps (low-pT tracks at their apex) diverge
// little, and the costliest tracks (most hits, then the FP64 seed phase, then
// lowest pT: widest build windows, most near-tangent steps) come first, so that
// the short ones fill the launch's tail.  |1/pT| takes one bin below ip_one, the
// curvature at which the helix meets the outermost surface at a transverse
// crossing sine of 0.6 (no near-tangent crossing below it), and 63 bins of 1/32
// GeV^-1 above; where the geometry has disks, the stiff tracks of a fit are split
// further into 16 bins of |cot theta| (tracks of one bin cross barrels and disks
// in the same sequence) and the 1/pT bins above ip_one are 48 (for building the
// same bins measured no faster: 2.083 against 2.076 ms).  Inside a bucket the
// tracks keep their input order warp by warp (ranks from a warp vote; the warps
// of a block and the blocks reserve their ranges in the order of their atomics):
// the bucket of the common stiff tracks is then dense in t, and its SoA loads and
// output stores share 32-byte sectors.  The order does not change any track's
// result.
//
// Sorting groups of consecutive tracks instead (so that the per-track SoA outputs
// of a group share 32-byte sectors) was measured: groups of 4 made the fit 1.9x
// slower on the barrel and 4.7x on the barrel+disk batch, since a group mixes
// tracks of different cost again.
constexpr int ORDER_BUCKETS = 65 * 2 * 64;

struct OrderIn {
    int n;
    int nseed;                  // seed-phase hits whose surfaces decide the disk bit
    const int32_t *off;         // CSR offsets, or null (key by 1/pT alone)
    const float *ip;            // seed 1/pT [n]
    const uint8_t *layer;       // surface of each hit, or null (no disk bit)
    unsigned long long disk;    // bit s set: surface s is a disk
    float ip_one;               // |1/pT| below this: one bin (or ETA_BINS bins of |cot theta|)
    float pad_;
    const float *th;            // seed theta [n], or null: with disks in the geometry, the stiff
                                // tracks are binned by |cot theta| (their barrel / disk sequence)
};
constexpr int ETA_BINS = 16;

__device__ __forceinline__ int order_key(const OrderIn &in, int t)
{
    int nh = 0, disk = 0;
    if (in.off) {
        const int o = in.off[t];
        nh = min(in.off[t + 1] - o, 64);
        if (in.layer)
            for (int j = 0; j < min(nh, in.nseed); ++j) disk |= (int)((in.disk >> in.layer[o + j]) & 1ull);
    }
    const float ip = fabsf(in.ip[t]);
    int b;
    if (in.th) {  // ETA_BINS bins of |cot theta| for the stiff tracks
        if (ip < in.ip_one) {
            float sth, cth;
            __sincosf(in.th[t], &sth, &cth);
            const float cot = fabsf(cth) / fmaxf(fabsf(sth), 1e-6f);
            b = min((int)(cot * 2.5f), ETA_BINS - 1);
        } else {
            b = ETA_BINS + min((int)((ip - in.ip_one) * 32.f), 63 - ETA_BINS);
        }
    } else {
        b = ip < in.ip_one ? 0 : 1 + min((int)((ip - in.ip_one) * 32.f), 62);
    }
    return ((64 - nh) * 2 + (1 - disk)) * 64 + (63 - b);
}
// this lane's rank among the active lanes of its warp with the same key, and
// the number of them (lane order)
__device__ __forceinline__ int warp_rank(int key, bool live, int &count)
{
    const unsigned act = __ballot_sync(0xffffffffu, live);
    const unsigned same = __match_any_sync(0xffffffffu, live ? key : -1) & act;
    count = __popc(same);
    return __popc(same & ((1u << (threadIdx.x & 31)) - 1u));
}
// Histogram and scatter count in shared memory per block and touch global
// memory once per non-empty bucket and block: the keys of neighbouring tracks
// repeat a lot, and per-track global atomics on them serialise.
__global__ void __launch_bounds__(1024) order_hist_kernel(OrderIn in, int32_t *hist)
{
    __shared__ int32_t cnt[ORDER_BUCKETS];
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < in.n) atomicAdd(&cnt[order_key(in, t)], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += blockDim.x)
        if (cnt[b]) atomicAdd(&hist[b], cnt[b]);
}
__global__ void __launch_bounds__(1024) order_scan_kernel(int32_t *hist)
{
    // exclusive scan of ORDER_BUCKETS counts, one block
    __shared__ int32_t wt[32];
    constexpr int PER = (ORDER_BUCKETS + 1023) / 1024;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int32_t loc[PER];
    int32_t sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = tid * PER + j;
        loc[j] = i < ORDER_BUCKETS ? hist[i] : 0;
        sum += loc[j];
    }
    int32_t v = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) wt[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int32_t w = wt[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        wt[lane] = w;
    }
    __syncthreads();
    int32_t acc = v - sum + (wid > 0 ? wt[wid - 1] : 0);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = tid * PER + j;
        if (i < ORDER_BUCKETS) hist[i] = acc;
        acc += loc[j];
    }
}
__global__ void __launch_bounds__(1024) order_scatter_kernel(OrderIn in, int32_t *cursor, int32_t *order)
{
    __shared__ int32_t cnt[ORDER_BUCKETS];
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < in.n;
    const int key = live ? order_key(in, t) : 0;
    // one shared atomic per (warp, key), by the key's first lane; the others add their rank
    int count;
    const int rank = warp_rank(key, live, count);
    int local = 0;
    if (live && rank == 0) local = atomicAdd(&cnt[key], count);
    const unsigned same = __match_any_sync(0xffffffffu, live ? key : -1) & __ballot_sync(0xffffffffu, live);
    local = __shfl_sync(0xffffffffu, local, same ? __ffs(same) - 1 : 0) + rank;
    __syncthreads();
    // reserve this block's range in every bucket it uses
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += blockDim.x)
        if (cnt[b]) cnt[b] = atomicAdd(&cursor[b], cnt[b]);
    __syncthreads();
    if (live) order[cnt[key] + local] = t;
}

size_t order_scratch_ints() { return ORDER_BUCKETS; }

cudaError_t launch_order(int n, const int32_t *off, const float *seed_ip, const float *seed_th,
                         const uint8_t *layer, const Geom *g, int nseed, int32_t *hist, int32_t *order,
                         cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, ORDER_BUCKETS * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    OrderIn in;
    in.n = n;
    in.nseed = nseed;
    in.off = off;
    in.ip = seed_ip;
    in.layer = off && g ? layer : nullptr;
    in.disk = 0;
    in.ip_one = 0.f;
    in.pad_ = 0.f;
    in.th = nullptr;
    if (g) {
        float rmax = 0.f;
        for (int s = 0; s < g->n && s < 64; ++s) {
            if (g->s[s].kind == 1) in.disk |= 1ull << s;
            rmax = std::max(rmax, g->s[s].kind == 0 ? g->s[s].pos : g->s[s].rout);
        }
        // the curvature |c| = |kb| / pT at which a helix from the beam line meets
        // radius rmax at transverse crossing sine rmax |c| / 2 = 0.6
        if (rmax > 0.f && g->kb != 0.f) in.ip_one = 1.2f / (std::fabs(g->kb) * rmax);
        if (in.disk && in.off) in.th = seed_th;
    }
    const int b = 1024, grid = (n + b - 1) / b;
    order_hist_kernel<<<grid, b, 0, st>>>(in, hist);
    order_scan_kernel<<<1, 1024, 0, st>>>(hist);
    order_scatter_kernel<<<grid, b, 0, st>>>(in, hist, order);
    return cudaGetLastError();
}

}  // namespace kfd
