// kf_df.cuh -- the seed phase of the mixed-precision fit in double-float
// arithmetic on the FP32 pipe, with the covariance update in U-D factored form.
//
// Why.  Under the 1e4 seed covariance the first updates of a fit (Sec. 2: the
// KF starts from the seed's rough estimate) cancel eight to ten digits: the
// covariance-form update needs FP64 there, and on this GPU the FP64 pipe runs
// at 1/64 of the FP32 rate.  A double-float number -- an unevaluated sum
// hi + lo of two floats, about 48 significant bits -- is carried on the FP32
// pipe at about 6 to 15 FP32 instructions per operation.  48 bits are not
// enough for the covariance-form (Joseph) update, but they are for Bierman's
// U-D factored update: the covariance P = U D U^T (U unit upper triangular, D
// diagonal) is updated one scalar measurement at a time, the variances as
// d' = d r / (r + d f^2), a ratio of positive terms that cancels nothing.
// In exact arithmetic the result is the Kalman update of Sec. 2 / 4.1.
//
// The U-D order of the state is (1/pT, phi, theta, x, y, z): the measured
// position coordinates come last, so that a scalar measurement of a position
// direction touches only the last three columns of U.
#pragma once

#include "kf_track.cuh"

namespace kfd {

// ------------------------------------------------------------------ double-float
// Knuth's two-sum for the exact sum of the leading parts, Dekker-style exact
// products by FMA (the rounding error of a * b is fma(a, b, -a * b)), and a
// fast two-sum to renormalise.  The explicit _rn intrinsics keep the compiler
// from contracting a product into a later addition, which would break the
// error-free transformations.
struct df {
    float hi, lo;
    df() = default;
    __device__ __forceinline__ constexpr df(float h) : hi(h), lo(0.f) {}
    __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
};

// renormalise s + e, |e| small against |s|
__device__ __forceinline__ df df_norm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return df(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ df operator+(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}
__device__ __forceinline__ df operator+(df a, float b)
{
    float s, e;
    two_sum(a.hi, b, s, e);
    return df_norm(s, __fadd_rn(e, a.lo));
}
__device__ __forceinline__ df operator+(float a, df b) { return b + a; }
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }
__device__ __forceinline__ df operator-(float a, df b) { return (-b) + a; }
__device__ __forceinline__ df operator*(df a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_norm(p, e);
}
__device__ __forceinline__ df operator*(float a, df b) { return b * a; }
__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm(p, e);
}
__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }
__device__ __forceinline__ df &operator+=(df &a, float b) { return a = a + b; }
__device__ __forceinline__ df &operator-=(df &a, df b) { return a = a - b; }

// c + a * b with one renormalisation
__device__ __forceinline__ df df_fma(df a, df b, df c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, e));
    return df_norm(s, t);
}
__device__ __forceinline__ df df_fma(df a, float b, df c)
{
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, e));
    return df_norm(s, t);
}

// 1 / a: the correctly rounded float reciprocal y of a.hi, then one Newton
// step y + y e with e = 1 - a y formed by FMAs (error about y e^2, 2^-48)
__device__ __forceinline__ df df_rcp(df a)
{
    const float y = __frcp_rn(a.hi);
    float e = fmaf(-a.hi, y, 1.f);
    e = fmaf(-a.lo, y, e);
    return df_norm(y, __fmul_rn(y, e));
}

__device__ __forceinline__ df df_from_d(double d)
{
    const float h = d2f(d);
    return df(h, d2f(d - f2d(h)));
}
__device__ __forceinline__ double df_to_d(df a) { return f2d(a.hi) + f2d(a.lo); }

// a double-float increment added to the float-float / float parts of the state
__device__ __forceinline__ void add_inc(ff &a, df d)
{
    a = ff_add(a, d.hi);
    a = ff_add(a, d.lo);
}
__device__ __forceinline__ void add_inc(float &a, df d)
{
    float s, e;
    two_sum(a, d.hi, s, e);
    a = __fadd_rn(s, __fadd_rn(e, d.lo));
}

// contraction-free float arithmetic for the few plain-float expressions of this
// file (every kernel that inlines them must round them alike)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dot2_rn(float a, float b, float c, float d)
{
    return __fadd_rn(__fmul_rn(a, b), __fmul_rn(c, d));
}
__device__ __forceinline__ float hypot_rn(float x, float y) { return __fsqrt_rn(dot2_rn(x, x, y, y)); }

// ------------------------------------------------------------------ the first update
// The update at the seed hit in closed form.  The prior is seed_cov * I6 plus
// the scattering noise on phi and theta, so the position block is c I3 and it
// has no correlation with the angles; R has the eigenvectors r-hat, phi-hat at
// the hit azimuth (variances a, b) and z-hat (variance rzz).  Then, along each
// eigenvector with variance v: gain c / (c + v), posterior variance
// c v / (c + v), chi2 term residual^2 / (c + v); the angle rows keep their
// prior.  These are the Kalman update's own results (S = cI + R is diagonal in
// that frame), written as ratios of positive terms.
__device__ __forceinline__ bool df_seed_update(Track<float, ff> &st, df p[21], float hx, float hy, float hz,
                                               const Surf &sf, df &chi2)
{
    const float r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    const df c = p[pk(0, 0)];
    const float va = sf.var_rad, vb = sf.var_rphi, vz = sf.var_zz;
    if (!(c.hi > 0.f) || !(va > 0.f) || !(vb > 0.f) || !(vz > 0.f)) return false;
    const df sa = c + va, sb = c + vb, sz = c + vz;
    const df ia = df_rcp(sa), ib = df_rcp(sb), iz = df_rcp(sz);
    const df ka = c * ia, kb = c * ib, kz = c * iz;  // gains
    const df pa = ka * va, pb = kb * vb, pzz = kz * vz;  // posterior variances
    df dx, dy;
    if (va == vb) {
        dx = ka * r0;
        dy = ka * r1;
        chi2 += (df(r0) * r0 + df(r1) * r1) * ia;
        p[pk(0, 0)] = pa;
        p[pk(1, 0)] = df(0.f);
        p[pk(1, 1)] = pa;
    } else {
        const float rh = hypot_rn(hx, hy);
        const float cs = __fdiv_rn(hx, rh), sn = __fdiv_rn(hy, rh);
        const df nr = df(r0) * cs + df(r1) * sn, nt = df(r1) * cs - df(r0) * sn;  // residual along r-hat, phi-hat
        const df gr = ka * nr, gt = kb * nt;
        dx = gr * cs - gt * sn;
        dy = gr * sn + gt * cs;
        chi2 += nr * nr * ia + nt * nt * ib;
        p[pk(0, 0)] = pa * cs * cs + pb * sn * sn;
        p[pk(1, 0)] = (pa - pb) * cs * sn;
        p[pk(1, 1)] = pa * sn * sn + pb * cs * cs;
    }
    chi2 += df(r2) * r2 * iz;
    p[pk(2, 0)] = df(0.f);
    p[pk(2, 1)] = df(0.f);
    p[pk(2, 2)] = pzz;
    add_inc(st.x, dx);
    add_inc(st.y, dy);
    add_inc(st.z, kz * r2);
    return true;
}

// ------------------------------------------------------------------ U-D factored update
// U-D order of the state: (1/pT, phi, theta, u3, u4, u5), the position last, in
// a frame that holds the surface normal at the predicted point as one axis:
// barrel (n, t, z), n radial and t = z-hat x n; disk (x, y, z), n = z.  After
// the transport the state lies on the surface and, in exact arithmetic, the
// covariance has a zero row and column along the normal.  What rounding and
// the FP32 Jacobian leave there is a residue with near-unit correlation to the
// angles, and a pivot on it would wreck the factorisation: that row is set to
// zero, its pivot to zero.
// strict upper triangle of U (i < j), column-major: column j holds rows 0..j-1
__host__ __device__ constexpr int uk(int i, int j) { return j * (j - 1) / 2 + i; }

// The U-D update below is written once for double-float (D = df: the seed
// phase, the near-tangent steps) and plain float (D = float); these are its
// scalar operations for both.
__device__ __forceinline__ df ud_fma(df a, df b, df c) { return df_fma(a, b, c); }
__device__ __forceinline__ df ud_fma(df a, float b, df c) { return df_fma(a, b, c); }
__device__ __forceinline__ float ud_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ df ud_rcp(df a) { return df_rcp(a); }
__device__ __forceinline__ float ud_rcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ float ud_lead(df a) { return a.hi; }
__device__ __forceinline__ float ud_lead(float a) { return a; }

template <class D>
struct UDT {
    D u[15];
    D d[6];
};
using UD = UDT<df>;

// the position frame: barrel, (cn, sn) the radial unit vector at the predicted point
struct PosFrame {
    bool barrel;
    float cn, sn;
};
__device__ __forceinline__ PosFrame pos_frame(const Track<float, ff> &st, const Surf &sf)
{
    PosFrame f;
    f.barrel = sf.kind == 0;
    f.cn = 1.f;
    f.sn = 0.f;
    if (f.barrel) {
        const float x = st.x.hi, y = st.y.hi;
        const float ir = __frsqrt_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
        f.cn = __fmul_rn(x, ir);
        f.sn = __fmul_rn(y, ir);
    }
    return f;
}
// index of the normal among the U-D indices
__device__ __forceinline__ int normal_index(const PosFrame &f) { return f.barrel ? 3 : 5; }

// native packed P -> A, U-D order in the position frame, the normal's row zero
template <class D>
__device__ __forceinline__ void ud_arrange(const D p[21], const PosFrame &fr, D a[21])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) a[pk(i, j)] = p[pk(i + 3, j + 3)];
    const D zero = D(0.f);
    if (fr.barrel) {
        const float c = fr.cn, s = fr.sn;  // t = -s x + c y
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a[pk(3, j)] = zero;
            a[pk(4, j)] = ud_fma(p[pk(1, j + 3)], c, p[pk(0, j + 3)] * (-s));
            a[pk(5, j)] = p[pk(2, j + 3)];
        }
        a[pk(3, 3)] = zero;
        a[pk(4, 3)] = zero;
        a[pk(5, 3)] = zero;
        // P_tt = s^2 Pxx - 2 s c Pxy + c^2 Pyy
        a[pk(4, 4)] = ud_fma(p[pk(1, 1)] * c, c, ud_fma(p[pk(1, 0)] * mul_rn(-2.f, s), c, p[pk(0, 0)] * s * s));
        a[pk(5, 4)] = ud_fma(p[pk(2, 1)], c, p[pk(2, 0)] * (-s));
        a[pk(5, 5)] = p[pk(2, 2)];
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a[pk(3, j)] = p[pk(0, j + 3)];
            a[pk(4, j)] = p[pk(1, j + 3)];
            a[pk(5, j)] = zero;
        }
        a[pk(3, 3)] = p[pk(0, 0)];
        a[pk(4, 3)] = p[pk(1, 0)];
        a[pk(4, 4)] = p[pk(1, 1)];
        a[pk(5, 3)] = zero;
        a[pk(5, 4)] = zero;
        a[pk(5, 5)] = zero;
    }
}

// A (U-D order, frame; the normal's row zero) -> native packed P
template <class D>
__device__ __forceinline__ void ud_unarrange(const D a[21], const PosFrame &fr, D p[21])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) p[pk(i + 3, j + 3)] = a[pk(i, j)];
    if (fr.barrel) {
        const float c = fr.cn, s = fr.sn;  // x = c n - s t, y = s n + c t, n fixed
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            p[pk(0, j + 3)] = a[pk(4, j)] * (-s);
            p[pk(1, j + 3)] = a[pk(4, j)] * c;
            p[pk(2, j + 3)] = a[pk(5, j)];
        }
        const D tt = a[pk(4, 4)];
        p[pk(0, 0)] = tt * s * s;
        p[pk(1, 0)] = -(tt * s * c);
        p[pk(1, 1)] = tt * c * c;
        p[pk(2, 0)] = a[pk(5, 4)] * (-s);
        p[pk(2, 1)] = a[pk(5, 4)] * c;
        p[pk(2, 2)] = a[pk(5, 5)];
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            p[pk(0, j + 3)] = a[pk(3, j)];
            p[pk(1, j + 3)] = a[pk(4, j)];
            p[pk(2, j + 3)] = D(0.f);
        }
        p[pk(0, 0)] = a[pk(3, 3)];
        p[pk(1, 0)] = a[pk(4, 3)];
        p[pk(1, 1)] = a[pk(4, 4)];
        p[pk(2, 0)] = D(0.f);
        p[pk(2, 1)] = D(0.f);
        p[pk(2, 2)] = D(0.f);
    }
}

// A = U D U^T (A in U-D order, overwritten), factored from the last index down;
// ZERO is the normal's index: pivot and column zero.  A pivot that rounding has
// left at or below zero is taken as zero with its column.
template <int ZERO, class D>
__device__ __forceinline__ void ud_factor(D a[21], UDT<D> &f)
{
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        const D dj = a[pk(j, j)];
        if (j != ZERO && ud_lead(dj) > 0.f) {
            f.d[j] = dj;
            const D inv = ud_rcp(dj);
#pragma unroll
            for (int i = 0; i < j; ++i) f.u[uk(i, j)] = a[pk(j, i)] * inv;
            // downdate of the leading block: a_ik -= a_ij u_kj (i >= k, both < j)
#pragma unroll
            for (int i = 0; i < j; ++i)
#pragma unroll
                for (int k = 0; k <= i; ++k) a[pk(i, k)] = ud_fma(-a[pk(j, i)], f.u[uk(k, j)], a[pk(i, k)]);
        } else {
            f.d[j] = D(0.f);
#pragma unroll
            for (int i = 0; i < j; ++i) f.u[uk(i, j)] = D(0.f);
        }
    }
}

// A (U-D order) = U D U^T
template <class D>
__device__ __forceinline__ void ud_compose(const UDT<D> &f, D a[21])
{
    // W = U D (strict upper part; the diagonal of W is d)
    D w[15];
#pragma unroll
    for (int j = 1; j < 6; ++j)
#pragma unroll
        for (int i = 0; i < j; ++i) w[uk(i, j)] = f.u[uk(i, j)] * f.d[j];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            // A_ij = sum_{k >= j} W_ik U_jk, U_jj = 1
            D v = i == j ? f.d[j] : w[uk(i, j)];
#pragma unroll
            for (int k = j + 1; k < 6; ++k) v = ud_fma(w[uk(i, k)], f.u[uk(j, k)], v);
            a[pk(j, i)] = v;
        }
}

// Bierman's scalar update for a measurement m = h . (u3, u4, u5) with variance r
// (FIRST = the first of h's position components that is nonzero, 3, 4 or 5)
// and innovation nu = m - h . x.  Updates U and D in place, returns the gain K
// (U-D order) through k and 1 / alpha, alpha = h P h^T + r the innovation
// variance.
template <int FIRST, class D>
__device__ __forceinline__ void ud_scalar(UDT<D> &f, float h3, float h4, float h5, float r, D k[6], D &ialpha)
{
    D fv[6], v[6];
    if (FIRST <= 3) fv[3] = D(h3);
    if (FIRST <= 4) fv[4] = FIRST <= 3 ? ud_fma(f.u[uk(3, 4)], h3, D(h4)) : D(h4);
    {
        D t = D(h5);
        if (FIRST <= 4) t = ud_fma(f.u[uk(4, 5)], h4, t);
        if (FIRST <= 3) t = ud_fma(f.u[uk(3, 5)], h3, t);
        fv[5] = t;
    }
#pragma unroll
    for (int j = FIRST; j < 6; ++j) v[j] = f.d[j] * fv[j];
    D b[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) b[i] = D(0.f);
    D al = D(r), ibeta = ud_rcp(al);
#pragma unroll
    for (int j = FIRST; j < 6; ++j) {
        const D beta = al;
        al = ud_fma(v[j], fv[j], beta);
        const D ia = ud_rcp(al);
        const D lam = -(fv[j] * ibeta);
        f.d[j] = f.d[j] * beta * ia;
#pragma unroll
        for (int i = 0; i < j; ++i) {
            const D uo = f.u[uk(i, j)];
            if (j > FIRST) {
                f.u[uk(i, j)] = ud_fma(b[i], lam, uo);
                b[i] = ud_fma(uo, v[j], b[i]);
            } else {
                b[i] = uo * v[j];  // b is still zero: this column of U stays
            }
        }
        b[j] = v[j];
        ibeta = ia;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) k[i] = b[i] * ibeta;
    ialpha = ibeta;
}

// Apply one scalar measurement: gain, chi2 term, state increment dx (U-D
// order) and the innovations of the measurements still to come (direction
// components in the frame: a, b).
template <int FIRST, class D, class C>
__device__ __forceinline__ void ud_measure(UDT<D> &f, float h3, float h4, float h5, float r, D nu, D dx[6], C &chi2,
                                           D &nu_a, float a3, float a4, float a5, D &nu_b, float b3, float b4,
                                           float b5)
{
    D k[6], ial;
    ud_scalar<FIRST>(f, h3, h4, h5, r, k, ial);
    chi2 += nu * nu * ial;
#pragma unroll
    for (int i = 0; i < 6; ++i) dx[i] = ud_fma(k[i], nu, dx[i]);
    // the state moved by k nu: the later innovations m - h' . x move by -h' . k nu
    const D kn3 = k[3] * nu, kn4 = k[4] * nu, kn5 = k[5] * nu;
    nu_a = nu_a - (kn3 * a3 + kn4 * a4 + kn5 * a5);
    nu_b = nu_b - (kn3 * b3 + kn4 * b4 + kn5 * b5);
}

// state increment dx (U-D order, frame) onto the track
template <class D>
__device__ __forceinline__ void ud_apply_state(Track<float, ff> &st, const D dx[6], const PosFrame &fr)
{
    add_inc(st.ip, dx[0]);
    add_inc(st.phi, dx[1]);
    st.phi = wrap(st.phi);
    add_inc(st.th, dx[2]);
    if (fr.barrel) {  // the normal coordinate does not move (dx[3] = 0)
        add_inc(st.x, dx[4] * (-fr.sn));
        add_inc(st.y, dx[4] * fr.cn);
        add_inc(st.z, dx[5]);
    } else {  // disk: z does not move
        add_inc(st.x, dx[3]);
        add_inc(st.y, dx[4]);
    }
}

// The 3-D update of Sec. 4.1 (H = [I3 | 0], R from the hit's azimuth) in U-D
// form: the measurement is taken as three scalar ones along R's eigenvectors
// (z-hat, then phi-hat and r-hat at the hit azimuth; when the two transverse
// variances are equal any orthonormal pair will do, and the frame's own t and n
// are taken), which gives the same posterior and chi2 = r^T S^-1 r as the joint
// update.  The measurement along the surface normal meets a zero prior
// variance: it adds its chi2 term and moves nothing.
template <class D, class C>
__device__ __forceinline__ bool ud_update3(Track<float, ff> &st, D p[21], float hx, float hy, float hz,
                                           const Surf &sf, C &chi2)
{
    const float r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    const float va = sf.var_rad, vb = sf.var_rphi, vz = sf.var_zz;
    if (!(va > 0.f) || !(vb > 0.f) || !(vz > 0.f)) return false;
    const PosFrame fr = pos_frame(st, sf);
    D a[21];
    ud_arrange(p, fr, a);
    UDT<D> f;
    if (fr.barrel) ud_factor<3>(a, f);
    else ud_factor<5>(a, f);
    D dx[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dx[i] = D(0.f);
    const bool iso = va == vb;
    float c1 = 1.f, s1 = 0.f;  // e1 = (c1, s1) with variance va, e2 = (-s1, c1) with vb
    if (iso && fr.barrel) {
        c1 = fr.cn;
        s1 = fr.sn;
    } else if (!iso) {
        const float rh = hypot_rn(hx, hy);
        c1 = __fdiv_rn(hx, rh);
        s1 = __fdiv_rn(hy, rh);
    }
    D n1 = ud_fma(D(r1), s1, D(r0) * c1), n2 = ud_fma(D(r1), c1, D(r0) * (-s1)), nz = D(r2);
    D dummy = D(0.f);
    if (fr.barrel) {
        // frame components of e1, e2; with iso they are n and t themselves
        float e1n = 1.f, e1t = 0.f, e2n = 0.f, e2t = 1.f;
        if (!iso) {
            e1n = dot2_rn(fr.cn, c1, fr.sn, s1);
            e1t = dot2_rn(fr.cn, s1, -fr.sn, c1);
            e2n = dot2_rn(fr.sn, c1, -fr.cn, s1);
            e2t = e1n;
        }
        ud_measure<5>(f, 0.f, 0.f, 1.f, vz, nz, dx, chi2, n2, e2n, e2t, 0.f, n1, e1n, e1t, 0.f);
        if (iso) {
            ud_measure<4>(f, 0.f, 1.f, 0.f, vb, n2, dx, chi2, n1, 1.f, 0.f, 0.f, dummy, 0.f, 0.f, 0.f);
            chi2 += n1 * n1 * ud_rcp(D(va));  // the normal: zero prior variance
        } else {
            ud_measure<3>(f, e2n, e2t, 0.f, vb, n2, dx, chi2, n1, e1n, e1t, 0.f, dummy, 0.f, 0.f, 0.f);
            ud_measure<3>(f, e1n, e1t, 0.f, va, n1, dx, chi2, dummy, 0.f, 0.f, 0.f, dummy, 0.f, 0.f, 0.f);
        }
    } else {
        chi2 += nz * nz * ud_rcp(D(vz));  // the disk normal z: zero prior variance
        if (s1 == 0.f) {  // e2 = +-y-hat
            ud_measure<4>(f, 0.f, c1, 0.f, vb, n2, dx, chi2, n1, c1, s1, 0.f, dummy, 0.f, 0.f, 0.f);
        } else {
            ud_measure<3>(f, -s1, c1, 0.f, vb, n2, dx, chi2, n1, c1, s1, 0.f, dummy, 0.f, 0.f, 0.f);
        }
        ud_measure<3>(f, c1, s1, 0.f, va, n1, dx, chi2, dummy, 0.f, 0.f, 0.f, dummy, 0.f, 0.f, 0.f);
    }
    ud_compose(f, a);
    ud_unarrange(a, fr, p);
    ud_apply_state(st, dx, fr);
    return true;
}

// The 2-D update of measurement model 1 (Sec. 4.1, the hit's own tangent
// plane, sf the cylinder through the hit): r-phi along t_h = (-sin a, cos a)
// with sig_rphi^2 and z with sig_z^2, a the hit azimuth; two scalar
// measurements.
template <class D, class C>
__device__ __forceinline__ bool ud_update2(Track<float, ff> &st, D p[21], float hx, float hy, float hz,
                                           const Surf &sf, C &chi2)
{
    const float r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    const float vt = sf.var_rphi, vz = sf.var_zz;
    if (!(vt > 0.f) || !(vz > 0.f)) return false;
    const float rh = hypot_rn(hx, hy);
    const float ca = __fdiv_rn(hx, rh), sa = __fdiv_rn(hy, rh);
    const PosFrame fr = pos_frame(st, sf);
    D a[21];
    ud_arrange(p, fr, a);
    UDT<D> f;
    ud_factor<3>(a, f);
    D dx[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dx[i] = D(0.f);
    // t_h in the frame (n, t)
    const float hn = dot2_rn(fr.sn, ca, -fr.cn, sa), ht = dot2_rn(fr.cn, ca, fr.sn, sa);
    D nt = ud_fma(D(r1), ca, D(r0) * (-sa)), nz = D(r2), dummy = D(0.f);
    ud_measure<5>(f, 0.f, 0.f, 1.f, vz, nz, dx, chi2, nt, hn, ht, 0.f, dummy, 0.f, 0.f, 0.f);
    ud_measure<3>(f, hn, ht, 0.f, vt, nt, dx, chi2, dummy, 0.f, 0.f, 0.f, dummy, 0.f, 0.f, 0.f);
    ud_compose(f, a);
    ud_unarrange(a, fr, p);
    ud_apply_state(st, dx, fr);
    return true;
}

// One step of the seed phase: propagate in FP32 (k > 0), transport the
// double-float covariance with the FP32 Jacobian (SEEDED: the covariance left
// by the closed-form first update), add the scattering noise, U-D update.
// TWO_D: the 2-D update on sf (the hit's own cylinder, model 1).
template <bool TWO_D>
__device__ __forceinline__ bool df_step_on(Track<float, ff> &st, df p[21], int k, float alpha, float mass2,
                                           int ms_on, const Surf &sf, float hx, float hy, float hz, df &chi2,
                                           unsigned &status, bool seeded)
{
    float cphi, sphi;
    if (k > 0) {
        Jac<float> J;
        if (!propagate(st, alpha, sf, J)) {
            status |= reach_bits(st);
            return false;
        }
        if (seeded) {
            // the first transport, from the seed hit, meets the full 1e4 angle
            // variances beside the hit-sized position block: FP64 here
            double pd[21];
#pragma unroll
            for (int i = 0; i < 21; ++i) pd[i] = df_to_d(p[i]);
            transport_seeded<double>(pd, widen(J));
#pragma unroll
            for (int i = 0; i < 21; ++i) p[i] = df_from_d(pd[i]);
        } else {
            transport<df>(p, J);
        }
        cphi = J.cphi1;
        sphi = J.sphi1;
    } else {
        sincos_pos(st.phi, sphi, cphi);
    }
    if (ms_on) status |= ms_noise<float, df>(st, sf, cphi, sphi, mass2, p);
    bool ok;
    if (k == 0) ok = df_seed_update(st, p, hx, hy, hz, sf, chi2);
    else if constexpr (TWO_D) ok = ud_update2(st, p, hx, hy, hz, sf, chi2);
    else ok = ud_update3(st, p, hx, hy, hz, sf, chi2);
    if (!ok) {
        status |= KF_ST_CHOL_FAIL;
        return false;
    }
    return true;
}

// A step of the FP32 layer loop at a near-tangent crossing (Jacobian entries
// growing like 1 / cos(alpha): FP32 arithmetic cannot carry the transport):
// FP32 propagation, then the transport, the scattering noise and the update in
// double-float U-D form from the FP32 covariance, rounded back to FP32.
// Returns false when the track ends here (status set).
template <bool TWO_D>
__device__ __forceinline__ bool df_step_from_f32(Track<float, ff> &st, float pf[21], float alpha, float mass2,
                                                 int ms_on, const Surf &sf, float hx, float hy, float hz,
                                                 double &chi2, unsigned &status)
{
    df p[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) p[i] = df(pf[i]);
    df c2 = df(0.f);
    const bool ok = df_step_on<TWO_D>(st, p, 1, alpha, mass2, ms_on, sf, hx, hy, hz, c2, status, false);
    if (!ok) return false;
    chi2 += df_to_d(c2);
#pragma unroll
    for (int i = 0; i < 21; ++i) pf[i] = p[i].hi;
    return true;
}

// A step of the FP32 layer loop at a near-tangent barrel crossing that is not
// steep: FP32 propagation, transport and noise, then the update in U-D form in
// FP32 (the standard-form FP32 update loses the covariance there; the U-D form,
// with the normal's row zeroed, keeps it).  TWO_D: the 2-D update on sf.
// Returns false when the track ends here (status set).
template <bool TWO_D>
__device__ __forceinline__ bool ud32_step(Track<float, ff> &st, float pf[21], float alpha, float mass2, int ms_on,
                                          const Surf &sf, float hx, float hy, float hz, double &chi2,
                                          unsigned &status)
{
    Jac<float> J;
    if (!propagate(st, alpha, sf, J)) {
        status |= reach_bits(st);
        return false;
    }
    transport<float>(pf, J);
    if (ms_on) status |= ms_noise<float, float>(st, sf, J.cphi1, J.sphi1, mass2, pf);
    bool ok;
    if constexpr (TWO_D) ok = ud_update2(st, pf, hx, hy, hz, sf, chi2);
    else ok = ud_update3(st, pf, hx, hy, hz, sf, chi2);
    if (!ok) {
        status |= KF_ST_CHOL_FAIL;
        return false;
    }
    return true;
}

// the seed covariance seed_cov * I6 in double-float
__device__ __forceinline__ void df_seed_cov(df p[21], double seed_cov)
{
    const df c = df_from_d(seed_cov);
#pragma unroll
    for (int i = 0; i < 21; ++i) p[i] = df(0.f);
#pragma unroll
    for (int i = 0; i < 6; ++i) p[pk(i, i)] = c;
}

}  // namespace kfd
