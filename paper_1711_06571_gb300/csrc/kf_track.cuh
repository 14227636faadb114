// kf_track.cuh -- per-track Kalman-filter steps, held in registers.
//
// One thread owns one track: state (x, y, z, 1/pT, phi, theta) and the packed
// 21-entry covariance live in registers for the whole layer loop.  Two type
// parameters select the precision:
//   T: arithmetic of propagation, Jacobian, transport and update
//      (float on the mixed path, double on the all-FP64 path)
//   P: storage of x, y, z, phi and theta (float-float on the mixed path, double):
//      FP32 storage alone would round these by ~1e-4 of their fitted sigma at
//      every update (100 cm, pi), which adds up over a 17-layer fit
// The 3x3 innovation-covariance solve is always FP64 (kf_common.cuh).
#pragma once

#include "kf_common.cuh"

namespace kfd {

// packed lower-triangle index, i >= j
__host__ __device__ constexpr int pk(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

template <class T, class P>
struct Track {
    P x, y, z, phi, th;  // extended precision (float-float on the mixed path)
    T ip;
};

// Pieces of the surface-constrained propagation Jacobian J = A + u w^T:
//   A = I + {ax3, ax4 (row x), ay3, ay4 (row y), az5 (row z), ap3 (row phi)},
//   u = d(state)/ds on rows x, y, z, phi, w = ds/d(state).
template <class T>
struct Jac {
    T ax3, ax4, ay3, ay4, az5, ap3;
    T u0, u1, u2, u4;
    T w[6];
    T cphi1, sphi1;  // cos, sin of the new phi
};

__device__ __forceinline__ double wide(float v) { return f2d(v); }
__device__ __forceinline__ double wide(double v) { return v; }

template <class T> __device__ __forceinline__ T tsqrt(T v);
template <> __device__ __forceinline__ float tsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double tsqrt<double>(double v) { return sqrt(v); }
__device__ __forceinline__ void tsincos(float a, float &s, float &c) { sincosf(a, &s, &c); }
__device__ __forceinline__ void tsincos(double a, double &s, double &c) { sincos(a, &s, &c); }
__device__ __forceinline__ float tlog(float v) { return logf(v); }
__device__ __forceinline__ double tlog(double v) { return log(v); }

template <class T> __device__ __forceinline__ T spos(const Surf &s);
template <> __device__ __forceinline__ float spos<float>(const Surf &s) { return s.pos; }
template <> __device__ __forceinline__ double spos<double>(const Surf &s) { return s.posd; }
template <class T> __device__ __forceinline__ T sxx0(const Surf &s);
template <> __device__ __forceinline__ float sxx0<float>(const Surf &s) { return s.x_x0; }
template <> __device__ __forceinline__ double sxx0<double>(const Surf &s) { return s.x_x0d; }

__device__ __forceinline__ float lo_part(ff a) { return a.lo; }
__device__ __forceinline__ double lo_part(double) { return 0.0; }
__device__ __forceinline__ float sub_lead(float Z, ff z) { return __fsub_rn(__fsub_rn(Z, z.hi), z.lo); }
__device__ __forceinline__ double sub_lead(double Z, double z) { return Z - z; }
__device__ __forceinline__ ff set_exact(float Z, ff) { return {Z, 0.f}; }
__device__ __forceinline__ double set_exact(double Z, double) { return Z; }

// x^2 + y^2 - R^2 for barrel surface sf
__device__ __forceinline__ float surf_excess(ff x, ff y, const Surf &sf) { return radial_excess(x, y, sf.pos2, sf.pos2lo); }
__device__ __forceinline__ double surf_excess(double x, double y, const Surf &sf)
{
    return radial_excess(x, y, sf.posd * sf.posd);
}

constexpr float MAX_PATH = 1.0e6f;  // longer transverse paths count as no intersection

// Propagate st along its helix to surface sf (Sec. 3 uniform field, Sec. 4.1
// propagation to the layer).  Barrel from inside: first crossing s > 0, found
// by Newton steps on |pos(s)|^2 - R^2 (to working precision, at most 12) from
// the second-order (parabolic) estimate; from outside: the crossing nearest s = 0.  Disk: s = (Z - z) tan(theta).
// alpha = -q * kappa * Bz (c = alpha / pT).  Returns false (state untouched)
// when the surface is not reached.
// The direction's sines and cosines of the state, which several propagations of
// the same state share (propagate_from).
template <class T>
struct Dir {
    T sphi, cphi, sth, cth;
};
template <class T, class P>
__device__ __forceinline__ Dir<T> direction(const Track<T, P> &st)
{
    Dir<T> d;
    sincos_pos(st.phi, d.sphi, d.cphi);
    sincos_pos(st.th, d.sth, d.cth);
    return d;
}

template <class T, class P>
__device__ __forceinline__ bool propagate_from(Track<T, P> &st, T alpha, const Surf &sf, Jac<T> &J, const Dir<T> &d)
{
    T c = alpha * st.ip;
    const T sphi = d.sphi, cphi = d.cphi, sth = d.sth, cth = d.cth;
    // theta outside (0, pi): an update has carried the polar angle through the
    // pole of the parametrisation, where cot(theta) diverges; the track ends
    if (!(sth > T(0))) return false;
    T cot = cth / sth;
    T s;
    const T X = lead(st.x), Y = lead(st.y);
    if (sf.kind == 0) {
        const T R = spos<T>(sf);
        const T g0 = surf_excess(st.x, st.y, sf);
        const T pt = X * cphi + Y * sphi, pn = -X * sphi + Y * cphi;
        const bool inside = g0 < T(0);
        if (inside) {
            // the helix circle reaches radius R iff |c| (R^2 - r^2) - 2 sgn(c) (p.n) <= 2 R
            T sg = c > T(0) ? T(1) : (c < T(0) ? T(-1) : T(0));
            if (fabs(c) * (-g0) - T(2) * sg * pn > T(2) * R) return false;
        }
        // second-order model |pos(s)|^2 - R^2 ~ A s^2 + 2 pt s + g0, A = 1 + c (p.n);
        // A < 0 near the apex of a curling track
        const T A = T(1) + c * pn;
        const T disc = pt * pt - A * g0;
        if (disc >= T(0)) {
            T sq = tsqrt<T>(disc);
            T den = inside ? (pt + sq) : (pt + copysign(sq, pt));
            s = -g0 / den;  // root nearest s = 0 in the direction of motion
        } else {
            s = -pt / A;  // the model's apex; Newton on the exact helix takes it from there
        }
        const T xl = lo_part(st.x), yl = lo_part(st.y);
        // Newton on the exact helix until the step is below the working precision
        const T tol = sizeof(T) == 8 ? T(1e-13) : T(2e-7);
        for (int it = 0; it < 12; ++it) {
            T sinc, ch, sh, f1;
            helix_factors(T(0.5) * c * s, sinc, ch, sh, f1);
            T cm = cphi * ch - sphi * sh, sm = sphi * ch + cphi * sh;
            T dx = s * sinc * cm, dy = s * sinc * sm;
            T g = g0 + T(2) * ((X + xl) * dx + (Y + yl) * dy) + dx * dx + dy * dy;
            T c1 = cm * ch - sm * sh, s1 = sm * ch + cm * sh;
            T gp = T(2) * ((X + dx) * c1 + (Y + dy) * s1);
            T ds = g / gp;
            s = s - ds;
            if (!(fabs(ds) > tol * (fabs(s) + T(1)))) break;
        }
        if (!isfinite(s) || (inside && !(s > T(0)))) return false;
    } else {
        if (cot == T(0)) return false;
        s = sub_lead(spos<T>(sf), st.z) / cot;
        if (!(fabs(s) <= T(MAX_PATH))) return false;
    }
    T sinc, ch, sh, f1;
    helix_factors(T(0.5) * c * s, sinc, ch, sh, f1);
    T cm = cphi * ch - sphi * sh, sm = sphi * ch + cphi * sh;  // direction of the chord
    T dx = s * sinc * cm, dy = s * sinc * sm;
    T c1 = cm * ch - sm * sh, s1 = sm * ch + cm * sh;  // new direction
    T s2 = s * s;
    J.ax4 = -dy;
    J.ay4 = dx;
    J.ax3 = alpha * s2 * (cm * f1 - sm * T(0.5) * sinc);
    J.ay3 = alpha * s2 * (sm * f1 + cm * T(0.5) * sinc);
    J.az5 = -s / (sth * sth);
    J.ap3 = alpha * s;
    J.u0 = c1;
    J.u1 = s1;
    J.u2 = cot;
    J.u4 = c;
    J.cphi1 = c1;
    J.sphi1 = s1;
    const P nx = inc(st.x, dx), ny = inc(st.y, dy);
#pragma unroll
    for (int j = 0; j < 6; ++j) J.w[j] = T(0);
    if (sf.kind == 0) {
        const T xp = lead(nx), yp = lead(ny);
        T D = xp * c1 + yp * s1;  // (1/2) d|pos|^2/ds
        if (D == T(0)) return false;
        T iD = T(1) / D;
        J.w[0] = -xp * iD;
        J.w[1] = -yp * iD;
        J.w[3] = -(xp * J.ax3 + yp * J.ay3) * iD;
        J.w[4] = -(xp * J.ax4 + yp * J.ay4) * iD;
        st.z = inc(st.z, s * cot);
    } else {
        T ic = T(1) / cot;
        J.w[2] = -ic;
        J.w[5] = -J.az5 * ic;
        st.z = set_exact(spos<T>(sf), st.z);
    }
    st.x = nx;
    st.y = ny;
    st.phi = wrap(inc(st.phi, c * s));
    return true;
}

template <class T, class P>
__device__ __forceinline__ bool propagate(Track<T, P> &st, T alpha, const Surf &sf, Jac<T> &J)
{
    return propagate_from(st, alpha, sf, J, direction(st));
}

// status bits of a track whose propagation failed (st as it was): the surface
// is out of reach, and theta has left (0, pi) if that is why
template <class T, class P>
__device__ __forceinline__ unsigned reach_bits(const Track<T, P> &st)
{
    T sth, cth;
    sincos_pos(st.th, sth, cth);
    return KF_ST_NO_INTERSECT | (sth > T(0) ? 0u : KF_ST_THETA_RANGE);
}

// Sine of the angle between track and radial direction where the helix meets
// the cylinder R, from the state before propagation: for the helix circle
// (radius 1/|c|, centre C) and the cylinder, the triangle origin-C-crossing
// gives u = (|c| (R^2 - r^2) - 2 sgn(c) (p.n)) / (2 R), n = (-sin phi, cos phi).
// u > 1: the cylinder is out of reach; u -> 1: the crossing is tangent, where
// the surface-constrained Jacobian grows like 1 / cos(alpha) and FP32 loses
// the covariance transport.
template <class T, class P>
__device__ __forceinline__ T crossing_sine(const Track<T, P> &st, T alpha, const Surf &sf, T sphi, T cphi)
{
    T c = alpha * st.ip;
    const T X = lead(st.x), Y = lead(st.y);
    const T R = spos<T>(sf);
    const T g0 = surf_excess(st.x, st.y, sf);
    const T pn = -X * sphi + Y * cphi;
    T sg = c > T(0) ? T(1) : (c < T(0) ? T(-1) : T(0));
    return (fabs(c) * (-g0) - T(2) * sg * pn) / (T(2) * R);
}
template <class T, class P>
__device__ __forceinline__ T crossing_sine(const Track<T, P> &st, T alpha, const Surf &sf)
{
    T sphi, cphi;
    sincos_pos(st.phi, sphi, cphi);
    return crossing_sine(st, alpha, sf, sphi, cphi);
}

// P <- J P J^T with J = A + u w^T, as A P A^T + a u^T + u a^T + gamma u u^T,
// y = P w, a = A y, gamma = w.y; A has six off-diagonal entries and u two
// structural zeros, so the product costs ~150 FMA instead of ~430 dense.
// JT: type of the Jacobian's entries (the FP32 Jacobian of the mixed path may
// transport a wider covariance T)
template <class T, class JT = T>
__device__ __forceinline__ void transport(T p[21], const Jac<JT> &J)
{
    T y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T v = T(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) v += p[pk(i, j)] * J.w[j];
        y[i] = v;
    }
    T gam = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) gam += J.w[i] * y[i];
    T a[6];
    a[0] = y[0] + J.ax3 * y[3] + J.ax4 * y[4];
    a[1] = y[1] + J.ay3 * y[3] + J.ay4 * y[4];
    a[2] = y[2] + J.az5 * y[5];
    a[3] = y[3];
    a[4] = y[4] + J.ap3 * y[3];
    a[5] = y[5];
    // B = A P
    T B[6][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        T p3 = p[pk(3, j)], p4 = p[pk(4, j)], p5 = p[pk(5, j)];
        B[0][j] = p[pk(0, j)] + J.ax3 * p3 + J.ax4 * p4;
        B[1][j] = p[pk(1, j)] + J.ay3 * p3 + J.ay4 * p4;
        B[2][j] = p[pk(2, j)] + J.az5 * p5;
        B[3][j] = p3;
        B[4][j] = p4 + J.ap3 * p3;
        B[5][j] = p5;
    }
    const JT u[6] = {J.u0, J.u1, J.u2, JT(0), J.u4, JT(0)};
    // C = B A^T (lower triangle) plus the rank-2 terms
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v;
            if (j == 0) v = B[i][0] + J.ax3 * B[i][3] + J.ax4 * B[i][4];
            else if (j == 1) v = B[i][1] + J.ay3 * B[i][3] + J.ay4 * B[i][4];
            else if (j == 2) v = B[i][2] + J.az5 * B[i][5];
            else if (j == 4) v = B[i][4] + J.ap3 * B[i][3];
            else v = B[i][j];
            if (i != 3 && i != 5) v += u[i] * a[j];
            if (j != 3 && j != 5) v += a[i] * u[j];
            if (i != 3 && i != 5 && j != 3 && j != 5) v += gam * u[i] * u[j];
            p[pk(i, j)] = v;
        }
    }
}

// transport for the covariance left by the structured first update (a diagonal
// seed covariance updated at the seed hit): P = [Q 0; 0 D], Q the 3x3 position
// block, D = diag(d3, d4, d5), no position-angle terms.  J P J^T = A P A^T +
// u a^T + a u^T + gamma u u^T as in transport, with A P A^T written out for this
// P (A = I + N, N's entries ax3, ax4, ay3, ay4, az5, ap3 all in columns 3..5):
// about 90 FMA instead of 180.
template <class T, class JT = T>
__device__ __forceinline__ void transport_seeded(T p[21], const Jac<JT> &J)
{
    const T d3 = p[pk(3, 3)], d4 = p[pk(4, 4)], d5 = p[pk(5, 5)];
    T y[6];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = p[pk(i, 0)] * J.w[0] + p[pk(i, 1)] * J.w[1] + p[pk(i, 2)] * J.w[2];
    y[3] = d3 * J.w[3];
    y[4] = d4 * J.w[4];
    y[5] = d5 * J.w[5];
    T gam = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) gam += J.w[i] * y[i];
    T a[6];
    a[0] = y[0] + J.ax3 * y[3] + J.ax4 * y[4];
    a[1] = y[1] + J.ay3 * y[3] + J.ay4 * y[4];
    a[2] = y[2] + J.az5 * y[5];
    a[3] = y[3];
    a[4] = y[4] + J.ap3 * y[3];
    a[5] = y[5];
    // A P A^T, lower triangle
    const T x3 = J.ax3 * d3, x4 = J.ax4 * d4, w3 = J.ay3 * d3, w4 = J.ay4 * d4, z5 = J.az5 * d5, q3 = J.ap3 * d3;
    T c[21];
    c[pk(0, 0)] = p[pk(0, 0)] + J.ax3 * x3 + J.ax4 * x4;
    c[pk(1, 0)] = p[pk(1, 0)] + J.ay3 * x3 + J.ay4 * x4;
    c[pk(1, 1)] = p[pk(1, 1)] + J.ay3 * w3 + J.ay4 * w4;
    c[pk(2, 0)] = p[pk(2, 0)];
    c[pk(2, 1)] = p[pk(2, 1)];
    c[pk(2, 2)] = p[pk(2, 2)] + J.az5 * z5;
    c[pk(3, 0)] = x3;
    c[pk(3, 1)] = w3;
    c[pk(3, 2)] = T(0);
    c[pk(3, 3)] = d3;
    c[pk(4, 0)] = x4 + J.ap3 * x3;
    c[pk(4, 1)] = w4 + J.ap3 * w3;
    c[pk(4, 2)] = T(0);
    c[pk(4, 3)] = q3;
    c[pk(4, 4)] = d4 + J.ap3 * q3;
    c[pk(5, 0)] = T(0);
    c[pk(5, 1)] = T(0);
    c[pk(5, 2)] = z5;
    c[pk(5, 3)] = T(0);
    c[pk(5, 4)] = T(0);
    c[pk(5, 5)] = d5;
    const JT u[6] = {J.u0, J.u1, J.u2, JT(0), J.u4, JT(0)};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v = c[pk(i, j)];
            if (i != 3 && i != 5) v += u[i] * a[j];
            if (j != 3 && j != 5) v += a[i] * u[j];
            if (i != 3 && i != 5 && j != 3 && j != 5) v += gam * u[i] * u[j];
            p[pk(i, j)] = v;
        }
    }
}

// The position block of J P J^T alone (packed entries 0..5: (0,0) (1,0) (1,1)
// (2,0) (2,1) (2,2)), by the same arithmetic as transport: what a hit's chi2
// needs when the state is only carried to the hit to score it.
template <class T>
__device__ __forceinline__ void transport_pos(const T p[21], const Jac<T> &J, T q[6])
{
    T y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T v = T(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) v += p[pk(i, j)] * J.w[j];
        y[i] = v;
    }
    T gam = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) gam += J.w[i] * y[i];
    T a[3];
    a[0] = y[0] + J.ax3 * y[3] + J.ax4 * y[4];
    a[1] = y[1] + J.ay3 * y[3] + J.ay4 * y[4];
    a[2] = y[2] + J.az5 * y[5];
    T B[3][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        T p3 = p[pk(3, j)], p4 = p[pk(4, j)], p5 = p[pk(5, j)];
        B[0][j] = p[pk(0, j)] + J.ax3 * p3 + J.ax4 * p4;
        B[1][j] = p[pk(1, j)] + J.ay3 * p3 + J.ay4 * p4;
        B[2][j] = p[pk(2, j)] + J.az5 * p5;
    }
    const T u[3] = {J.u0, J.u1, J.u2};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T v;
            if (j == 0) v = B[i][0] + J.ax3 * B[i][3] + J.ax4 * B[i][4];
            else if (j == 1) v = B[i][1] + J.ay3 * B[i][3] + J.ay4 * B[i][4];
            else v = B[i][2] + J.az5 * B[i][5];
            v += u[i] * a[j];
            v += a[i] * u[j];
            v += gam * u[i] * u[j];
            q[pk(i, j)] = v;
        }
    }
}

// Widen a float Jacobian for an FP64 transport.
__device__ __forceinline__ Jac<double> widen(const Jac<float> &J)
{
    Jac<double> D;
    D.ax3 = f2d(J.ax3); D.ax4 = f2d(J.ax4); D.ay3 = f2d(J.ay3); D.ay4 = f2d(J.ay4); D.az5 = f2d(J.az5);
    D.ap3 = f2d(J.ap3);
    D.u0 = f2d(J.u0); D.u1 = f2d(J.u1); D.u2 = f2d(J.u2); D.u4 = f2d(J.u4);
#pragma unroll
    for (int j = 0; j < 6; ++j) D.w[j] = f2d(J.w[j]);
    D.cphi1 = f2d(J.cphi1);
    D.sphi1 = f2d(J.sphi1);
    return D;
}
__device__ __forceinline__ const Jac<double> &widen(const Jac<double> &J) { return J; }

// the Jacobian in the covariance's type C
template <class C> struct JacAs;
template <> struct JacAs<float> {
    __device__ static const Jac<float> &get(const Jac<float> &J) { return J; }
};
template <> struct JacAs<double> {
    __device__ static Jac<double> get(const Jac<float> &J) { return widen(J); }
    __device__ static const Jac<double> &get(const Jac<double> &J) { return J; }
};

// Multiple scattering (Sec. 2), Highland angle with p = pT / sin(theta) and
// thickness t = (x/X0) / max(|cos alpha|, 0.05):
//   theta0 = 0.0136 (1/p) sqrt(1 + m^2/p^2) sqrt(t) (1 + 0.038 ln(t (1 + m^2/p^2)))
// (the PDG form with 1/beta = sqrt(1 + m^2/p^2)); P_theta += theta0^2,
// P_phi += theta0^2 / sin^2(theta).  Returns KF_ST_GRAZING if the guard was used.
template <class T, class C, class Pp>
__device__ __forceinline__ unsigned ms_noise(const Track<T, Pp> &st, const Surf &sf, T cphi, T sphi, T mass2, C p[21])
{
    T xx0 = sxx0<T>(sf);
    if (!(xx0 > T(0))) return 0u;
    T sth, cth;
    sincos_pos(st.th, sth, cth);
    T ca;
    if (sf.kind == 0) {
        T X = lead(st.x), Y = lead(st.y);
        ca = sth * (X * cphi + Y * sphi) / tsqrt<T>(X * X + Y * Y);
    } else {
        ca = cth;
    }
    ca = fabs(ca);
    unsigned flag = 0u;
    if (ca < T(0.05)) {
        ca = T(0.05);
        flag = KF_ST_GRAZING;
    }
    T t = xx0 / ca;
    T invp = fabs(st.ip) * sth;
    if (invp > T(0)) {
        T ib2 = T(1) + mass2 * invp * invp;
        T th0 = T(0.0136) * invp * tsqrt<T>(ib2) * tsqrt<T>(t) * (T(1) + T(0.038) * tlog(t * ib2));
        T th02 = th0 * th0;
        p[pk(5, 5)] += C(th02);
        p[pk(4, 4)] += C(th02 / (sth * sth));
    }
    return flag;
}

// Hit covariance R at the hit azimuth (Sec. 4.1 tangent plane):
// variance var_rad along r-hat, var_rphi along phi-hat, var_zz along z.
template <class T>
__device__ __forceinline__ void meas_cov(const Surf &sf, float hx, float hy, T &rxx, T &rxy, T &ryy, T &rzz)
{
    const bool d = sizeof(T) == 8;
    T a = d ? T(sf.var_radd) : T(sf.var_rad), b = d ? T(sf.var_rphid) : T(sf.var_rphi);
    rzz = d ? T(sf.var_zzd) : T(sf.var_zz);
    if (a == b) {
        rxx = a;
        ryy = a;
        rxy = T(0);
        return;
    }
    T r2 = T(hx) * T(hx) + T(hy) * T(hy);
    T cs = T(hx), sn = T(hy);
    T ir2 = T(1) / r2;
    rxx = (a * cs * cs + b * sn * sn) * ir2;
    rxy = (a - b) * cs * sn * ir2;
    ryy = (a * sn * sn + b * cs * cs) * ir2;
}

__device__ __forceinline__ void add_inc(ff &a, double d)
{
    float h = (float)d;
    a = ff_add(a, h);
    a = ff_add(a, (float)(d - (double)h));
}
__device__ __forceinline__ void add_inc(double &a, double d) { a += d; }
__device__ __forceinline__ void add_inc(ff &a, float d) { a = ff_add(a, d); }
__device__ __forceinline__ void add_inc(float &a, double d) { a = (float)((double)a + d); }
__device__ __forceinline__ void add_inc(float &a, float d) { a += d; }

// Kalman update with the 3-D hit, H = [I3 | 0] (Sec. 4.1):
//   r = m - x, S = P_pos + R, chi2 = r^T S^-1 r (FP64 LDL^T),
//   K = P H^T S^-1, x += K r,
//   JOSEPH = false: P -= K (H P)                          (standard form)
//   JOSEPH = true:  P = (I - K H) P (I - K H)^T + K R K^T  (Joseph form, written
//                   as P - K G^T + (K S - G) K^T with G = P H^T; stays positive
//                   definite under the 1e4 seed covariance)
// C is the covariance type; returns false if S is not positive definite.
// The gain and the state and covariance update of kf_update, given the LDL^T
// factor f of S (entries s11..s33) and the residual r.
template <bool JOSEPH, class C, class T, class Pp, class R>
__device__ __forceinline__ void kf_apply_gain(Track<T, Pp> &st, C p[21], R r0, R r1, R r2, const Ldl3 &f, C s11,
                                              C s21, C s22, C s31, C s32, C s33)
{
    C a11, a21, a22, a31, a32, a33;
    ldl3_inverse<C>(f, a11, a21, a22, a31, a32, a33);
    C G[6][3], K[6][3];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        G[i][0] = p[pk(i, 0)];
        G[i][1] = p[pk(i, 1)];
        G[i][2] = p[pk(i, 2)];
        K[i][0] = G[i][0] * a11 + G[i][1] * a21 + G[i][2] * a31;
        K[i][1] = G[i][0] * a21 + G[i][1] * a22 + G[i][2] * a32;
        K[i][2] = G[i][0] * a31 + G[i][1] * a32 + G[i][2] * a33;
    }
    C d[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = K[i][0] * C(r0) + K[i][1] * C(r1) + K[i][2] * C(r2);
    add_inc(st.x, d[0]);
    add_inc(st.y, d[1]);
    add_inc(st.z, d[2]);
    add_inc(st.ip, d[3]);
    add_inc(st.phi, d[4]);
    st.phi = wrap(st.phi);
    add_inc(st.th, d[5]);  // float-float or double
    if (JOSEPH) {
        // W = K S - G and P - K G^T + W K^T, each as one chain of fused
        // multiply-adds from its accumulator (no separate products or sums: the
        // FP64 pipe issues an FMA in the slot of a multiply or an add)
        C W[6][3];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            W[i][0] = fma(K[i][2], s31, fma(K[i][1], s21, fma(K[i][0], s11, -G[i][0])));
            W[i][1] = fma(K[i][2], s32, fma(K[i][1], s22, fma(K[i][0], s21, -G[i][1])));
            W[i][2] = fma(K[i][2], s33, fma(K[i][1], s32, fma(K[i][0], s31, -G[i][2])));
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                C v = fma(-K[i][0], G[j][0], p[pk(i, j)]);
                v = fma(-K[i][1], G[j][1], v);
                v = fma(-K[i][2], G[j][2], v);
                v = fma(W[i][0], K[j][0], v);
                v = fma(W[i][1], K[j][1], v);
                p[pk(i, j)] = fma(W[i][2], K[j][2], v);
            }
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j)
                p[pk(i, j)] -= K[i][0] * G[j][0] + K[i][1] * G[j][1] + K[i][2] * G[j][2];
    }
}

template <bool JOSEPH, class C, class T, class Pp>
__device__ __forceinline__ bool kf_update(Track<T, Pp> &st, C p[21], float hx, float hy, float hz, const Surf &sf,
                                          double &chi2)
{
    const auto r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);  // float or double
    C rxx, rxy, ryy, rzz;
    meas_cov<C>(sf, hx, hy, rxx, rxy, ryy, rzz);
    C s11 = p[pk(0, 0)] + rxx, s21 = p[pk(1, 0)] + rxy, s22 = p[pk(1, 1)] + ryy;
    C s31 = p[pk(2, 0)], s32 = p[pk(2, 1)], s33 = p[pk(2, 2)] + rzz;
    Ldl3 f;
    if (!ldl3<sizeof(C) == 8>(wide(s11), wide(s21), wide(s22), wide(s31), wide(s32), wide(s33), f)) return false;
    chi2 += ldl3_chi2(f, wide(r0), wide(r1), wide(r2));
    kf_apply_gain<JOSEPH>(st, p, r0, r1, r2, f, s11, s21, s22, s31, s32, s33);
    return true;
}

// Update on the mixed path (FP32 covariance).  The standard form loses about
// log10(prior / hit variance) digits to cancellation; where the prior position
// variance exceeds the hit variance along x, y or z by more than
// UPDATE_FP64_RATIO (after layers without an accepted hit, a long extrapolation,
// a seed phase) the update runs in FP64, Joseph form.
constexpr float UPDATE_FP64_RATIO = 100.f;

// A mixed-path track handed by value to an out-of-line FP64 routine.  The
// rarely taken FP64 branches of the FP32 layer loop are kept out of line so that
// the loop's own code stays compact in the instruction cache (warps of a
// persistent kernel run different parts of the loop at the same time).
struct MixedIO {
    Track<float, ff> st;
    float p[21];
    double chi2;
    unsigned status;
    int ok;
};

__device__ __forceinline__ void mixed_pack(MixedIO &m, const Track<float, ff> &st, const float p[21], double chi2,
                                           unsigned status)
{
    m.st = st;
#pragma unroll
    for (int i = 0; i < 21; ++i) m.p[i] = p[i];
    m.chi2 = chi2;
    m.status = status;
    m.ok = 0;
}
__device__ __forceinline__ bool mixed_unpack(const MixedIO &m, Track<float, ff> &st, float p[21], double &chi2,
                                             unsigned &status)
{
    st = m.st;
#pragma unroll
    for (int i = 0; i < 21; ++i) p[i] = m.p[i];
    chi2 = m.chi2;
    status = m.status;
    return m.ok != 0;
}

// the FP64 Joseph update of an FP32 covariance, out of line
static __device__ __noinline__ MixedIO kf_update_fp64_of_f32(MixedIO m, float hx, float hy, float hz,
                                                             const Surf *sf)
{
    double pd[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pd[i] = f2d(m.p[i]);
    m.ok = kf_update<true>(m.st, pd, hx, hy, hz, *sf, m.chi2);
#pragma unroll
    for (int i = 0; i < 21; ++i) m.p[i] = d2f(pd[i]);
    return m;
}

template <class Pp>
__device__ __forceinline__ bool kf_update_mixed(Track<float, Pp> &st, float p[21], float hx, float hy, float hz,
                                                const Surf &sf, double &chi2)
{
    float rxx, rxy, ryy, rzz;
    meas_cov<float>(sf, hx, hy, rxx, rxy, ryy, rzz);
    const bool informative = p[pk(0, 0)] > UPDATE_FP64_RATIO * rxx || p[pk(1, 1)] > UPDATE_FP64_RATIO * ryy ||
                             p[pk(2, 2)] > UPDATE_FP64_RATIO * rzz;
    if (informative) {
        MixedIO m;
        unsigned status = 0u;
        mixed_pack(m, st, p, chi2, status);
        m = kf_update_fp64_of_f32(m, hx, hy, hz, &sf);
        return mixed_unpack(m, st, p, chi2, status);
    }
    return kf_update<false>(st, p, hx, hy, hz, sf, chi2);
}
template <class Pp>
__device__ __forceinline__ bool kf_update_mixed(Track<double, Pp> &st, double p[21], float hx, float hy, float hz,
                                                const Surf &sf, double &chi2)
{
    return kf_update<false>(st, p, hx, hy, hz, sf, chi2);
}

// kf_update_mixed for a hit whose S the caller has already factored (f, from the
// same FP32 sums kf_update would form) and whose chi2 it has computed (c2): the
// standard-form update without a second factorisation.  Strongly informative
// updates still take the FP64 Joseph path.
template <class Pp>
__device__ __forceinline__ bool kf_update_mixed_factored(Track<float, Pp> &st, float p[21], float hx, float hy,
                                                         float hz, const Surf &sf, double &chi2, const Ldl3 &f,
                                                         double c2)
{
    float rxx, rxy, ryy, rzz;
    meas_cov<float>(sf, hx, hy, rxx, rxy, ryy, rzz);
    const bool informative = p[pk(0, 0)] > UPDATE_FP64_RATIO * rxx || p[pk(1, 1)] > UPDATE_FP64_RATIO * ryy ||
                             p[pk(2, 2)] > UPDATE_FP64_RATIO * rzz;
    if (informative) return kf_update_mixed(st, p, hx, hy, hz, sf, chi2);
    const float r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    chi2 += c2;
    kf_apply_gain<false>(st, p, r0, r1, r2, f, p[pk(0, 0)] + rxx, p[pk(1, 0)] + rxy, p[pk(1, 1)] + ryy, p[pk(2, 0)],
                         p[pk(2, 1)], p[pk(2, 2)] + rzz);
    return true;
}

// ---------------------------------------------------------------- measurement model 1
// Sec. 4.1, non-ideal geometry: a barrel hit need not lie on its layer's average
// cylinder.  The state is carried to the cylinder through the hit and updated on
// the plane tangent to it there, with the two coordinates measured on that plane:
// H has rows t = (-sin a, cos a, 0, ..) and (0, 0, 1, ..), a the hit azimuth;
// R = diag(sig_rphi^2, sig_z^2); chi2 and S^-1 from a 2x2 LDL^T in FP64.

// the cylinder through a barrel hit: R^2 = hx^2 + hy^2 as a float-float (the
// squares exact by FMA, their sum by two_sum; about 48 bits) for the FP32
// propagation, R in FP64 for the FP64 one
__device__ __forceinline__ Surf hit_surface(const Surf &sf, float hx, float hy)
{
    Surf h = sf;
    const float p1 = __fmul_rn(hx, hx), e1 = fmaf(hx, hx, -p1);
    const float p2 = __fmul_rn(hy, hy), e2 = fmaf(hy, hy, -p2);
    float s, e;
    two_sum(p1, p2, s, e);
    const float lo = e + (e1 + e2);
    h.pos2 = s + lo;
    h.pos2lo = lo - (h.pos2 - s);
    h.pos = sqrtf(h.pos2);
    h.posd = sqrt((double)h.pos2 + (double)h.pos2lo);
    return h;
}


template <bool JOSEPH, class C, class T, class Pp>
__device__ __forceinline__ bool kf_update2d(Track<T, Pp> &st, C p[21], float hx, float hy, float hz, const Surf &sf,
                                            double &chi2)
{
    const auto r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    const bool d = sizeof(C) == 8;
    const C rh = sqrt(C(hx) * C(hx) + C(hy) * C(hy));
    const C ca = C(hx) / rh, sa = C(hy) / rh;
    const C vt = d ? C(sf.var_rphid) : C(sf.var_rphi), vz = d ? C(sf.var_zzd) : C(sf.var_zz);
    // G = P H^T (6x2)
    C G[6][2];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        G[i][0] = -sa * p[pk(i, 0)] + ca * p[pk(i, 1)];
        G[i][1] = p[pk(i, 2)];
    }
    const C s11 = -sa * G[0][0] + ca * G[1][0] + vt, s21 = G[2][0], s22 = p[pk(2, 2)] + vz;
    const double e11 = wide(s11), e21 = wide(s21), e22 = wide(s22);
    if (!(e11 > 0.0)) return false;
    const double i1 = rcp_d(e11), l21 = e21 * i1, d2 = fma(-l21, e21, e22);
    if (!(d2 > 0.0)) return false;
    const double i2 = rcp_d(d2);
    const double rt = -wide(sa) * wide(C(r0)) + wide(ca) * wide(C(r1)), rz = wide(C(r2));
    const double z2 = fma(-l21, rt, rz);
    chi2 += fma(z2 * i2, z2, rt * i1 * rt);
    // S^-1 = L^-T D^-1 L^-1
    const C a11 = to_t(fma(l21 * l21, i2, i1), C(0)), a21 = to_t(-l21 * i2, C(0)), a22 = to_t(i2, C(0));
    C K[6][2];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        K[i][0] = G[i][0] * a11 + G[i][1] * a21;
        K[i][1] = G[i][0] * a21 + G[i][1] * a22;
    }
    const C ct = to_t(rt, C(0)), cz = to_t(rz, C(0));
    C dd[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dd[i] = K[i][0] * ct + K[i][1] * cz;
    add_inc(st.x, dd[0]);
    add_inc(st.y, dd[1]);
    add_inc(st.z, dd[2]);
    add_inc(st.ip, dd[3]);
    add_inc(st.phi, dd[4]);
    st.phi = wrap(st.phi);
    add_inc(st.th, dd[5]);
    if (JOSEPH) {
        // P - K G^T + (K S - G) K^T, as chains of fused multiply-adds (kf_apply_gain)
        C W[6][2];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            W[i][0] = fma(K[i][1], s21, fma(K[i][0], s11, -G[i][0]));
            W[i][1] = fma(K[i][1], s22, fma(K[i][0], s21, -G[i][1]));
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                C v = fma(-K[i][0], G[j][0], p[pk(i, j)]);
                v = fma(-K[i][1], G[j][1], v);
                v = fma(W[i][0], K[j][0], v);
                p[pk(i, j)] = fma(W[i][1], K[j][1], v);
            }
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) p[pk(i, j)] -= K[i][0] * G[j][0] + K[i][1] * G[j][1];
    }
    return true;
}

// chi2 of a hit under model 1 without the update (the S of kf_update2d), or -1
// when S is not positive definite: chi2 = (s22 rt^2 - 2 s21 rt rz + s11 rz^2) /
// det S in FP64 from the entries of S and the residual in C (the candidate
// score of a build step; the update recomputes chi2 through its LDL^T factor).
template <class C, class T, class Pp>
__device__ __forceinline__ double kf_chi2_2d(const Track<T, Pp> &st, const C p[21], float hx, float hy, float hz,
                                             const Surf &sf)
{
    const auto r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    const bool d = sizeof(C) == 8;
    const C rh = sqrt(C(hx) * C(hx) + C(hy) * C(hy));
    const C ca = C(hx) / rh, sa = C(hy) / rh;
    const C vt = d ? C(sf.var_rphid) : C(sf.var_rphi), vz = d ? C(sf.var_zzd) : C(sf.var_zz);
    const C g0 = -sa * p[pk(0, 0)] + ca * p[pk(1, 0)], g1 = -sa * p[pk(1, 0)] + ca * p[pk(1, 1)];
    const double e11 = wide(C(-sa * g0 + ca * g1 + vt));
    const double e21 = wide(C(-sa * p[pk(2, 0)] + ca * p[pk(2, 1)])), e22 = wide(C(p[pk(2, 2)] + vz));
    const double det = fma(e11, e22, -e21 * e21);
    if (!(e11 > 0.0) || !(det > 0.0)) return -1.0;
    const double rt = wide(C(-sa * C(r0) + ca * C(r1))), rz = wide(C(r2));
    const double num = fma(e22 * rt, rt, fma(-2.0 * e21 * rt, rz, e11 * rz * rz));
    return num * rcp_d(det);
}

// the FP64 Joseph 2-D update of an FP32 covariance, out of line
static __device__ __noinline__ MixedIO kf_update2d_fp64_of_f32(MixedIO m, float hx, float hy, float hz,
                                                               const Surf *sf)
{
    double pd[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) pd[i] = f2d(m.p[i]);
    m.ok = kf_update2d<true>(m.st, pd, hx, hy, hz, *sf, m.chi2);
#pragma unroll
    for (int i = 0; i < 21; ++i) m.p[i] = d2f(pd[i]);
    return m;
}

// model-1 update on the mixed path: FP64 Joseph when the prior on the measured
// directions exceeds the hit variance by UPDATE_FP64_RATIO (as kf_update_mixed)
template <class Pp>
__device__ __forceinline__ bool kf_update2d_mixed(Track<float, Pp> &st, float p[21], float hx, float hy, float hz,
                                                  const Surf &sf, double &chi2)
{
    const bool informative = p[pk(0, 0)] + p[pk(1, 1)] > UPDATE_FP64_RATIO * sf.var_rphi ||
                             p[pk(2, 2)] > UPDATE_FP64_RATIO * sf.var_zz;
    if (informative) {
        MixedIO m;
        unsigned status = 0u;
        mixed_pack(m, st, p, chi2, status);
        m = kf_update2d_fp64_of_f32(m, hx, hy, hz, &sf);
        return mixed_unpack(m, st, p, chi2, status);
    }
    return kf_update2d<false>(st, p, hx, hy, hz, sf, chi2);
}
template <class Pp>
__device__ __forceinline__ bool kf_update2d_mixed(Track<double, Pp> &st, double p[21], float hx, float hy, float hz,
                                                  const Surf &sf, double &chi2)
{
    return kf_update2d<false>(st, p, hx, hy, hz, sf, chi2);
}

// The first update, at the seed: the prior is seed_cov * I plus scattering
// noise on phi and theta only, so the position block is seed_cov * I and the
// position-angle blocks are zero.  The Joseph update then leaves the angle rows
// untouched (K = 0 there) and acts on the 3x3 position block alone; this
// evaluates exactly the nonzero part of kf_update<true>'s arithmetic.
template <class T, class Pp>
__device__ __forceinline__ bool kf_seed_update(Track<T, Pp> &st, double p[21], float hx, float hy, float hz,
                                               const Surf &sf, double &chi2)
{
    const auto r0 = resid(hx, st.x), r1 = resid(hy, st.y), r2 = resid(hz, st.z);
    double rxx, rxy, ryy, rzz;
    meas_cov<double>(sf, hx, hy, rxx, rxy, ryy, rzz);
    const double c = p[pk(0, 0)];  // == p(1,1) == p(2,2); off-diagonal position and cross terms are 0
    const double s11 = c + rxx, s21 = rxy, s22 = c + ryy, s33 = c + rzz;
    Ldl3 f;
    if (!ldl3(s11, s21, s22, 0.0, 0.0, s33, f)) return false;
    chi2 += ldl3_chi2(f, wide(r0), wide(r1), wide(r2));
    double a11, a21, a22, a31, a32, a33;
    ldl3_inverse<double>(f, a11, a21, a22, a31, a32, a33);
    // K = c S^-1 on the position rows
    const double K[3][3] = {{c * a11, c * a21, c * a31}, {c * a21, c * a22, c * a32}, {c * a31, c * a32, c * a33}};
    const double rr[3] = {wide(r0), wide(r1), wide(r2)};
    double d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = K[i][0] * rr[0] + K[i][1] * rr[1] + K[i][2] * rr[2];
    add_inc(st.x, d[0]);
    add_inc(st.y, d[1]);
    add_inc(st.z, d[2]);
    // Joseph: P = P - K G^T + (K S - G) K^T with G = c I on the position block
    // (S has no x-z or y-z terms here; chains of fused multiply-adds as in kf_apply_gain)
    double W[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        W[i][0] = fma(K[i][1], s21, fma(K[i][0], s11, i == 0 ? -c : 0.0));
        W[i][1] = fma(K[i][1], s22, fma(K[i][0], s21, i == 1 ? -c : 0.0));
        W[i][2] = fma(K[i][2], s33, i == 2 ? -c : 0.0);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
            p[pk(i, j)] = fma(W[i][2], K[j][2], fma(W[i][1], K[j][1], fma(W[i][0], K[j][0], fma(-K[i][j], c, p[pk(i, j)]))));
    return true;
}

// one surface crossing + update on surface sf; returns false when the track
// ends here.  TWO_D: the 2-D update on the plane tangent to sf at the hit
// (model 1, sf the hit's own cylinder).
// SEEDED, or seeded at run time: P is the one left by the structured first
// update (transport_seeded).
// dir: the direction's sines and cosines of st when the caller has them, else null
template <bool JOSEPH, class C, bool TWO_D, bool SEEDED = false, class T, class P>
__device__ __forceinline__ bool fit_step_on(Track<T, P> &st, C p[21], int k, T alpha, T mass2, int ms_on,
                                            const Surf &sf, float hx, float hy, float hz, double &chi2,
                                            unsigned &status, bool seeded = false, const Dir<T> *dir = nullptr)
{
    T cphi, sphi;
    if (k > 0) {
        Jac<T> J;
        if (!(dir ? propagate_from(st, alpha, sf, J, *dir) : propagate(st, alpha, sf, J))) {
            status |= reach_bits(st);
            return false;
        }
        if (SEEDED || seeded) transport_seeded<C>(p, JacAs<C>::get(J));
        else transport<C>(p, JacAs<C>::get(J));
        cphi = J.cphi1;
        sphi = J.sphi1;
    } else {
        sincos_pos(st.phi, sphi, cphi);
    }
    if (ms_on) status |= ms_noise<T, C>(st, sf, cphi, sphi, mass2, p);
    bool ok;
    if constexpr (TWO_D) {
        if constexpr (JOSEPH) ok = kf_update2d<true>(st, p, hx, hy, hz, sf, chi2);
        else ok = kf_update2d_mixed(st, p, hx, hy, hz, sf, chi2);
    } else {
        if constexpr (JOSEPH) ok = kf_update<true>(st, p, hx, hy, hz, sf, chi2);
        else ok = kf_update_mixed(st, p, hx, hy, hz, sf, chi2);
    }
    if (!ok) {
        status |= KF_ST_CHOL_FAIL;
        return false;
    }
    return true;
}

}  // namespace kfd
