// kf_common.cuh -- device-side types and small arithmetic helpers of libkf.
//
// Geometry is passed to every kernel by value (a few KB of kernel parameters)
// and copied into shared memory at block start, so concurrent calls with
// different detectors never race and divergent layer lookups hit shared memory
// instead of serialising in the constant cache.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/kf.h"

namespace kfd {

constexpr double KAPPA = 0.299792458e-2;  // GeV / (T cm): pT = KAPPA * B * rho
constexpr int MAX_SURF = KF_MAX_SURFACES;
constexpr float PI_F = 3.14159265358979323846f;

// One surface, FP32 and FP64 copies of what the kernels read.
struct Surf {
    int kind;   // 0 barrel, 1 disk
    int pad_;
    float pos, pos2, half, rout;  // pos2 + pos2lo: pos^2 as a float-float (barrel)
    float x_x0;
    float var_rad;   // variance along r-hat (barrel: sig_n^2, disk: sig_3^2)
    float var_rphi;  // along phi-hat
    float var_zz;    // along z (barrel: sig_3^2, disk: sig_n^2)
    float dr;        // barrel: radial half-extent of the layer's modules (model 1 window)
    float pos2lo;
    double posd, halfd, x_x0d, var_radd, var_rphid, var_zzd;
};

struct Geom {
    int n;
    int pad_;
    float kb;     // KAPPA * Bz
    float mass2;  // m^2
    double kbd, mass2d;
    Surf s[MAX_SURF];
};

// ------------------------------------------------------------ float-float
// An unevaluated sum hi + lo of two floats (Dekker / Knuth two-sum), used for
// the position and phi of the mixed-precision path: ~48 significant bits, so
// that storing 100 cm or pi does not cost the 1e-3 sigma accuracy target.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff ff_add(ff a, float b)
{
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    float h = __fadd_rn(s, e);
    float l = __fsub_rn(e, __fsub_rn(h, s));
    return {h, l};
}

// 2 pi as float-float
constexpr float TWO_PI_HI = 6.28318548202514648f;
constexpr float TWO_PI_LO = -1.74845553146951785e-07f;

__device__ __forceinline__ ff ff_wrap_phi(ff p)
{
    if (p.hi > PI_F) {
        p = ff_add(p, -TWO_PI_HI);
        p = ff_add(p, -TWO_PI_LO);
    } else if (p.hi <= -PI_F) {
        p = ff_add(p, TWO_PI_HI);
        p = ff_add(p, TWO_PI_LO);
    }
    return p;
}

__device__ __forceinline__ double wrap_phi_d(double p)
{
    const double PI = 3.14159265358979323846;
    if (p > PI) p -= 2.0 * PI;
    else if (p <= -PI) p += 2.0 * PI;
    return p;
}

// Position/angle accessors shared by the float-float (mixed) and double paths.
__device__ __forceinline__ float lead(ff a) { return a.hi; }
__device__ __forceinline__ double lead(double a) { return a; }
__device__ __forceinline__ ff inc(ff a, float d) { return ff_add(a, d); }
__device__ __forceinline__ double inc(double a, double d) { return a + d; }
__device__ __forceinline__ float resid(float m, ff a) { return __fsub_rn(__fsub_rn(m, a.hi), a.lo); }
__device__ __forceinline__ double resid(float m, double a) { return (double)m - a; }
__device__ __forceinline__ double to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_d(double a) { return a; }
template <class P> __device__ __forceinline__ P from_f(float v);
template <> __device__ __forceinline__ ff from_f<ff>(float v) { return {v, 0.f}; }
template <> __device__ __forceinline__ double from_f<double>(float v) { return (double)v; }
__device__ __forceinline__ ff wrap(ff p) { return ff_wrap_phi(p); }
__device__ __forceinline__ double wrap(double p) { return wrap_phi_d(p); }

// sin and cos of an angle held as float-float / double
__device__ __forceinline__ void sincos_pos(ff a, float &s, float &c)
{
    float s0, c0;
    sincosf(a.hi, &s0, &c0);
    s = fmaf(c0, a.lo, s0);
    c = fmaf(-s0, a.lo, c0);
}
__device__ __forceinline__ void sincos_pos(double a, double &s, double &c) { sincos(a, &s, &c); }

// x^2 + y^2 - R^2 for a point held in extended precision
__device__ __forceinline__ float radial_excess(ff x, ff y, float R2, float R2lo)
{
    float p1 = __fmul_rn(x.hi, x.hi), e1 = fmaf(x.hi, x.hi, -p1);
    float p2 = __fmul_rn(y.hi, y.hi), e2 = fmaf(y.hi, y.hi, -p2);
    float s, e, s2, e3;
    two_sum(p1, p2, s, e);
    two_sum(s, -R2, s2, e3);
    float lo = e + e3 - R2lo + e1 + e2 + 2.0f * (x.hi * x.lo + y.hi * y.lo);
    return s2 + lo;
}
__device__ __forceinline__ double radial_excess(double x, double y, double R2) { return x * x + y * y - R2; }

// ------------------------------------------------------------ small-angle helix factors
// For h = c s / 2: sinc(h) = sin h / h, cos h, and f1(h) = (cos h - sinc h) / (2 h)
// (the curvature derivative factor).  Taylor series for |h| < 0.5, direct forms above.
__device__ __forceinline__ void helix_factors(float h, float &sinc, float &ch, float &sh, float &f1)
{
    float ah = fabsf(h);
    if (ah < 0.5f) {
        float h2 = h * h;
        sinc = 1.f + h2 * (-1.f / 6.f + h2 * (1.f / 120.f + h2 * (-1.f / 5040.f + h2 * (1.f / 362880.f))));
        ch = 1.f + h2 * (-0.5f + h2 * (1.f / 24.f + h2 * (-1.f / 720.f + h2 * (1.f / 40320.f))));
        sh = h * sinc;
        f1 = h * (-1.f / 6.f + h2 * (1.f / 60.f + h2 * (-1.f / 1680.f + h2 * (1.f / 90720.f))));
    } else {
        sincosf(h, &sh, &ch);
        sinc = sh / h;
        f1 = (ch - sinc) / (2.f * h);
    }
}
__device__ __forceinline__ void helix_factors(double h, double &sinc, double &ch, double &sh, double &f1)
{
    double ah = fabs(h);
    if (ah < 0.25) {
        double h2 = h * h;
        // series to h^16: truncation below 1e-17 for |h| < 0.25
        sinc = 1.0 + h2 * (-1.0 / 6 + h2 * (1.0 / 120 + h2 * (-1.0 / 5040 + h2 * (1.0 / 362880 +
               h2 * (-1.0 / 39916800 + h2 * (1.0 / 6227020800.0 + h2 * (-1.0 / 1307674368000.0)))))));
        ch = 1.0 + h2 * (-0.5 + h2 * (1.0 / 24 + h2 * (-1.0 / 720 + h2 * (1.0 / 40320 +
             h2 * (-1.0 / 3628800 + h2 * (1.0 / 479001600.0 + h2 * (-1.0 / 87178291200.0)))))));
        sh = h * sinc;
        // f1 = sum_n (-1)^n n h^(2n-1) / (2n+1)!
        f1 = h * (-1.0 / 6 + h2 * (2.0 / 120 + h2 * (-3.0 / 5040 + h2 * (4.0 / 362880 +
             h2 * (-5.0 / 39916800 + h2 * (6.0 / 6227020800.0 + h2 * (-7.0 / 1307674368000.0)))))));
    } else {
        sincos(h, &sh, &ch);
        sinc = sh / h;
        f1 = (ch - sinc) / (2.0 * h);
    }
}

// ------------------------------------------------------------ conversions on the integer pipe
// On this GPU the FP64 pipe also executes F2F conversions and it is the fit's
// bottleneck, so float <-> double goes through bit operations on the (idle)
// integer pipe instead.  Float -> double is exact for normal numbers, zero,
// infinity and NaN (subnormal floats flush to zero); double -> float rounds
// the 29 dropped mantissa bits to nearest (ties away from zero) and flushes
// results below the float normal range to zero.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const unsigned ed = e == 0xffu ? 0x7ffu : (e == 0u ? 0u : e + 896u);
    const unsigned mm = e == 0u ? 0u : m;
    return __hiloint2double((int)(sign | (ed << 20) | (mm >> 3)), (int)(mm << 29));
}

__device__ __forceinline__ float d2f(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // float exponent field
    unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned r = (sign | ((unsigned)e << 23)) + m + ((lo >> 28) & 1u);  // carry may bump the exponent
    if (e <= 0) r = sign;                                              // below the normal range: signed zero
    if (e >= 255) r = sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);  // overflow, inf, NaN
    return __uint_as_float(r);
}

// ------------------------------------------------------------ FP64 3x3 solve
// Reciprocal in FP64 for the positive pivots of S: the hardware approximation
// rcp.approx.ftz.f64 (about 20 correct bits) refined by one Newton-Raphson step
// in the series form y (1 + e + e^2), e = 1 - d y, which triples the number of
// correct bits (cubic convergence), i.e. to full double precision.
__device__ __forceinline__ double rcp_d(double d)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
// The same with one quadratic Newton step, y (1 + e): twice the approximation's
// correct bits (about 40 of 53), for the pivots of an S whose entries come from
// an FP32 covariance (7 significant digits to begin with).
__device__ __forceinline__ double rcp_d_half(double d)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    return fma(y, fma(-d, y, 1.0), y);
}

// S = L D L^T with L unit lower triangular (square-root-free Cholesky).
struct Ldl3 {
    double l21, l31, l32, i1, i2, i3;  // L entries and 1/D
};

// FULL: reciprocals to full double precision (rcp_d); false: rcp_d_half, for an
// S formed from an FP32 covariance.
template <bool FULL = true>
__device__ __forceinline__ bool ldl3(double s11, double s21, double s22, double s31, double s32, double s33, Ldl3 &f)
{
    auto rcp = [](double v) { return FULL ? rcp_d(v) : rcp_d_half(v); };
    if (!(s11 > 0.0)) return false;
    f.i1 = rcp(s11);
    f.l21 = s21 * f.i1;
    f.l31 = s31 * f.i1;
    double d2 = fma(-f.l21, s21, s22);
    if (!(d2 > 0.0)) return false;
    f.i2 = rcp(d2);
    double t32 = fma(-f.l31, s21, s32);
    f.l32 = t32 * f.i2;
    double d3 = fma(-f.l32, t32, fma(-f.l31, s31, s33));
    if (!(d3 > 0.0)) return false;
    f.i3 = rcp(d3);
    return true;
}

// chi2 = r^T S^-1 r = sum_k (L^-1 r)_k^2 / D_k
__device__ __forceinline__ double ldl3_chi2(const Ldl3 &f, double r1, double r2, double r3)
{
    double z1 = r1;
    double z2 = fma(-f.l21, z1, r2);
    double z3 = fma(-f.l32, z2, fma(-f.l31, z1, r3));
    return fma(z3 * f.i3, z3, fma(z2 * f.i2, z2, z1 * f.i1 * z1));
}

// S^-1 = L^-T D^-1 L^-1 (symmetric, six entries), in type T
__device__ __forceinline__ float to_t(double v, float) { return d2f(v); }
__device__ __forceinline__ double to_t(double v, double) { return v; }

template <class T>
__device__ __forceinline__ void ldl3_inverse(const Ldl3 &f, T &a11, T &a21, T &a22, T &a31, T &a32, T &a33)
{
    const T z = T(0);
    T l21 = to_t(f.l21, z), l31 = to_t(f.l31, z), l32 = to_t(f.l32, z), i1 = to_t(f.i1, z), i2 = to_t(f.i2, z),
      i3 = to_t(f.i3, z);
    T m21 = -l21, m32 = -l32, m31 = l21 * l32 - l31;  // L^-1
    a33 = i3;
    a32 = m32 * i3;
    a31 = m31 * i3;
    a22 = i2 + m32 * a32;
    a21 = m21 * i2 + m31 * a32;
    a11 = i1 + m21 * m21 * i2 + m31 * a31;
}

}  // namespace kfd
