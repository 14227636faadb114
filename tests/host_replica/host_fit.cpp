// host_fit.cpp -- the per-track fit of the device code (kf_track.cuh,
// kf_df.cuh and the fit section of kf_fit.cu) compiled for the host CPU, one
// track at a time.  Test and study tool only: the library never runs this.
//
// The device intrinsics the headers use are given host definitions with the
// same IEEE rounding (single and double precision, round to nearest; volatile
// stores keep the compiler from contracting or reassociating them).  Two
// functions differ from the GPU: the FP64 reciprocal approximation of the S
// pivots (rcp.approx.ftz.f64, ~20 bits) becomes the FP32 reciprocal (~24 bits),
// which the following Newton step refines all the same, and the single- and
// double-precision sines, cosines and logarithms are the C library's, which
// may differ from CUDA's in the last unit.  tests/host_replica.py assembles
// and builds it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { volatile float r = fmaf(a, b, c); return r; }
static inline float __frcp_rn(float a) { volatile float r = 1.0f / a; return r; }
static inline float __fsqrt_rn(float a) { volatile float r = sqrtf(a); return r; }
static inline float __fdiv_rn(float a, float b) { volatile float r = a / b; return r; }
static inline float __frsqrt_rn(float a) { volatile float r = 1.0f / sqrtf(a); return r; }
static inline double __dadd_rn(double a, double b) { volatile double r = a + b; return r; }
static inline double __dmul_rn(double a, double b) { volatile double r = a * b; return r; }
static inline int __double2hiint(double d) { uint64_t u; memcpy(&u, &d, 8); return (int)(u >> 32); }
static inline int __double2loint(double d) { uint64_t u; memcpy(&u, &d, 8); return (int)(u & 0xffffffffu); }
static inline double __hiloint2double(int h, int l)
{
    uint64_t u = ((uint64_t)(uint32_t)h << 32) | (uint32_t)l;
    double d;
    memcpy(&d, &u, 8);
    return d;
}
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline int __float_as_int(float f) { int u; memcpy(&u, &f, 4); return u; }
static inline float __int_as_float(int u) { float f; memcpy(&f, &u, 4); return f; }
using std::isfinite;
using std::max;
using std::min;
#define __noinline__ __attribute__((noinline))
struct HostDim3 {
    int x;
};
static HostDim3 threadIdx{0}, blockDim{1}, blockIdx{0};
static inline void __syncthreads() {}

#include "fit_track.h"

using namespace kfd;

// sp: [nsurf][9] per surface: kind, pos, half length or inner radius, outer
// radius, x/X0, sigma along the normal, sigma r-phi, sigma of the third
// coordinate, dr.  Arrays as kf_fit's, host memory; seed [6][n] FP32.
extern "C" void host_fit(int nsurf, const double *sp, double bz, double mass, int n, const int32_t *off,
                         const uint8_t *layer, const float *hx, const float *hy, const float *hz, const float *seed,
                         const int8_t *q, int seed_df, int n64, int fp64, int meas_model, double *o_state,
                         double *o_cov, double *o_chi2, int32_t *o_ndof, uint32_t *o_status)
{
    static Geom G;
    memset(&G, 0, sizeof G);
    G.n = nsurf;
    G.kbd = KAPPA * bz;
    G.kb = (float)G.kbd;
    G.mass2d = mass * mass;
    G.mass2 = (float)G.mass2d;
    for (int i = 0; i < nsurf; ++i) {
        const double *s = sp + 9 * i;
        Surf &d = G.s[i];
        d.kind = (int)s[0];
        d.posd = s[1];
        d.pos = (float)s[1];
        d.pos2 = (float)(s[1] * s[1]);
        d.pos2lo = (float)(s[1] * s[1] - (double)d.pos2);
        d.halfd = s[2];
        d.half = (float)s[2];
        d.rout = (float)s[3];
        d.x_x0d = s[4];
        d.x_x0 = (float)s[4];
        const double rad = d.kind == 0 ? s[5] : s[7], zz = d.kind == 0 ? s[7] : s[5];
        d.var_radd = rad * rad;
        d.var_rphid = s[6] * s[6];
        d.var_zzd = zz * zz;
        d.var_rad = (float)d.var_radd;
        d.var_rphi = (float)d.var_rphid;
        d.var_zz = (float)d.var_zzd;
        d.dr = d.kind == 0 ? (float)s[8] : 0.f;
    }
    FitArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.count = n;
    a.n64 = n64;
    a.seed_cov = 1e4;
    a.ms_on = 1;
    a.seed_df = seed_df;
    a.meas_model = meas_model;
    a.seed_state = seed;
    a.q = q;
    a.off = off;
    a.layer = layer;
    a.hx = hx;
    a.hy = hy;
    a.hz = hz;
    a.o_state = o_state;
    a.o_cov = o_cov;
    a.o_chi2 = o_chi2;
    a.o_ndof = o_ndof;
    a.o_status = o_status;
    for (int t = 0; t < n; ++t) {
        if (fp64) fit_track<true>(t, a, G.s, G.kb, G.mass2, G.kbd, G.mass2d);
        else if (meas_model == 1) fit_track<false, true>(t, a, G.s, G.kb, G.mass2, G.kbd, G.mass2d);
        else fit_track<false>(t, a, G.s, G.kb, G.mass2, G.kbd, G.mass2d);
    }
}
