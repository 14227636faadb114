/*
 * kf_oracle.c -- plain, slow, FP64 CPU oracle for batched Kalman-filter
 * track fitting and best-hit track building (arXiv:1711.06571).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library; the two are written separately from the paper.
 *
 * Every routine works on one track at a time, in double precision, with full
 * 6x6 matrices and no use of symmetry or sparsity, so that each step can be
 * read against the method:
 *   - state in hybrid coordinates (x, y, z, 1/pT, phi, theta): Sec. 3
 *   - helix propagation in a uniform longitudinal field: Sec. 3
 *   - propagation to a layer surface, update on the plane tangent to the
 *     hit radius: Sec. 4.1
 *   - multiple scattering folded into the trajectory estimate: Sec. 2
 *   - seeding / building / final fit stages: Sec. 2
 *   - hit-selection data structure for building: Sec. 3.1
 * Where the paper gives no formula (helix equations, Jacobian, Highland
 * scattering angle, measurement covariance, seed estimate, binning, window,
 * chi2 cut) the reading used here is the one written out beside each routine.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared kf_oracle.c -lm
 * (-ffp-contract=off so that x86 and aarch64 hosts round identically).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* pT [GeV] = OR_KAPPA * B [T] * rho [cm] */
#define OR_KAPPA 0.299792458e-2
#define OR_PI 3.14159265358979323846
/* a transverse path longer than this (cm) counts as no intersection */
#define OR_MAX_PATH 1.0e6

/* status bits, oracle's own copy */
#define OR_ST_NO_INTERSECT 1u
#define OR_ST_CHOL_FAIL 2u
#define OR_ST_NONFINITE 4u
#define OR_ST_CAND_CAPPED 8u
#define OR_ST_GRAZING 16u
#define OR_ST_THETA_RANGE 32u

/* One detector surface.  kind 0: barrel cylinder r = pos, |z| <= half_or_rin.
 * kind 1: disk z = pos, half_or_rin <= r <= r_out.
 * sig_n: resolution along the surface normal, sig_rphi: along phi-hat,
 * sig_3: along z (barrel) or r (disk).  x_x0: thickness in radiation lengths
 * at normal incidence. */
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
    double dr; /* barrel: radial half-extent of the layer's modules (0: a cylinder) */
} or_surf;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double wrap_phi(double p)
{
    /* into (-pi, pi]; non-finite values are returned as they are */
    if (!isfinite(p)) return p;
    if (p > OR_PI || p <= -OR_PI) p = remainder(p, 2.0 * OR_PI);
    if (p <= -OR_PI) p += 2.0 * OR_PI;
    return p;
}

/* signed transverse curvature, dphi/ds, of charge q with state st in field bz.
 * Sign reading: F = q v x B with B along +z turns a positive charge clockwise,
 * so dphi/ds = -q * kappa * B / pT. */
double or_curvature(const double st[6], int q, double bz)
{
    return -(double)q * OR_KAPPA * bz * st[3];
}

/* ------------------------------------------------------------------ */
/* helix (Sec. 3: uniform longitudinal field, hybrid coordinates)      */
/* ------------------------------------------------------------------ */

/* State after transverse path length s along the helix.  Chord form:
 *   phi(s) = phi + c s
 *   x(s)   = x + s * sinc(c s / 2) * cos(phi + c s / 2)
 *   y(s)   = y + s * sinc(c s / 2) * sin(phi + c s / 2)
 *   z(s)   = z + s * cot(theta)
 * which equals x + (sin phi(s) - sin phi)/c, y - (cos phi(s) - cos phi)/c and
 * stays exact as c -> 0 (straight line). */
void or_helix_at(const double st[6], double c, double s, double out[6])
{
    double h = 0.5 * c * s;
    double sinc = (fabs(h) < 1e-4) ? 1.0 - h * h / 6.0 + h * h * h * h / 120.0 : sin(h) / h;
    double phim = st[4] + h;
    out[0] = st[0] + s * sinc * cos(phim);
    out[1] = st[1] + s * sinc * sin(phim);
    out[2] = st[2] + s * cos(st[5]) / sin(st[5]);
    out[3] = st[3];
    out[4] = wrap_phi(st[4] + c * s);
    out[5] = st[5];
}

/* Path length to the cylinder r = R along the helix.  From inside (r < R):
 * the smallest s > 0 with x(s)^2 + y(s)^2 = R^2 (the outgoing crossing).
 * From outside or on it (r >= R, possible only when a measurement has pulled
 * the state just past a closely following surface): the crossing of smallest
 * |s|, which is then behind the state (s <= 0).  Closed form (intersection of
 * the helix circle with the cylinder circle), then a Newton polish on the
 * exact helix.  Returns 0 or OR_ST_NO_INTERSECT. */
int or_path_to_barrel(const double st[6], double c, double R, double *s_out)
{
    double x = st[0], y = st[1];
    double cp = cos(st[4]), sp = sin(st[4]);
    double r2 = x * x + y * y;
    int inside = r2 < R * R;
    double s;
    if (c == 0.0) {
        /* straight line: s^2 + 2 (p.t) s + r2 - R^2 = 0 */
        double b = x * cp + y * sp;
        double disc = b * b + (R * R - r2);
        double s1, s2;
        if (disc < 0.0) return (int)OR_ST_NO_INTERSECT;
        s1 = -b + sqrt(disc);
        s2 = -b - sqrt(disc);
        s = inside ? s1 : (fabs(s1) < fabs(s2) ? s1 : s2);
    } else {
        /* circle of radius rho = 1/|c| centred at C = p + n/c, n = (-sin phi, cos phi) */
        double rho = 1.0 / fabs(c);
        double turn = 2.0 * OR_PI / fabs(c); /* path of one full turn */
        double cx = x - sp / c, cy = y + cp / c;
        double d = sqrt(cx * cx + cy * cy);
        double pn = -x * sp + y * cp;
        /* a = (R^2 - rho^2 + d^2) / (2 d), using d^2 - rho^2 = r2 + 2 (p.n)/c */
        double a = (R * R + r2 + 2.0 * pn / c) / (2.0 * d);
        double h2 = R * R - a * a;
        double best = 0.0;
        int k, have = 0;
        if (d + rho < R || fabs(d - rho) > R || h2 < 0.0) return (int)OR_ST_NO_INTERSECT;
        for (k = 0; k < 2; ++k) {
            double sg = k ? -1.0 : 1.0;
            double hh = sqrt(h2);
            double X = a * cx / d - sg * hh * cy / d;
            double Y = a * cy / d + sg * hh * cx / d;
            double dx = X - x, dy = Y - y;
            double L = sqrt(dx * dx + dy * dy);
            double arg = 0.5 * L * fabs(c);
            double sk;
            if (arg > 1.0) arg = 1.0;
            /* forward arc to the point, in [0, turn): the chord leads the tangent
             * for arcs shorter than half a turn */
            if (dx * cp + dy * sp > 0.0)
                sk = 2.0 * asin(arg) / fabs(c);
            else
                sk = (2.0 * OR_PI - 2.0 * asin(arg)) / fabs(c);
            if (inside) {
                if (sk > 0.0 && (!have || sk < best)) {
                    best = sk;
                    have = 1;
                }
            } else {
                double sb = sk - turn; /* the same point reached backwards */
                double cand = fabs(sk) < fabs(sb) ? sk : sb;
                if (!have || fabs(cand) < fabs(best)) {
                    best = cand;
                    have = 1;
                }
            }
        }
        if (!have) return (int)OR_ST_NO_INTERSECT;
        s = best;
    }
    /* Newton polish on g(s) = x(s)^2 + y(s)^2 - R^2 */
    {
        int it;
        for (it = 0; it < 8; ++it) {
            double o[6], g, gp, ds;
            or_helix_at(st, c, s, o);
            g = o[0] * o[0] + o[1] * o[1] - R * R;
            gp = 2.0 * (o[0] * cos(o[4]) + o[1] * sin(o[4]));
            if (gp == 0.0) break;
            ds = g / gp;
            s -= ds;
            if (fabs(ds) <= 1e-15 * (1.0 + fabs(s))) break;
        }
    }
    if (!isfinite(s) || (inside && !(s > 0.0))) return (int)OR_ST_NO_INTERSECT;
    *s_out = s;
    return 0;
}

/* Path length to the disk z = Z: s = (Z - z) tan(theta), of either sign (a
 * measurement may have pulled the state just past a closely following disk);
 * |s| > OR_MAX_PATH (theta at pi/2 up to rounding) is no intersection. */
int or_path_to_disk(const double st[6], double Z, double *s_out)
{
    double cot = cos(st[5]) / sin(st[5]);
    double s;
    if (cot == 0.0) return (int)OR_ST_NO_INTERSECT;
    s = (Z - st[2]) / cot;
    if (!isfinite(s) || fabs(s) > OR_MAX_PATH) return (int)OR_ST_NO_INTERSECT;
    *s_out = s;
    return 0;
}

/* d x(s) / d c and d y(s) / d c at fixed s (x(s), y(s) as in or_helix_at).
 * Direct form (s cos phi(s) - dx)/c, (s sin phi(s) - dy)/c when |c s| > 0.01;
 * its Taylor series in h = c s / 2 otherwise. */
static void dxy_dc(const double st[6], double c, double s, double *dxdc, double *dydc)
{
    double u = c * s;
    if (fabs(u) > 0.01) {
        double phi1 = st[4] + u;
        double dx = (sin(phi1) - sin(st[4])) / c;
        double dy = -(cos(phi1) - cos(st[4])) / c;
        *dxdc = (s * cos(phi1) - dx) / c;
        *dydc = (s * sin(phi1) - dy) / c;
    } else {
        /* (s cos phi' - dx)/c = s^2 [cos(phim) f1 - sin(phim) f2], with
         * f1 = (cos h - sin h / h) / (2h), f2 = sin h / (2h), phim = phi + h */
        double h = 0.5 * u, h2 = h * h;
        double f1 = -h / 6.0 + h * h2 / 60.0 - h * h2 * h2 / 1680.0 + h * h2 * h2 * h2 / 90720.0;
        double f2 = 0.5 * (1.0 - h2 / 6.0 + h2 * h2 / 120.0 - h2 * h2 * h2 / 5040.0);
        double phim = st[4] + h;
        *dxdc = s * s * (cos(phim) * f1 - sin(phim) * f2);
        *dydc = s * s * (sin(phim) * f1 + cos(phim) * f2);
    }
}

/* Propagate to a surface and return the 6x6 Jacobian J[i*6+j] = d out_i / d st_j
 * of the surface-constrained map (Sec. 2.1 / Sec. 4.1).  J = A + u w^T with
 *   A = d out / d st at fixed s,
 *   u = d out / d s,
 *   w = d s / d st from the surface condition g(out) = 0:
 *       w = -(dg/d st at fixed s) / (dg/ds).
 * J may be NULL.  Returns 0, OR_ST_NO_INTERSECT, or OR_ST_NO_INTERSECT |
 * OR_ST_THETA_RANGE when theta is outside (0, pi). */
int or_propagate(const double st[6], int q, double bz, const or_surf *sf, double out[6], double *J)
{
    double c = or_curvature(st, q, bz);
    double alpha = -(double)q * OR_KAPPA * bz; /* dc / d(1/pT) */
    double s;
    int rc;
    /* theta outside (0, pi): an update has carried the polar angle through the
     * pole of the parametrisation, where dz/ds = cot(theta) diverges and changes
     * sign.  Reading: the state has no next crossing and the track ends. */
    if (!(sin(st[5]) > 0.0)) return (int)(OR_ST_NO_INTERSECT | OR_ST_THETA_RANGE);
    if (sf->kind == 0)
        rc = or_path_to_barrel(st, c, sf->pos, &s);
    else
        rc = or_path_to_disk(st, sf->pos, &s);
    if (rc) return rc;
    or_helix_at(st, c, s, out);
    if (sf->kind == 1) out[2] = sf->pos; /* on the plane by construction */
    if (J) {
        double A[36], u[6], w[6], dg[6], dgds = 0.0;
        double phi1 = st[4] + c * s;
        double dxdc, dydc, sn = sin(st[5]);
        int i, j;
        memset(A, 0, sizeof A);
        for (i = 0; i < 6; ++i) A[i * 6 + i] = 1.0;
        dxy_dc(st, c, s, &dxdc, &dydc);
        /* x' = x + dx(s, c, phi): d/dphi = -(y' - y), d/d(1/pT) = alpha dx/dc */
        A[0 * 6 + 3] = alpha * dxdc;
        A[0 * 6 + 4] = -(out[1] - st[1]);
        A[1 * 6 + 3] = alpha * dydc;
        A[1 * 6 + 4] = (out[0] - st[0]);
        /* z' = z + s cot(theta) */
        A[2 * 6 + 5] = -s / (sn * sn);
        /* phi' = phi + c s */
        A[4 * 6 + 3] = alpha * s;
        /* d out / d s */
        u[0] = cos(phi1);
        u[1] = sin(phi1);
        u[2] = cos(st[5]) / sn;
        u[3] = 0.0;
        u[4] = c;
        u[5] = 0.0;
        /* surface condition */
        for (j = 0; j < 6; ++j) dg[j] = 0.0;
        if (sf->kind == 0) {
            /* g = x'^2 + y'^2 - R^2 */
            for (j = 0; j < 6; ++j) dg[j] = 2.0 * (out[0] * A[0 * 6 + j] + out[1] * A[1 * 6 + j]);
            dgds = 2.0 * (out[0] * u[0] + out[1] * u[1]);
        } else {
            /* g = z' - Z */
            for (j = 0; j < 6; ++j) dg[j] = A[2 * 6 + j];
            dgds = u[2];
        }
        for (j = 0; j < 6; ++j) w[j] = -dg[j] / dgds;
        for (i = 0; i < 6; ++i)
            for (j = 0; j < 6; ++j) J[i * 6 + j] = A[i * 6 + j] + u[i] * w[j];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* multiple scattering (Sec. 2), Highland form of the PDG               */
/* ------------------------------------------------------------------ */

/* theta0 = 13.6 MeV / (beta c p) * sqrt(t) * (1 + 0.038 ln(t / beta^2)),
 * unit charge, p in GeV, t = thickness in radiation lengths along the path. */
double or_highland(double p, double mass, double t)
{
    double E, beta;
    if (!(p > 0.0) || isinf(p)) return 0.0;
    E = sqrt(p * p + mass * mass);
    beta = p / E;
    return 0.0136 / (beta * p) * sqrt(t) * (1.0 + 0.038 * log(t / (beta * beta)));
}

/* cos of the angle between the direction and the surface normal */
double or_cos_incidence(const double st[6], const or_surf *sf)
{
    if (sf->kind == 0) {
        double r = sqrt(st[0] * st[0] + st[1] * st[1]);
        return sin(st[5]) * (st[0] * cos(st[4]) + st[1] * sin(st[4])) / r;
    }
    return cos(st[5]);
}

/* Add the process noise of crossing surface sf to P (6x6), evaluated at st:
 * t = (x/X0) / max(|cos alpha|, 0.05);  P_theta,theta += theta0^2,
 * P_phi,phi += theta0^2 / sin^2(theta).  Returns OR_ST_GRAZING when the
 * incidence guard was used. */
int or_ms_noise(const double st[6], double mass, const or_surf *sf, double P[36])
{
    double ca = fabs(or_cos_incidence(st, sf));
    unsigned flag = 0;
    double t, p, th0, sn;
    if (sf->x_x0 <= 0.0) return 0;
    if (ca < 0.05) {
        ca = 0.05;
        flag = OR_ST_GRAZING;
    }
    t = sf->x_x0 / ca;
    sn = sin(st[5]);
    p = 1.0 / (fabs(st[3]) * sn);
    th0 = or_highland(p, mass, t);
    P[5 * 6 + 5] += th0 * th0;
    P[4 * 6 + 4] += th0 * th0 / (sn * sn);
    return (int)flag;
}

/* ------------------------------------------------------------------ */
/* measurement model and KF update (Sec. 4.1: tangent-plane update)    */
/* ------------------------------------------------------------------ */

/* R = sig_n^2 n n^T + sig_rphi^2 e_phi e_phi^T + sig_3^2 e3 e3^T at the hit
 * azimuth; barrel: n = radial, e3 = z; disk: n = z, e3 = radial. */
void or_meas_cov(const or_surf *sf, const double hit[3], double R[9])
{
    double r = sqrt(hit[0] * hit[0] + hit[1] * hit[1]);
    double cs = hit[0] / r, sn = hit[1] / r;
    double er[3] = {cs, sn, 0.0}, ep[3] = {-sn, cs, 0.0}, ez[3] = {0.0, 0.0, 1.0};
    const double *n, *e3;
    int i, j;
    if (sf->kind == 0) {
        n = er;
        e3 = ez;
    } else {
        n = ez;
        e3 = er;
    }
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j)
            R[i * 3 + j] = sf->sig_n * sf->sig_n * n[i] * n[j] + sf->sig_rphi * sf->sig_rphi * ep[i] * ep[j] +
                           sf->sig_3 * sf->sig_3 * e3[i] * e3[j];
}

/* Cholesky L L^T = S of a 3x3 SPD matrix; returns 0 or OR_ST_CHOL_FAIL */
static int chol3(const double S[9], double L[9])
{
    int i, j, k;
    memset(L, 0, 9 * sizeof(double));
    for (j = 0; j < 3; ++j) {
        double d = S[j * 3 + j];
        for (k = 0; k < j; ++k) d -= L[j * 3 + k] * L[j * 3 + k];
        if (!(d > 0.0)) return (int)OR_ST_CHOL_FAIL;
        L[j * 3 + j] = sqrt(d);
        for (i = j + 1; i < 3; ++i) {
            double v = S[i * 3 + j];
            for (k = 0; k < j; ++k) v -= L[i * 3 + k] * L[j * 3 + k];
            L[i * 3 + j] = v / L[j * 3 + j];
        }
    }
    return 0;
}

/* chi2 = r^T S^-1 r of residual r with innovation covariance S, via Cholesky */
int or_chi2(const double S[9], const double r[3], double *chi2)
{
    double L[9], y[3];
    int i, k, rc = chol3(S, L);
    if (rc) return rc;
    for (i = 0; i < 3; ++i) {
        double v = r[i];
        for (k = 0; k < i; ++k) v -= L[i * 3 + k] * y[k];
        y[i] = v / L[i * 3 + i];
    }
    *chi2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    return 0;
}

/* Kalman update with the 3-D hit position, H = [I3 | 0]:
 *   r = m - H x,  S = H P H^T + R,  chi2 = r^T S^-1 r,
 *   K = P H^T S^-1,  x += K r,  P = (I - K H) P (I - K H)^T + K R K^T,
 *   P = (P + P^T) / 2.
 * phi is wrapped into (-pi, pi].  Returns 0 or OR_ST_CHOL_FAIL. */
int or_update(double st[6], double P[36], const double hit[3], const double R[9], double *chi2)
{
    double r[3], S[9], L[9], Li[9], Si[9], K[18], HP[18], Pn[36];
    int i, j, k, rc;
    for (i = 0; i < 3; ++i) r[i] = hit[i] - st[i];
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) S[i * 3 + j] = P[i * 6 + j] + R[i * 3 + j];
    rc = chol3(S, L);
    if (rc) return rc;
    /* L^-1 by forward substitution, then S^-1 = L^-T L^-1 */
    memset(Li, 0, sizeof Li);
    for (j = 0; j < 3; ++j) {
        Li[j * 3 + j] = 1.0 / L[j * 3 + j];
        for (i = j + 1; i < 3; ++i) {
            double v = 0.0;
            for (k = j; k < i; ++k) v -= L[i * 3 + k] * Li[k * 3 + j];
            Li[i * 3 + j] = v / L[i * 3 + i];
        }
    }
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) {
            double v = 0.0;
            for (k = 0; k < 3; ++k) v += Li[k * 3 + i] * Li[k * 3 + j];
            Si[i * 3 + j] = v;
        }
    or_chi2(S, r, chi2);
    /* H P: the first three rows of P */
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 6; ++j) HP[i * 6 + j] = P[i * 6 + j];
    /* K = P H^T S^-1 (6x3) */
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 3; ++j) {
            double v = 0.0;
            for (k = 0; k < 3; ++k) v += P[i * 6 + k] * Si[k * 3 + j];
            K[i * 3 + j] = v;
        }
    for (i = 0; i < 6; ++i) {
        double v = 0.0;
        for (k = 0; k < 3; ++k) v += K[i * 3 + k] * r[k];
        st[i] += v;
    }
    st[4] = wrap_phi(st[4]);
    /* Joseph form P = (I - K H) P (I - K H)^T + K R K^T: equal to P - K H P
     * for the optimal gain, but a sum of positive semi-definite terms, so it
     * stays positive definite when the seed covariance (1e4 * I) makes the
     * position block of P six to nine orders of magnitude larger than R. */
    {
        double M[36], MP[36], KR[18];
        (void)HP;
        for (i = 0; i < 6; ++i)
            for (j = 0; j < 6; ++j) M[i * 6 + j] = (i == j ? 1.0 : 0.0) - (j < 3 ? K[i * 3 + j] : 0.0);
        for (i = 0; i < 6; ++i)
            for (j = 0; j < 6; ++j) {
                double v = 0.0;
                for (k = 0; k < 6; ++k) v += M[i * 6 + k] * P[k * 6 + j];
                MP[i * 6 + j] = v;
            }
        for (i = 0; i < 6; ++i)
            for (j = 0; j < 3; ++j) {
                double v = 0.0;
                for (k = 0; k < 3; ++k) v += K[i * 3 + k] * R[k * 3 + j];
                KR[i * 3 + j] = v;
            }
        for (i = 0; i < 6; ++i)
            for (j = 0; j < 6; ++j) {
                double v = 0.0;
                for (k = 0; k < 6; ++k) v += MP[i * 6 + k] * M[j * 6 + k];
                for (k = 0; k < 3; ++k) v += KR[i * 3 + k] * K[j * 3 + k];
                Pn[i * 6 + j] = v;
            }
    }
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) P[i * 6 + j] = 0.5 * (Pn[i * 6 + j] + Pn[j * 6 + i]);
    return 0;
}

/* P <- J P J^T (plain dense product) */
void or_transport(const double J[36], double P[36])
{
    double T[36];
    int i, j, k;
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) {
            double v = 0.0;
            for (k = 0; k < 6; ++k) v += J[i * 6 + k] * P[k * 6 + j];
            T[i * 6 + j] = v;
        }
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) {
            double v = 0.0;
            for (k = 0; k < 6; ++k) v += T[i * 6 + k] * J[j * 6 + k];
            P[i * 6 + j] = v;
        }
}

/* ------------------------------------------------------------------ */
/* seed estimate (Sec. 2: seeding gives the initial estimate from a few */
/* inner hits; the estimate itself is a reading, see below)             */
/* ------------------------------------------------------------------ */

/* Circle through the three hits in x-y; signed curvature
 *   k = 2 (a x b)_z / (|a| |b| |b - a|),  a = p2 - p1, b = p3 - p1
 * (k > 0: counter-clockwise).  q = -sign(k) (q = +1 when k == 0),
 * 1/pT = |k| / (kappa |B|) (0 without field); phi = direction of the chord p1->p2 minus half the
 * turning angle along it; theta = atan2(arc13, z3 - z1) with arc13 the
 * transverse arc length p1 -> p3; position = hit 1. */
void or_seed(const double h1[3], const double h2[3], const double h3[3], double bz, double st[6], int *q)
{
    double ax = h2[0] - h1[0], ay = h2[1] - h1[1];
    double bx = h3[0] - h1[0], by = h3[1] - h1[1];
    double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
    double lab = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    double cr = ax * by - ay * bx;
    double k = 2.0 * cr / (la * lb * lab);
    double ak = fabs(k);
    double sg = (k > 0.0) ? 1.0 : ((k < 0.0) ? -1.0 : 0.0);
    double arc13 = (ak > 0.0) ? 2.0 * asin(fmin(1.0, 0.5 * lb * ak)) / ak : lb;
    st[0] = h1[0];
    st[1] = h1[1];
    st[2] = h1[2];
    st[3] = (bz != 0.0) ? ak / (OR_KAPPA * fabs(bz)) : 0.0; /* no field: 1/pT unmeasurable, set 0 */
    st[4] = wrap_phi(atan2(ay, ax) - sg * asin(fmin(1.0, 0.5 * la * ak)));
    st[5] = atan2(arc13, h3[2] - h1[2]);
    *q = (k > 0.0) ? -1 : 1;
}

/* Which hits of a track make its seed: hit 0, then the first hit at least
 * OR_SEED_DMIN cm (transverse) from it, then the first later hit at least
 * OR_SEED_DMIN cm from that one; indices 1, 2 if no such hits exist.  On a
 * barrel with layers further apart than OR_SEED_DMIN this is hits 0, 1, 2;
 * it skips the near-duplicate hits a track leaves where a disk and a barrel
 * overlap, which make a three-point circle meaningless. */
#define OR_SEED_DMIN 2.0
void or_seed_hits(int nh, const float *hx, const float *hy, int *i1, int *i2)
{
    int j, a = -1, b = -1;
    for (j = 1; j < nh; ++j) {
        double dx = (double)hx[j] - hx[0], dy = (double)hy[j] - hy[0];
        if (dx * dx + dy * dy >= OR_SEED_DMIN * OR_SEED_DMIN) {
            a = j;
            break;
        }
    }
    if (a > 0)
        for (j = a + 1; j < nh; ++j) {
            double dx = (double)hx[j] - hx[a], dy = (double)hy[j] - hy[a];
            if (dx * dx + dy * dy >= OR_SEED_DMIN * OR_SEED_DMIN) {
                b = j;
                break;
            }
        }
    if (a < 0 || b < 0) {
        a = 1;
        b = 2;
    }
    *i1 = a;
    *i2 = b;
}

/* ------------------------------------------------------------------ */
/* track fit (Sec. 2: fitting = the KF applied over a known hit list)  */
/* ------------------------------------------------------------------ */

typedef struct {
    double bz;
    double mass;
    double seed_cov; /* seed covariance = seed_cov * I6 */
    int32_t ms_on;   /* add multiple-scattering noise */
    int32_t meas_model; /* 0: 3-D hit on the layer surface; 1: on the hit's own radius, 2-D (Sec. 4.1) */
} or_fit_cfg;

/* ------------------------------------------------------------------ */
/* measurement model 1 (Sec. 4.1, non-ideal geometry): a barrel hit need  */
/* not lie on its layer's average cylinder; the state is carried to the   */
/* cylinder through the hit and updated on the plane tangent to it there, */
/* with the two coordinates measured on that plane: r-phi and z.  The    */
/* first hit of a fit is the exception: the state starts there, with no   */
/* propagation, so the hit's radius is the state's own and the update is  */
/* the 3-D one of model 0 (a reading: the surface's radial resolution     */
/* sig_n then fixes the start on the hit's cylinder).                     */
/* ------------------------------------------------------------------ */

/* the cylinder through a barrel hit: the layer surface with the hit's radius */
static or_surf hit_cylinder(const or_surf *sf, const double hit[3])
{
    or_surf h = *sf;
    h.pos = sqrt(hit[0] * hit[0] + hit[1] * hit[1]);
    return h;
}

/* 2-D update on the tangent plane at the hit azimuth: H (2x6) has rows
 * (-sin a, cos a, 0, 0, 0, 0) and (0, 0, 1, 0, 0, 0) with a the hit azimuth,
 * R = diag(sig_rphi^2, sig_3^2), r = H (m - x).  Joseph form, symmetrised.
 * Returns 0 or OR_ST_CHOL_FAIL. */
int or_update2d(double st[6], double P[36], const double hit[3], const or_surf *sf, double *chi2)
{
    const double rh = sqrt(hit[0] * hit[0] + hit[1] * hit[1]);
    const double ca = hit[0] / rh, sa = hit[1] / rh;
    double H[12] = {0}, R2[4] = {sf->sig_rphi * sf->sig_rphi, 0.0, 0.0, sf->sig_3 * sf->sig_3};
    double r[2], HP[12], S[4], Si[4], det, K[12], M[36], MP[36], Pn[36];
    int i, j, k;
    H[0 * 6 + 0] = -sa;
    H[0 * 6 + 1] = ca;
    H[1 * 6 + 2] = 1.0;
    r[0] = -sa * (hit[0] - st[0]) + ca * (hit[1] - st[1]);
    r[1] = hit[2] - st[2];
    for (i = 0; i < 2; ++i)
        for (j = 0; j < 6; ++j) {
            double v = 0.0;
            for (k = 0; k < 6; ++k) v += H[i * 6 + k] * P[k * 6 + j];
            HP[i * 6 + j] = v;
        }
    for (i = 0; i < 2; ++i)
        for (j = 0; j < 2; ++j) {
            double v = R2[i * 2 + j];
            for (k = 0; k < 6; ++k) v += HP[i * 6 + k] * H[j * 6 + k];
            S[i * 2 + j] = v;
        }
    det = S[0] * S[3] - S[1] * S[2];
    if (!(S[0] > 0.0) || !(det > 0.0)) return (int)OR_ST_CHOL_FAIL;
    Si[0] = S[3] / det;
    Si[1] = -S[1] / det;
    Si[2] = -S[2] / det;
    Si[3] = S[0] / det;
    *chi2 = r[0] * (Si[0] * r[0] + Si[1] * r[1]) + r[1] * (Si[2] * r[0] + Si[3] * r[1]);
    /* K = P H^T S^-1 (6x2) */
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 2; ++j) {
            double v = 0.0;
            for (k = 0; k < 2; ++k) v += HP[k * 6 + i] * Si[k * 2 + j];
            K[i * 2 + j] = v;
        }
    for (i = 0; i < 6; ++i) st[i] += K[i * 2 + 0] * r[0] + K[i * 2 + 1] * r[1];
    st[4] = wrap_phi(st[4]);
    /* Joseph: (I - K H) P (I - K H)^T + K R K^T */
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) M[i * 6 + j] = (i == j ? 1.0 : 0.0) - (K[i * 2 + 0] * H[0 * 6 + j] + K[i * 2 + 1] * H[1 * 6 + j]);
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) {
            double v = 0.0;
            for (k = 0; k < 6; ++k) v += M[i * 6 + k] * P[k * 6 + j];
            MP[i * 6 + j] = v;
        }
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) {
            double v = 0.0;
            for (k = 0; k < 6; ++k) v += MP[i * 6 + k] * M[j * 6 + k];
            v += K[i * 2 + 0] * R2[0] * K[j * 2 + 0] + K[i * 2 + 1] * R2[3] * K[j * 2 + 1];
            Pn[i * 6 + j] = v;
        }
    for (i = 0; i < 6; ++i)
        for (j = 0; j < 6; ++j) P[i * 6 + j] = 0.5 * (Pn[i * 6 + j] + Pn[j * 6 + i]);
    return 0;
}

/* chi2 of a hit under model 1 without updating */
static int or_chi2_2d(const double st[6], const double P[36], const double hit[3], const or_surf *sf, double *chi2)
{
    double s2[6], P2[36];
    memcpy(s2, st, sizeof s2);
    memcpy(P2, P, sizeof P2);
    return or_update2d(s2, P2, hit, sf, chi2);
}

/* Fit one track over its hits in path order.  The seed is placed at hit 1
 * with covariance seed_cov * I; hit 1 is used with no propagation; every
 * later hit: propagate to its surface, transport P, add scattering noise,
 * update.  A failed propagation ends the track (later hits unused).
 * If lin_ref is given (nh x 6 reference states on the surfaces), the
 * propagation is replaced by its linearisation about that trajectory:
 *   x_k = ref_k + J(ref_{k-1}) (x_{k-1} - ref_{k-1})
 * which turns the filter into a linear Gaussian one (used to pin the update
 * equations against a global least-squares fit).
 * Outputs: state at the last used hit, its 6x6 covariance, sum of chi2,
 * ndof = 2 * used - 5, number of used hits; returns the status bits. */
/* or_fit_one with the initial covariance P0 (6x6) instead of seed_cov * I when
 * P0 is given */
static unsigned or_fit_from(const or_fit_cfg *cfg, const or_surf *surfs, int nh, const uint8_t *layer,
                            const float *hx, const float *hy, const float *hz, const double seed[6], const double *P0,
                            int q, const double *lin_ref, double st[6], double P[36], double *chi2_sum, int *ndof,
                            int *n_used, double *chi2_each)
{
    unsigned status = 0;
    int k, i;
    memcpy(st, seed, 6 * sizeof(double));
    memset(P, 0, 36 * sizeof(double));
    for (i = 0; i < 6; ++i) P[i * 6 + i] = cfg->seed_cov;
    if (P0) memcpy(P, P0, 36 * sizeof(double));
    *chi2_sum = 0.0;
    *n_used = 0;
    for (k = 0; k < nh; ++k) {
        double hit[3] = {(double)hx[k], (double)hy[k], (double)hz[k]};
        const int m1 = cfg->meas_model == 1 && k > 0 && surfs[layer[k]].kind == 0;
        const or_surf hcyl = hit_cylinder(&surfs[layer[k]], hit);
        const or_surf *sf = m1 ? &hcyl : &surfs[layer[k]];
        double Rm[9], chi2 = 0.0;
        int rc;
        if (k > 0) {
            double nx[6], J[36];
            if (lin_ref) {
                double dv[6], o[6];
                rc = or_propagate(&lin_ref[(k - 1) * 6], q, cfg->bz, sf, o, J);
                if (rc) {
                    status |= (unsigned)rc;
                    break;
                }
                for (i = 0; i < 6; ++i) dv[i] = st[i] - lin_ref[(k - 1) * 6 + i];
                dv[4] = wrap_phi(dv[4]);
                for (i = 0; i < 6; ++i) {
                    int j;
                    double v = lin_ref[k * 6 + i];
                    for (j = 0; j < 6; ++j) v += J[i * 6 + j] * dv[j];
                    nx[i] = v;
                }
                nx[4] = wrap_phi(nx[4]);
            } else {
                rc = or_propagate(st, q, cfg->bz, sf, nx, J);
                if (rc) {
                    status |= (unsigned)rc;
                    break;
                }
            }
            memcpy(st, nx, sizeof nx);
            or_transport(J, P);
        }
        if (cfg->ms_on) status |= (unsigned)or_ms_noise(st, cfg->mass, sf, P);
        if (m1) {
            rc = or_update2d(st, P, hit, sf, &chi2);
        } else {
            or_meas_cov(sf, hit, Rm);
            rc = or_update(st, P, hit, Rm, &chi2);
        }
        if (rc) {
            status |= (unsigned)rc;
            break;
        }
        if (chi2_each) chi2_each[k] = chi2;
        *chi2_sum += chi2;
        *n_used += 1;
    }
    for (i = 0; i < 6; ++i)
        if (!isfinite(st[i])) status |= OR_ST_NONFINITE;
    *ndof = 2 * (*n_used) - 5;
    return status;
}

unsigned or_fit_one(const or_fit_cfg *cfg, const or_surf *surfs, int nh, const uint8_t *layer, const float *hx,
                    const float *hy, const float *hz, const double seed[6], int q, const double *lin_ref,
                    double st[6], double P[36], double *chi2_sum, int *ndof, int *n_used, double *chi2_each)
{
    return or_fit_from(cfg, surfs, nh, layer, hx, hy, hz, seed, NULL, q, lin_ref, st, P, chi2_sum, ndof, n_used,
                       chi2_each);
}

/* Fit tracks [t0, t1) of a batch.  Hits are CSR: track t owns hits
 * offsets[t] .. offsets[t+1]-1 in path order.  If seeds is NULL the seed of
 * each track is estimated from three of its first hits (or_seed_hits, or_seed);
 * seeds_out
 * (n x 6) and q_out receive the seed used.  Outputs are track-major:
 * state (n x 6), cov (n x 36), chi2, ndof, status. */
void or_fit_tracks(const or_fit_cfg *cfg, const or_surf *surfs, int t0, int t1, const int32_t *offsets,
                   const uint8_t *layer, const float *hx, const float *hy, const float *hz, const double *seeds,
                   const int8_t *q_in, double *seeds_out, int8_t *q_out, double *state, double *cov, double *chi2,
                   int32_t *ndof, uint32_t *status)
{
    int t;
    for (t = t0; t < t1; ++t) {
        int o = offsets[t], nh = offsets[t + 1] - offsets[t];
        double seed[6];
        int q, nd = 0, nu = 0;
        unsigned st;
        if (seeds) {
            memcpy(seed, &seeds[t * 6], sizeof seed);
            q = q_in[t];
        } else {
            double h1[3], h2[3], h3[3];
            int i1, i2;
            if (nh < 3) {
                status[t] = OR_ST_NO_INTERSECT;
                chi2[t] = 0.0;
                ndof[t] = 0;
                continue;
            }
            or_seed_hits(nh, hx + o, hy + o, &i1, &i2);
            h1[0] = hx[o];
            h1[1] = hy[o];
            h1[2] = hz[o];
            h2[0] = hx[o + i1];
            h2[1] = hy[o + i1];
            h2[2] = hz[o + i1];
            h3[0] = hx[o + i2];
            h3[1] = hy[o + i2];
            h3[2] = hz[o + i2];
            or_seed(h1, h2, h3, cfg->bz, seed, &q);
        }
        if (seeds_out) memcpy(&seeds_out[t * 6], seed, sizeof seed);
        if (q_out) q_out[t] = (int8_t)q;
        st = or_fit_one(cfg, surfs, nh, layer + o, hx + o, hy + o, hz + o, seed, q, NULL, &state[t * 6],
                        &cov[t * 36], &chi2[t], &nd, &nu, NULL);
        ndof[t] = nd;
        status[t] = st;
    }
}

/* ------------------------------------------------------------------ */
/* hit binning (Sec. 3.1: data structure for selecting hit candidates) */
/* ------------------------------------------------------------------ */

#define OR_NPHI 1024
#define OR_NZ 64

/* bin of one hit of a barrel layer with half length hz_len, in FP64:
 *   phi_bin = clamp(floor(((atan2(y,x) + pi) * 1024) / (2 pi)), 0, 1023)
 *   z_bin   = clamp(floor(((z + Lz) * 64) / (2 Lz)), 0, 63)
 *   key     = z_bin * 1024 + phi_bin */
int32_t or_bin_key(float x, float y, float z, double hz_len)
{
    double u = ((atan2((double)y, (double)x) + OR_PI) * 1024.0) / (2.0 * OR_PI);
    double v = (((double)z + hz_len) * 64.0) / (2.0 * hz_len);
    double fu = floor(u), fv = floor(v);
    int pb, zb;
    if (fu < 0.0) fu = 0.0;
    if (fu > OR_NPHI - 1) fu = OR_NPHI - 1;
    if (fv < 0.0) fv = 0.0;
    if (fv > OR_NZ - 1) fv = OR_NZ - 1;
    pb = (int)fu;
    zb = (int)fv;
    return zb * OR_NPHI + pb;
}

/* Stable counting sort of one layer's hits by key (ties in original order).
 * perm[i] = original index of the i-th hit in binned order;
 * offsets[k] .. offsets[k+1]-1 are the positions of key k (65537 entries). */
void or_bin_layer(int n, const float *x, const float *y, const float *z, double hz_len, int32_t *perm,
                  int32_t *offsets)
{
    int i, k;
    int32_t *key = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(OR_NPHI * OR_NZ) * sizeof(int32_t));
    for (k = 0; k <= OR_NPHI * OR_NZ; ++k) offsets[k] = 0;
    for (i = 0; i < n; ++i) {
        key[i] = or_bin_key(x[i], y[i], z[i], hz_len);
        offsets[key[i] + 1] += 1;
    }
    for (k = 0; k < OR_NPHI * OR_NZ; ++k) offsets[k + 1] += offsets[k];
    for (k = 0; k < OR_NPHI * OR_NZ; ++k) cur[k] = offsets[k];
    for (i = 0; i < n; ++i) perm[cur[key[i]]++] = i;
    free(key);
    free(cur);
}

/* ------------------------------------------------------------------ */
/* best-hit building (Sec. 2: project outwards, keep the most likely    */
/* continuation; here one candidate per seed, min chi2 per layer)       */
/* ------------------------------------------------------------------ */

typedef struct {
    double nsigma;   /* window half width in sigmas */
    double chi2_cut; /* accept best only if chi2 < cut */
    int32_t max_cand; /* candidates per step, in enumeration order */
    int32_t pad_;
} or_build_cfg;

/* One binned layer of one event: hits in original order, the binning of
 * or_bin_layer, and the surface index in the geometry. */
typedef struct {
    int32_t n;
    int32_t surf;
    const float *x, *y, *z;
    const int32_t *perm;
    const int32_t *offsets;
} or_layer;

/* Per (track, build layer) record of what the oracle saw, for the tests. */
typedef struct {
    double pred[6];    /* predicted state after propagation (before update) */
    double chi2_best;  /* smallest chi2 among candidates (or -1) */
    double chi2_second;/* second smallest (or -1) */
    int32_t phi_lo, phi_n; /* first phi bin (may be <0 or >1023 before wrap) and count */
    int32_t z_lo, z_hi;
    int32_t n_cand;
    int32_t capped;
    int32_t best;       /* chosen original hit index or -1 */
    int32_t status;
} or_step_rec;

/* Half widths of the candidate window of a build step around the predicted
 * state st with covariance P on layer surface sf (a barrel of radius R):
 *   phi: nsigma * sqrt(var(phi of the position) + (sig_rphi / R)^2), with the
 *        variance of the azimuth of (x, y) to first order,
 *        (y^2 P_xx + x^2 P_yy - 2 x y P_xy) / r^4;
 *   z:   nsigma * sqrt(P_zz + sig_3^2).
 * Measurement model 1 (hits within +-dr of the average radius): each widens by
 * what the track sweeps while it crosses dr radially, with a the angle between
 * the direction and the radial direction at the prediction:
 *   dphi += dr tan(a) / R,  dz += dr |cot(theta)| / cos(a)
 * (the whole layer when cos(a) <= 1e-3).  Reading of Sec. 3.1 / 4.1. */
void or_window(const double st[6], const double P[36], const or_surf *sf, double nsigma, int meas_model,
               double *dphi_out, double *dz_out)
{
    const double xp = st[0], yp = st[1], R = sf->pos, Lz = sf->half_or_rin;
    const double r2 = xp * xp + yp * yp;
    const double phip = atan2(yp, xp);
    const double sphi2 = (yp * yp * P[0 * 6 + 0] + xp * xp * P[1 * 6 + 1] - 2.0 * xp * yp * P[0 * 6 + 1]) / (r2 * r2);
    double dphi = nsigma * sqrt(sphi2 + (sf->sig_rphi / R) * (sf->sig_rphi / R));
    double dz = nsigma * sqrt(P[2 * 6 + 2] + sf->sig_3 * sf->sig_3);
    if (meas_model == 1 && sf->dr > 0.0) {
        const double ca = fabs(cos(st[4] - phip)), sa = fabs(sin(st[4] - phip));
        const double cot = cos(st[5]) / sin(st[5]);
        if (ca > 1e-3) {
            dphi += sf->dr * sa / (ca * R);
            dz += sf->dr * fabs(cot) / ca;
        } else {
            dphi = OR_PI;
            dz = 2.0 * Lz;
        }
    }
    *dphi_out = dphi;
    *dz_out = dz;
}

static int floor_clamp(double v, int lo, int hi)
{
    double f = floor(v);
    if (f < lo) return lo;
    if (f > hi) return hi;
    return (int)f;
}

/* One best-hit step (reading of Sec. 2 "most likely continuation", Sec. 3.1
 * binned hit selection) on layer ly, from the predicted state st and its 6x6
 * covariance P on the layer's surface sf (after propagation and scattering
 * noise): the window of or_window around the predicted position; its bins in
 * order -- z ascending, phi from the low edge with wrap, each bin's hits in
 * binned order -- at most max_cand candidates (capped beyond); the chi2 of
 * each (measurement model 0: r^T S^-1 r with S = P_pos + R at the hit azimuth;
 * model 1: carried on to the cylinder through the hit, 2-D there); the
 * smallest, ties to the lower original index.  The chi2 cut is not applied
 * here.  Fills rc (may be NULL).  Returns the best original index or -1, its
 * chi2 in *chi2_best. */
int or_besthit_step(const or_fit_cfg *fc, const or_build_cfg *bc, const or_surf *sf, const or_layer *ly,
                    const double st[6], const double P[36], int q, double *chi2_best, or_step_rec *rc)
{
    const double Lz = sf->half_or_rin;
    double phip, dphi, dz, bchi = 0.0, second = -1.0;
    int phi_lo, phi_hi, nphi, z_lo, z_hi, zb, k, ncand = 0, capped = 0, best = -1;
    int32_t cand[1024];
    /* window (under model 1 widened by the sweep over +-dr) */
    phip = atan2(st[1], st[0]);
    or_window(st, P, sf, bc->nsigma, fc->meas_model, &dphi, &dz);
    phi_lo = (int)floor(((phip - dphi + OR_PI) * 1024.0) / (2.0 * OR_PI));
    phi_hi = (int)floor(((phip + dphi + OR_PI) * 1024.0) / (2.0 * OR_PI));
    nphi = phi_hi - phi_lo + 1;
    if (nphi > OR_NPHI) nphi = OR_NPHI;
    z_lo = floor_clamp(((st[2] - dz + Lz) * 64.0) / (2.0 * Lz), 0, OR_NZ - 1);
    z_hi = floor_clamp(((st[2] + dz + Lz) * 64.0) / (2.0 * Lz), 0, OR_NZ - 1);
    /* enumerate candidates */
    for (zb = z_lo; zb <= z_hi && !capped; ++zb) {
        for (k = 0; k < nphi && !capped; ++k) {
            int pb = ((phi_lo + k) % OR_NPHI + OR_NPHI) % OR_NPHI;
            int key = zb * OR_NPHI + pb, j;
            for (j = ly->offsets[key]; j < ly->offsets[key + 1]; ++j) {
                if (ncand >= bc->max_cand) {
                    capped = 1;
                    break;
                }
                cand[ncand++] = ly->perm[j];
            }
        }
    }
    /* score */
    for (k = 0; k < ncand; ++k) {
        int h = cand[k];
        double hit[3] = {(double)ly->x[h], (double)ly->y[h], (double)ly->z[h]};
        double Rm[9], S[9], r[3], c2 = -1.0;
        int a, b;
        if (fc->meas_model == 1) {
            /* second step: from the layer's average cylinder to the hit's own */
            const or_surf hc = hit_cylinder(sf, hit);
            double s2[6], P2[36], J2[36];
            memcpy(P2, P, sizeof P2);
            if (or_propagate(st, q, fc->bz, &hc, s2, J2) || (or_transport(J2, P2), or_chi2_2d(s2, P2, hit, &hc, &c2)))
                c2 = -1.0;
        } else {
            or_meas_cov(sf, hit, Rm);
            for (a = 0; a < 3; ++a) {
                r[a] = hit[a] - st[a];
                for (b = 0; b < 3; ++b) S[a * 3 + b] = P[a * 6 + b] + Rm[a * 3 + b];
            }
            if (or_chi2(S, r, &c2)) c2 = -1.0;
        }
        if (c2 < 0.0) continue;
        if (best < 0 || c2 < bchi || (c2 == bchi && h < best)) {
            if (best >= 0) second = bchi;
            best = h;
            bchi = c2;
        } else if (second < 0.0 || c2 < second) {
            second = c2;
        }
    }
    if (rc) {
        memcpy(rc->pred, st, 6 * sizeof(double));
        rc->chi2_best = best >= 0 ? bchi : -1.0;
        rc->chi2_second = second;
        rc->phi_lo = phi_lo;
        rc->phi_n = nphi;
        rc->z_lo = z_lo;
        rc->z_hi = z_hi;
        rc->n_cand = ncand;
        rc->capped = capped;
        rc->status = 0;
    }
    *chi2_best = bchi;
    return best;
}

/* Build one track.  Seed from its three seed hits (layers 0..2 of the
 * layer list), KF fit over them, then for each later layer: propagate,
 * add scattering noise, open a window of +-nsigma in phi and z, score every
 * hit in the window's bins (z ascending, phi ascending with wrap, binned
 * order; at most max_cand), keep the smallest chi2 below the cut (ties: lower
 * original index) and update with it.  idx receives the chosen original hit
 * index per layer (-1: none).  Under measurement model 1 (Sec. 4.1, non-ideal
 * geometry) the propagation takes two steps: to the layer's average cylinder
 * (noise and window there), then from there to each candidate hit's own
 * cylinder, where its chi2 is taken and the update made (2-D, tangent plane). */
unsigned or_build_one(const or_fit_cfg *fc, const or_build_cfg *bc, const or_surf *surfs, int nlay,
                      const or_layer *lays, const float seed_hits[9], const int32_t seed_idx[3], int32_t *idx,
                      double st[6], double P[36], double *chi2_sum, int *ndof, or_step_rec *rec)
{
    double h1[3], h2[3], h3[3], seed[6];
    uint8_t lyr[3];
    int q, nu = 0, L, i;
    unsigned status;
    float sx[3], sy[3], sz[3];
    for (i = 0; i < 3; ++i) {
        sx[i] = seed_hits[i * 3 + 0];
        sy[i] = seed_hits[i * 3 + 1];
        sz[i] = seed_hits[i * 3 + 2];
        lyr[i] = (uint8_t)lays[i].surf;
    }
    h1[0] = sx[0]; h1[1] = sy[0]; h1[2] = sz[0];
    h2[0] = sx[1]; h2[1] = sy[1]; h2[2] = sz[1];
    h3[0] = sx[2]; h3[1] = sy[2]; h3[2] = sz[2];
    or_seed(h1, h2, h3, fc->bz, seed, &q);
    status = or_fit_one(fc, surfs, 3, lyr, sx, sy, sz, seed, q, NULL, st, P, chi2_sum, ndof, &nu, NULL);
    for (i = 0; i < 3; ++i) idx[i] = seed_idx[i];
    for (L = 3; L < nlay; ++L) idx[L] = -1;
    if (status & (OR_ST_NO_INTERSECT | OR_ST_CHOL_FAIL | OR_ST_NONFINITE)) return status;
    for (L = 3; L < nlay; ++L) {
        const or_layer *ly = &lays[L];
        const or_surf *sf = &surfs[ly->surf];
        double nx[6], J[36], bchi = 0.0;
        int best;
        or_step_rec local;
        or_step_rec *rc = rec ? &rec[L] : &local;
        int prc = or_propagate(st, q, fc->bz, sf, nx, J);
        if (prc) {
            status |= (unsigned)prc;
            rc->status = prc;
            break;
        }
        memcpy(st, nx, sizeof nx);
        or_transport(J, P);
        if (fc->ms_on) status |= (unsigned)or_ms_noise(st, fc->mass, sf, P);
        best = or_besthit_step(fc, bc, sf, ly, st, P, q, &bchi, rc);
        if (rc->capped) status |= OR_ST_CAND_CAPPED;
        if (best >= 0 && bchi < bc->chi2_cut) {
            double hit[3] = {(double)ly->x[best], (double)ly->y[best], (double)ly->z[best]};
            double Rm[9], c2;
            int urc;
            if (fc->meas_model == 1) {
                const or_surf hc = hit_cylinder(sf, hit);
                double s2[6], J2[36];
                urc = or_propagate(st, q, fc->bz, &hc, s2, J2);
                if (!urc) {
                    memcpy(st, s2, sizeof s2);
                    or_transport(J2, P);
                    urc = or_update2d(st, P, hit, &hc, &c2);
                }
            } else {
                or_meas_cov(sf, hit, Rm);
                urc = or_update(st, P, hit, Rm, &c2);
            }
            if (urc) {
                status |= OR_ST_CHOL_FAIL;
                break;
            }
            *chi2_sum += c2;
            nu += 1;
            idx[L] = best;
        }
        rc->best = idx[L];
    }
    *ndof = 2 * nu - 5;
    for (i = 0; i < 6; ++i)
        if (!isfinite(st[i])) status |= OR_ST_NONFINITE;
    return status;
}

/* Build tracks [t0, t1) of one event: seed_hits (n x 9: three hits x,y,z),
 * seed_idx (n x 3), idx out (n x nlay), state (n x 6), cov (n x 36), chi2,
 * ndof, status; rec (n x nlay) may be NULL. */
void or_build_tracks(const or_fit_cfg *fc, const or_build_cfg *bc, const or_surf *surfs, int nlay,
                     const or_layer *lays, int t0, int t1, const float *seed_hits, const int32_t *seed_idx,
                     int32_t *idx, double *state, double *cov, double *chi2, int32_t *ndof, uint32_t *status,
                     or_step_rec *rec)
{
    int t;
    for (t = t0; t < t1; ++t) {
        int nd = 0;
        status[t] = or_build_one(fc, bc, surfs, nlay, lays, &seed_hits[t * 9], &seed_idx[t * 3], &idx[t * nlay],
                                 &state[t * 6], &cov[t * 36], &chi2[t], &nd, rec ? &rec[t * nlay] : NULL);
        ndof[t] = nd;
    }
}

/* ------------------------------------------------------------------ */
/* combinatorial building (Sec. 2: building branches to explore several */
/* candidates per seed after finding compatible hits on a layer; Sec.   */
/* 4.3: a fixed number of candidate slots per seed, the best kept)      */
/* ------------------------------------------------------------------ */
/*
 * Reading.  Each seed keeps at most n_slots candidates, ranked.  On every
 * build layer each candidate is propagated and scattered as in best-hit
 * building, its window (the same one) is searched, and it has children:
 * one per window hit with chi2 below the cut (the candidate updated with
 * that hit), and one without a hit on this layer (a hole: the predicted
 * state).  A candidate that cannot reach the layer stops and is carried
 * unchanged.  All children of the seed are ranked -- more hits first, then
 * smaller total chi2, then the lower rank of the parent, then the lower hit
 * index (a hole after the hits of its parent) -- and the first n_slots are
 * kept, in that order.  After the last layer the first candidate is the
 * track.  With n_slots = 1 this is best-hit building.
 */

typedef struct {
    double nsigma;
    double chi2_cut;
    int32_t max_cand; /* window hits scored per candidate */
    int32_t n_slots;  /* candidates kept per seed */
} or_ckf_cfg;

/* How close one seed came to a different decision, for the tests: the
 * smallest relative chi2 gap between two children of equal hit count where the
 * order decided something (the last kept against the first dropped on every
 * layer, the first against the second on the last layer), the smallest
 * relative distance of a scored hit's chi2 to the cut, and the smallest
 * distance (in bins) of a window edge to a bin boundary. */
typedef struct {
    double rank_gap;
    double cut_gap;
    double edge_gap;
    int32_t capped;
    int32_t n_kept_last; /* candidates alive after the last layer */
} or_ckf_margin;

typedef struct {
    double st[6], P[36];
    double chi2;
    int32_t nh, nu, stopped;
    uint32_t status;
} or_cand;

typedef struct {
    double chi2; /* total chi2 of the child */
    int32_t nh;
    int32_t parent;
    int32_t hit;  /* original hit index, -1: hole or stopped */
    int32_t pad_;
    uint32_t status;
} or_child;

/* 1 when child a ranks before child b */
static int child_before(const or_child *a, const or_child *b)
{
    long long ha = a->hit < 0 ? 0x7fffffffLL : a->hit, hb = b->hit < 0 ? 0x7fffffffLL : b->hit;
    if (a->nh != b->nh) return a->nh > b->nh;
    if (a->chi2 != b->chi2) return a->chi2 < b->chi2;
    if (a->parent != b->parent) return a->parent < b->parent;
    return ha < hb;
}

static void rank_gap_update(or_ckf_margin *mg, const or_child *a, const or_child *b)
{
    double den, g;
    if (a->nh != b->nh) return;
    den = fabs(b->chi2) > 1e-300 ? fabs(b->chi2) : 1e-300;
    g = (b->chi2 - a->chi2) / den;
    if (g < mg->rank_gap) mg->rank_gap = g;
}

static double edge_dist(double u)
{
    double f = u - floor(u);
    return f < 1.0 - f ? f : 1.0 - f;
}

/* Combinatorial building of one seed.  Arguments as or_build_one; idx gets
 * the chosen hit per layer of the best candidate; margin may be NULL. */
unsigned or_ckf_one(const or_fit_cfg *fc, const or_ckf_cfg *cc, const or_surf *surfs, int nlay, const or_layer *lays,
                    const float seed_hits[9], const int32_t seed_idx[3], int32_t *idx, double st_out[6],
                    double P_out[36], double *chi2_out, int *ndof, or_ckf_margin *margin)
{
    const int C = cc->n_slots;
    double h1[3], h2[3], h3[3], seed[6];
    uint8_t lyr[3];
    float sx[3], sy[3], sz[3];
    int q, nu = 0, L, i, nc = 1;
    unsigned status;
    or_cand *cands, *next, *pred;
    or_child *kids;
    int32_t *bp_parent, *bp_hit;
    int max_kids;
    or_ckf_margin mg = {1e300, 1e300, 1e300, 0, 0};
    for (i = 0; i < 3; ++i) {
        sx[i] = seed_hits[i * 3 + 0];
        sy[i] = seed_hits[i * 3 + 1];
        sz[i] = seed_hits[i * 3 + 2];
        lyr[i] = (uint8_t)lays[i].surf;
    }
    h1[0] = sx[0]; h1[1] = sy[0]; h1[2] = sz[0];
    h2[0] = sx[1]; h2[1] = sy[1]; h2[2] = sz[1];
    h3[0] = sx[2]; h3[1] = sy[2]; h3[2] = sz[2];
    or_seed(h1, h2, h3, fc->bz, seed, &q);
    for (i = 0; i < 3; ++i) idx[i] = seed_idx[i];
    for (L = 3; L < nlay; ++L) idx[L] = -1;
    cands = (or_cand *)calloc((size_t)C, sizeof(or_cand));
    next = (or_cand *)calloc((size_t)C, sizeof(or_cand));
    pred = (or_cand *)calloc((size_t)C, sizeof(or_cand));
    max_kids = C * (cc->max_cand + 1);
    kids = (or_child *)calloc((size_t)max_kids, sizeof(or_child));
    bp_parent = (int32_t *)calloc((size_t)nlay * C, sizeof(int32_t));
    bp_hit = (int32_t *)calloc((size_t)nlay * C, sizeof(int32_t));
    status = or_fit_one(fc, surfs, 3, lyr, sx, sy, sz, seed, q, NULL, cands[0].st, cands[0].P, &cands[0].chi2, ndof,
                        &nu, NULL);
    cands[0].nh = 3;
    cands[0].nu = nu;
    cands[0].status = status;
    if (status & (OR_ST_NO_INTERSECT | OR_ST_CHOL_FAIL | OR_ST_NONFINITE)) {
        memcpy(st_out, cands[0].st, 6 * sizeof(double));
        memcpy(P_out, cands[0].P, 36 * sizeof(double));
        *chi2_out = cands[0].chi2;
        goto done;
    }
    for (L = 3; L < nlay; ++L) {
        const or_layer *ly = &lays[L];
        const or_surf *sf = &surfs[ly->surf];
        const double Lz = sf->half_or_rin;
        int nk = 0, r, k, keep;
        for (r = 0; r < nc; ++r) {
            or_cand *c = &cands[r];
            or_cand *pr = &pred[r];
            double nx[6], J[36], phip, dphi, dz, ulo, uhi, vlo, vhi;
            int32_t cand[1024];
            int phi_lo, phi_hi, nphi, z_lo, z_hi, zb, ncand = 0, capped = 0, prc;
            unsigned step = 0;
            *pr = *c;
            if (c->stopped) { /* carried unchanged */
                or_child *kd = &kids[nk++];
                kd->chi2 = c->chi2;
                kd->nh = c->nh;
                kd->parent = r;
                kd->hit = -1;
                kd->status = 0;
                continue;
            }
            prc = or_propagate(c->st, q, fc->bz, sf, nx, J);
            if (prc) {
                or_child *kd = &kids[nk++];
                pr->stopped = 1;
                kd->chi2 = c->chi2;
                kd->nh = c->nh;
                kd->parent = r;
                kd->hit = -1;
                kd->status = (unsigned)prc;
                continue;
            }
            memcpy(pr->st, nx, sizeof nx);
            or_transport(J, pr->P);
            if (fc->ms_on) step |= (unsigned)or_ms_noise(pr->st, fc->mass, sf, pr->P);
            /* window, as in best-hit building (measurement model 0) */
            phip = atan2(pr->st[1], pr->st[0]);
            or_window(pr->st, pr->P, sf, cc->nsigma, 0, &dphi, &dz);
            ulo = ((phip - dphi + OR_PI) * 1024.0) / (2.0 * OR_PI);
            uhi = ((phip + dphi + OR_PI) * 1024.0) / (2.0 * OR_PI);
            vlo = ((pr->st[2] - dz + Lz) * 64.0) / (2.0 * Lz);
            vhi = ((pr->st[2] + dz + Lz) * 64.0) / (2.0 * Lz);
            phi_lo = (int)floor(ulo);
            phi_hi = (int)floor(uhi);
            nphi = phi_hi - phi_lo + 1;
            if (nphi > OR_NPHI) nphi = OR_NPHI;
            z_lo = floor_clamp(vlo, 0, OR_NZ - 1);
            z_hi = floor_clamp(vhi, 0, OR_NZ - 1);
            if (edge_dist(ulo) < mg.edge_gap) mg.edge_gap = edge_dist(ulo);
            if (edge_dist(uhi) < mg.edge_gap) mg.edge_gap = edge_dist(uhi);
            if (vlo > 0.0 && vlo < OR_NZ && edge_dist(vlo) < mg.edge_gap) mg.edge_gap = edge_dist(vlo);
            if (vhi > 0.0 && vhi < OR_NZ && edge_dist(vhi) < mg.edge_gap) mg.edge_gap = edge_dist(vhi);
            for (zb = z_lo; zb <= z_hi && !capped; ++zb) {
                for (k = 0; k < nphi && !capped; ++k) {
                    int pb = ((phi_lo + k) % OR_NPHI + OR_NPHI) % OR_NPHI;
                    int key = zb * OR_NPHI + pb, j;
                    for (j = ly->offsets[key]; j < ly->offsets[key + 1]; ++j) {
                        if (ncand >= cc->max_cand) {
                            capped = 1;
                            break;
                        }
                        cand[ncand++] = ly->perm[j];
                    }
                }
            }
            if (capped) {
                step |= OR_ST_CAND_CAPPED;
                mg.capped = 1;
            }
            pr->status = c->status | step;
            for (k = 0; k < ncand; ++k) {
                int h = cand[k], a, b;
                double hit[3] = {(double)ly->x[h], (double)ly->y[h], (double)ly->z[h]};
                double Rm[9], S[9], rr[3], c2 = -1.0;
                or_meas_cov(sf, hit, Rm);
                for (a = 0; a < 3; ++a) {
                    rr[a] = hit[a] - pr->st[a];
                    for (b = 0; b < 3; ++b) S[a * 3 + b] = pr->P[a * 6 + b] + Rm[a * 3 + b];
                }
                if (or_chi2(S, rr, &c2)) continue;
                if (fabs(c2 - cc->chi2_cut) / cc->chi2_cut < mg.cut_gap) mg.cut_gap = fabs(c2 - cc->chi2_cut) / cc->chi2_cut;
                if (c2 < cc->chi2_cut) {
                    or_child *kd = &kids[nk++];
                    kd->chi2 = c->chi2 + c2;
                    kd->nh = c->nh + 1;
                    kd->parent = r;
                    kd->hit = h;
                    kd->status = step;
                }
            }
            {
                or_child *kd = &kids[nk++];
                kd->chi2 = c->chi2;
                kd->nh = c->nh;
                kd->parent = r;
                kd->hit = -1;
                kd->status = step;
            }
        }
        /* rank all children (insertion sort: short lists) */
        for (k = 1; k < nk; ++k) {
            or_child t = kids[k];
            int j = k - 1;
            while (j >= 0 && child_before(&t, &kids[j])) {
                kids[j + 1] = kids[j];
                --j;
            }
            kids[j + 1] = t;
        }
        keep = nk < C ? nk : C;
        /* decisions that matter: who is kept (the last kept against the first
         * dropped) and, on the last layer, which candidate is the track */
        if (nk > keep) rank_gap_update(&mg, &kids[keep - 1], &kids[keep]);
        if (L == nlay - 1 && keep > 1) rank_gap_update(&mg, &kids[0], &kids[1]);
        /* the kept children become the candidates */
        for (k = 0; k < keep; ++k) {
            const or_child *kd = &kids[k];
            const or_cand *pr = &pred[kd->parent];
            or_cand *nw = &next[k];
            *nw = *pr;
            nw->status = pr->status | kd->status;
            if (kd->status & OR_ST_NO_INTERSECT) nw->stopped = 1;
            if (kd->hit >= 0) {
                double hit[3] = {(double)ly->x[kd->hit], (double)ly->y[kd->hit], (double)ly->z[kd->hit]};
                double Rm[9], c2 = 0.0;
                or_meas_cov(sf, hit, Rm);
                if (or_update(nw->st, nw->P, hit, Rm, &c2)) {
                    /* cannot happen: S was factored when the hit was scored */
                    nw->status |= OR_ST_CHOL_FAIL;
                }
                nw->chi2 = kd->chi2;
                nw->nh = kd->nh;
                nw->nu += 1;
            }
            bp_parent[L * C + k] = kd->parent;
            bp_hit[L * C + k] = kd->hit;
        }
        nc = keep;
        memcpy(cands, next, (size_t)keep * sizeof(or_cand));
    }
    /* the first candidate is the track; its hits by walking the back pointers */
    {
        int s = 0;
        for (L = nlay - 1; L >= 3; --L) {
            idx[L] = bp_hit[L * C + s];
            s = bp_parent[L * C + s];
        }
    }
    memcpy(st_out, cands[0].st, 6 * sizeof(double));
    memcpy(P_out, cands[0].P, 36 * sizeof(double));
    *chi2_out = cands[0].chi2;
    status = cands[0].status;
    nu = cands[0].nu;
    *ndof = 2 * nu - 5;
    mg.n_kept_last = nc;
done:
    for (i = 0; i < 6; ++i)
        if (!isfinite(st_out[i])) status |= OR_ST_NONFINITE;
    if (margin) *margin = mg;
    free(cands);
    free(next);
    free(pred);
    free(kids);
    free(bp_parent);
    free(bp_hit);
    return status;
}

/* Combinatorial building of tracks [t0, t1) of one event; arrays as
 * or_build_tracks, margin (n) may be NULL. */
void or_ckf_tracks(const or_fit_cfg *fc, const or_ckf_cfg *cc, const or_surf *surfs, int nlay, const or_layer *lays,
                   int t0, int t1, const float *seed_hits, const int32_t *seed_idx, int32_t *idx, double *state,
                   double *cov, double *chi2, int32_t *ndof, uint32_t *status, or_ckf_margin *margin)
{
    int t;
    for (t = t0; t < t1; ++t) {
        int nd = 0;
        status[t] = or_ckf_one(fc, cc, surfs, nlay, lays, &seed_hits[t * 9], &seed_idx[t * 3], &idx[t * nlay],
                               &state[t * 6], &cov[t * 36], &chi2[t], &nd, margin ? &margin[t] : NULL);
        ndof[t] = nd;
    }
}

/* ------------------------------------------------------------------ */
/* outward-inward refit (the final fit of Sec. 2, run a second time     */
/* from the last hit back to the first: the estimate at the first hit   */
/* then uses every hit)                                                 */
/* ------------------------------------------------------------------ */
/*
 * Reading.  The track is run backwards by reversing its direction of motion:
 * (x, y, z, 1/pT, phi, theta), q  ->  (x, y, z, 1/pT, phi + pi, pi - theta), -q,
 * the same helix traversed the other way.  The hits the forward fit used
 * (the first (ndof + 5) / 2 of the track), in reverse order, are fitted like
 * any track, starting at the last used hit from the forward fit's state there
 * with the forward covariance multiplied by cov_scale (reversed like the
 * state), and the result at the first hit is turned back: phi - pi,
 * pi - theta, q; in the covariance the theta row and column change sign.
 * Starting from the inflated forward covariance rather than from seed_cov * I
 * keeps the backward filter on the fitted trajectory from its first step: a
 * track that ends near its apex meets its near-tangent crossings first, and
 * there a covariance of 1e4 turns the rounding of the seed into differences of
 * up to 0.3 sigma (measured: moving the seed phi by 1e-14 rad).  The forward
 * information counts once more with weight 1 / cov_scale.
 */
static void or_reverse_state(double st[6])
{
    st[4] = wrap_phi(st[4] + OR_PI);
    st[5] = OR_PI - st[5];
}

static void or_reverse_cov(double P[36])
{
    int i;
    for (i = 0; i < 6; ++i) {
        if (i == 5) continue;
        P[i * 6 + 5] = -P[i * 6 + 5];
        P[5 * 6 + i] = -P[5 * 6 + i];
    }
}

/* fwd_state, fwd_ndof: the forward fit's state at its last used hit and its
 * ndof; outputs at the first hit, in the forward direction */
unsigned or_refit_inward(const or_fit_cfg *cfg, const or_surf *surfs, int nh_all, const uint8_t *layer,
                         const float *hx, const float *hy, const float *hz, const double fwd_state[6],
                         const double fwd_cov[36], double cov_scale, int q, int fwd_ndof, double st[6], double P[36],
                         double *chi2_sum, int *ndof)
{
    const int nh = (fwd_ndof + 5) / 2 < 0 ? 0 : ((fwd_ndof + 5) / 2 > nh_all ? nh_all : (fwd_ndof + 5) / 2);
    uint8_t *rl = (uint8_t *)malloc((size_t)(nh > 0 ? nh : 1));
    float *rx = (float *)malloc(sizeof(float) * (size_t)(nh > 0 ? nh : 1));
    float *ry = (float *)malloc(sizeof(float) * (size_t)(nh > 0 ? nh : 1));
    float *rz = (float *)malloc(sizeof(float) * (size_t)(nh > 0 ? nh : 1));
    double seed[6], P0[36];
    int k, nu = 0;
    unsigned status;
    for (k = 0; k < nh; ++k) {
        rl[k] = layer[nh - 1 - k];
        rx[k] = hx[nh - 1 - k];
        ry[k] = hy[nh - 1 - k];
        rz[k] = hz[nh - 1 - k];
    }
    memcpy(seed, fwd_state, sizeof seed);
    or_reverse_state(seed);
    for (k = 0; k < 36; ++k) P0[k] = cov_scale * fwd_cov[k];
    or_reverse_cov(P0);
    status = or_fit_from(cfg, surfs, nh, rl, rx, ry, rz, seed, P0, -q, NULL, st, P, chi2_sum, ndof, &nu, NULL);
    or_reverse_state(st);
    or_reverse_cov(P);
    free(rl);
    free(rx);
    free(ry);
    free(rz);
    return status;
}

void or_refit_tracks(const or_fit_cfg *cfg, const or_surf *surfs, int t0, int t1, const int32_t *offsets,
                     const uint8_t *layer, const float *hx, const float *hy, const float *hz, const double *fwd,
                     const double *fwd_cov, double cov_scale, const int8_t *q, const int32_t *fwd_ndof,
                     double *state, double *cov, double *chi2, int32_t *ndof, uint32_t *status)
{
    int t;
    for (t = t0; t < t1; ++t) {
        int o = offsets[t], nd = 0;
        status[t] = or_refit_inward(cfg, surfs, offsets[t + 1] - o, layer + o, hx + o, hy + o, hz + o, &fwd[t * 6],
                                    &fwd_cov[t * 36], cov_scale, q[t], fwd_ndof[t], &state[t * 6], &cov[t * 36],
                                    &chi2[t], &nd);
        ndof[t] = nd;
    }
}
