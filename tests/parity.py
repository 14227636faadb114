"""Comparison helpers for the GPU-vs-oracle parity tests.

Fitted states are compared in the local frame of the surface where the fit
ended, because the global covariance is singular along the surface normal:
barrel -> (r phi, z), disk -> (r phi, r); plus q/pT, phi, theta.  Each
difference is divided by the oracle's own sigma of that parameter.
"""
import numpy as np

# tolerances stated for this path: parameters within 1e-3 of their own sigma,
# chi2 within 1e-3 relative
TOL_PARAM_SIGMA = 1e-3
TOL_CHI2_REL = 1e-3
# covariance: entries of the local 5x5 covariance, normalised by sqrt(C_ii C_jj);
# the same 1e-3 bound (a reading: the path states no covariance tolerance)
TOL_COV_NORM = 1e-3


def last_surface(tk, ndof):
    """Surface index of the last hit each fit used (ndof = 2 used - 5)."""
    off = tk["offsets"]
    used = (np.asarray(ndof) + 5) // 2
    idx = off[:-1] + np.maximum(used, 1) - 1
    return tk["layer"][idx].astype(int)


def local_frame(state_ref, kind):
    """(n,5,6) projection onto (u1, u2, q/pT-like, phi, theta) at the reference point."""
    n = len(state_ref)
    a = np.arctan2(state_ref[:, 1], state_ref[:, 0])
    T = np.zeros((n, 5, 6))
    T[:, 0, 0] = -np.sin(a)
    T[:, 0, 1] = np.cos(a)
    barrel = kind == 0
    T[barrel, 1, 2] = 1.0
    T[~barrel, 1, 0] = np.cos(a[~barrel])
    T[~barrel, 1, 1] = np.sin(a[~barrel])
    T[:, 2, 3] = 1.0
    T[:, 3, 4] = 1.0
    T[:, 4, 5] = 1.0
    return T


def compare_fits(gpu, orc, kinds, mask=None):
    """Per-track max |dp|/sigma over the 5 local parameters, chi2 relative error and the
    normalised local-covariance difference.  q/pT is compared as the signed curvature
    parameter q * (1/pT), since a seed of the wrong charge sign legitimately ends with
    the opposite signs of both."""
    n = len(orc["state"])
    if mask is None:
        mask = np.ones(n, bool)
    so, sg = orc["state"][mask], gpu["state"][mask]
    Co, Cg = orc["cov"][mask], gpu["cov"][mask]
    T = local_frame(so, kinds[mask])
    d = sg - so
    d[:, 4] = (d[:, 4] + np.pi) % (2 * np.pi) - np.pi
    d[:, 3] = gpu["q"][mask] * sg[:, 3] - orc["q"][mask] * so[:, 3]
    # the sign of 1/pT follows q: express both covariances in terms of q/pT
    sgn_o = orc["q"][mask].astype(float)
    sgn_g = gpu["q"][mask].astype(float)
    Fo = np.ones((len(so), 6))
    Fo[:, 3] = sgn_o
    Fg = np.ones((len(so), 6))
    Fg[:, 3] = sgn_g
    Co = Co * Fo[:, :, None] * Fo[:, None, :]
    Cg = Cg * Fg[:, :, None] * Fg[:, None, :]
    dl = np.einsum("nij,nj->ni", T, d)
    C5o = np.einsum("nai,nij,nbj->nab", T, Co, T)
    C5g = np.einsum("nai,nij,nbj->nab", T, Cg, T)
    sig = np.sqrt(np.maximum(np.diagonal(C5o, axis1=1, axis2=2), 1e-300))
    pull = np.abs(dl) / sig
    norm = sig[:, :, None] * sig[:, None, :]
    dcov = np.abs(C5g - C5o) / norm
    chi2o, chi2g = orc["chi2"][mask], gpu["chi2"][mask]
    chi2rel = np.abs(chi2g - chi2o) / np.maximum(np.abs(chi2o), 1e-300)
    return dict(pull=pull, max_pull=pull.max(axis=1), chi2rel=chi2rel, dcov=dcov.reshape(len(so), -1).max(axis=1))


def summary(res):
    return (f"max|dp|/sigma={res['max_pull'].max():.3e} (p99 {np.percentile(res['max_pull'], 99):.2e}) "
            f"max dchi2/chi2={res['chi2rel'].max():.3e} max dcov={res['dcov'].max():.3e}")


def oracle_self_noise(oracle_mod, geom, tk, orc, kinds, eps=1e-14, threads=4):
    """Per-track numerical resolution of the FP64 oracle itself: the largest max |dp|/sigma
    between the oracle's fit and the same fit from a seed moved by a rounding-sized step,
    over eight directions (phi and theta by +-eps rad, 1/pT and z by +-eps relative).  Under the
    1e4 seed covariance the covariance-form update amplifies rounding by up to ~1e9 in
    the first updates; on most tracks the result moves by ~1e-7 sigma, on rare steep
    barrel+disk tracks by up to ~5e-3 sigma, and one direction alone can miss a track's
    sensitivity by an order of magnitude.  No implementation can be compared more finely
    than this."""
    ok = (orc["status"] & 7) == 0
    noise = np.zeros(len(ok))
    for comp, relative in ((4, False), (5, False), (3, True), (2, True)):
        for sgn in (1.0, -1.0):
            s = orc["seed"].copy()
            s[:, comp] += sgn * eps * (np.abs(s[:, comp]) if relative else 1.0)
            o2 = oracle_mod.fit(geom, tk, seeds=s, q=orc["q"], threads=threads)
            res = compare_fits(o2, orc, kinds, ok)
            noise[ok] = np.maximum(noise[ok], res["max_pull"])
    return noise
