"""FP64 CPU oracle for the batched Kalman-filter track fit, best-hit and combinatorial build.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  The
arithmetic lives in ``kf_oracle.c`` (plain double precision, one track at a
time, dense 6x6 matrices); this module compiles it with gcc and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library.

Parity: every routine is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (closed forms, finite differences, global
least squares, brute force, statistics); no routine is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_NO_INTERSECT = 1
ST_CHOL_FAIL = 2
ST_NONFINITE = 4
ST_CAND_CAPPED = 8
ST_GRAZING = 16
ST_THETA_RANGE = 32


def build_lib(force: bool = False) -> str:
    """Compile kf_oracle.c into oracle/_build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Surf(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("pos", C.c_double),
                ("half_or_rin", C.c_double), ("r_out", C.c_double), ("x_x0", C.c_double),
                ("sig_n", C.c_double), ("sig_rphi", C.c_double), ("sig_3", C.c_double), ("dr", C.c_double)]


class FitCfg(C.Structure):
    _fields_ = [("bz", C.c_double), ("mass", C.c_double), ("seed_cov", C.c_double),
                ("ms_on", C.c_int32), ("meas_model", C.c_int32)]


class BuildCfg(C.Structure):
    _fields_ = [("nsigma", C.c_double), ("chi2_cut", C.c_double), ("max_cand", C.c_int32),
                ("pad_", C.c_int32)]


class Layer(C.Structure):
    _fields_ = [("n", C.c_int32), ("surf", C.c_int32),
                ("x", C.POINTER(C.c_float)), ("y", C.POINTER(C.c_float)), ("z", C.POINTER(C.c_float)),
                ("perm", C.POINTER(C.c_int32)), ("offsets", C.POINTER(C.c_int32))]


class StepRec(C.Structure):
    _fields_ = [("pred", C.c_double * 6), ("chi2_best", C.c_double), ("chi2_second", C.c_double),
                ("phi_lo", C.c_int32), ("phi_n", C.c_int32), ("z_lo", C.c_int32), ("z_hi", C.c_int32),
                ("n_cand", C.c_int32), ("capped", C.c_int32), ("best", C.c_int32), ("status", C.c_int32)]


class CkfCfg(C.Structure):
    _fields_ = [("nsigma", C.c_double), ("chi2_cut", C.c_double), ("max_cand", C.c_int32), ("n_slots", C.c_int32)]


CKF_MARGIN_DTYPE = np.dtype([("rank_gap", "<f8"), ("cut_gap", "<f8"), ("edge_gap", "<f8"), ("capped", "<i4"),
                             ("n_kept_last", "<i4")])

STEP_DTYPE = np.dtype([("pred", "<f8", (6,)), ("chi2_best", "<f8"), ("chi2_second", "<f8"),
                       ("phi_lo", "<i4"), ("phi_n", "<i4"), ("z_lo", "<i4"), ("z_hi", "<i4"),
                       ("n_cand", "<i4"), ("capped", "<i4"), ("best", "<i4"), ("status", "<i4")])
assert STEP_DTYPE.itemsize == C.sizeof(StepRec)

_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I32 = C.POINTER(C.c_int32)
_I8 = C.POINTER(C.c_int8)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib()
            L = C.CDLL(path)
            L.or_curvature.restype = C.c_double
            L.or_curvature.argtypes = [_D, C.c_int, C.c_double]
            L.or_helix_at.restype = None
            L.or_helix_at.argtypes = [_D, C.c_double, C.c_double, _D]
            L.or_path_to_barrel.restype = C.c_int
            L.or_path_to_barrel.argtypes = [_D, C.c_double, C.c_double, _D]
            L.or_path_to_disk.restype = C.c_int
            L.or_path_to_disk.argtypes = [_D, C.c_double, _D]
            L.or_propagate.restype = C.c_int
            L.or_propagate.argtypes = [_D, C.c_int, C.c_double, C.POINTER(Surf), _D, _D]
            L.or_highland.restype = C.c_double
            L.or_highland.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_cos_incidence.restype = C.c_double
            L.or_cos_incidence.argtypes = [_D, C.POINTER(Surf)]
            L.or_ms_noise.restype = C.c_int
            L.or_ms_noise.argtypes = [_D, C.c_double, C.POINTER(Surf), _D]
            L.or_meas_cov.restype = None
            L.or_meas_cov.argtypes = [C.POINTER(Surf), _D, _D]
            L.or_chi2.restype = C.c_int
            L.or_chi2.argtypes = [_D, _D, _D]
            L.or_update.restype = C.c_int
            L.or_update.argtypes = [_D, _D, _D, _D, _D]
            L.or_transport.restype = None
            L.or_transport.argtypes = [_D, _D]
            L.or_seed.restype = None
            L.or_seed.argtypes = [_D, _D, _D, C.c_double, _D, C.POINTER(C.c_int)]
            L.or_seed_hits.restype = None
            L.or_seed_hits.argtypes = [C.c_int, _F, _F, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.or_fit_one.restype = C.c_uint
            L.or_fit_one.argtypes = [C.POINTER(FitCfg), C.POINTER(Surf), C.c_int, _U8, _F, _F, _F, _D, C.c_int,
                                     _D, _D, _D, _D, C.POINTER(C.c_int), C.POINTER(C.c_int), _D]
            L.or_fit_tracks.restype = None
            L.or_fit_tracks.argtypes = [C.POINTER(FitCfg), C.POINTER(Surf), C.c_int, C.c_int, _I32, _U8, _F, _F,
                                        _F, _D, _I8, _D, _I8, _D, _D, _D, _I32, _U32]
            L.or_bin_key.restype = C.c_int32
            L.or_bin_key.argtypes = [C.c_float, C.c_float, C.c_float, C.c_double]
            L.or_bin_layer.restype = None
            L.or_bin_layer.argtypes = [C.c_int, _F, _F, _F, C.c_double, _I32, _I32]
            L.or_build_tracks.restype = None
            L.or_build_tracks.argtypes = [C.POINTER(FitCfg), C.POINTER(BuildCfg), C.POINTER(Surf), C.c_int,
                                          C.POINTER(Layer), C.c_int, C.c_int, _F, _I32, _I32, _D, _D, _D, _I32,
                                          _U32, C.c_void_p]
            L.or_ckf_tracks.restype = None
            L.or_ckf_tracks.argtypes = [C.POINTER(FitCfg), C.POINTER(CkfCfg), C.POINTER(Surf), C.c_int,
                                        C.POINTER(Layer), C.c_int, C.c_int, _F, _I32, _I32, _D, _D, _D, _I32,
                                        _U32, C.c_void_p]
            L.or_besthit_step.restype = C.c_int
            L.or_besthit_step.argtypes = [C.POINTER(FitCfg), C.POINTER(BuildCfg), C.POINTER(Surf), C.POINTER(Layer),
                                          _D, _D, C.c_int, _D, C.POINTER(StepRec)]
            L.or_window.restype = None
            L.or_window.argtypes = [_D, _D, C.POINTER(Surf), C.c_double, C.c_int, _D, _D]
            L.or_update2d.restype = C.c_int
            L.or_update2d.argtypes = [_D, _D, _D, C.POINTER(Surf), _D]
            L.or_refit_tracks.restype = None
            L.or_refit_tracks.argtypes = [C.POINTER(FitCfg), C.POINTER(Surf), C.c_int, C.c_int, _I32, C.c_void_p,
                                          _F, _F, _F, _D, _D, C.c_double, C.POINTER(C.c_int8), _I32, _D, _D, _D,
                                          _I32, _U32]
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def surfaces(geom) -> "C.Array":
    """ctypes array of Surf from a geometry dict (see the synth module)."""
    arr = (Surf * len(geom["surfaces"]))()
    for i, s in enumerate(geom["surfaces"]):
        arr[i].kind = int(s["kind"])
        arr[i].pos = float(s["pos"])
        arr[i].half_or_rin = float(s["half_or_rin"])
        arr[i].r_out = float(s.get("r_out", 0.0))
        arr[i].x_x0 = float(s["x_x0"])
        arr[i].sig_n = float(s["sig_n"])
        arr[i].sig_rphi = float(s["sig_rphi"])
        arr[i].sig_3 = float(s["sig_3"])
        arr[i].dr = float(s.get("dr", 0.0))
    return arr


def fit_cfg(geom, seed_cov=1e4, ms_on=True, meas_model=0) -> FitCfg:
    return FitCfg(bz=float(geom["bz"]), mass=float(geom["mass"]), seed_cov=float(seed_cov), ms_on=int(bool(ms_on)),
                  meas_model=int(meas_model))


# ---------------------------------------------------------------- single-step helpers (pins)

def curvature(st, q, bz):
    st = np.ascontiguousarray(st, dtype=np.float64)
    return lib().or_curvature(_p(st, C.c_double), int(q), float(bz))


def helix_at(st, c, s):
    st = np.ascontiguousarray(st, dtype=np.float64)
    out = np.zeros(6)
    lib().or_helix_at(_p(st, C.c_double), float(c), float(s), _p(out, C.c_double))
    return out


def path_to_barrel(st, c, R):
    st = np.ascontiguousarray(st, dtype=np.float64)
    s = C.c_double(0.0)
    rc = lib().or_path_to_barrel(_p(st, C.c_double), float(c), float(R), C.byref(s))
    return rc, s.value


def propagate(st, q, bz, surf, want_jac=True):
    st = np.ascontiguousarray(st, dtype=np.float64)
    out = np.zeros(6)
    J = np.zeros(36)
    sarr = surfaces({"surfaces": [surf]})
    rc = lib().or_propagate(_p(st, C.c_double), int(q), float(bz), sarr, _p(out, C.c_double),
                            _p(J, C.c_double) if want_jac else None)
    return rc, out, J.reshape(6, 6)


def window(st, P, surf, nsigma=3.0, meas_model=0):
    """Half widths (dphi, dz) of the build window around state st with covariance P (6x6)."""
    st = np.ascontiguousarray(st, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    dphi, dz = C.c_double(0.0), C.c_double(0.0)
    lib().or_window(_p(st, C.c_double), _p(P, C.c_double), surfaces({"surfaces": [surf]}), float(nsigma),
                    int(meas_model), C.byref(dphi), C.byref(dz))
    return dphi.value, dz.value


def highland(p, mass, t):
    return lib().or_highland(float(p), float(mass), float(t))


def ms_noise(st, mass, surf, P):
    st = np.ascontiguousarray(st, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64).copy()
    rc = lib().or_ms_noise(_p(st, C.c_double), float(mass), surfaces({"surfaces": [surf]}), _p(P, C.c_double))
    return rc, P


def meas_cov(surf, hit):
    hit = np.ascontiguousarray(hit, dtype=np.float64)
    R = np.zeros(9)
    lib().or_meas_cov(surfaces({"surfaces": [surf]}), _p(hit, C.c_double), _p(R, C.c_double))
    return R.reshape(3, 3)


def update(st, P, hit, R):
    st = np.ascontiguousarray(st, dtype=np.float64).copy()
    P = np.ascontiguousarray(P, dtype=np.float64).copy()
    hit = np.ascontiguousarray(hit, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    chi2 = C.c_double(0.0)
    rc = lib().or_update(_p(st, C.c_double), _p(P, C.c_double), _p(hit, C.c_double), _p(R, C.c_double),
                         C.byref(chi2))
    return rc, st, P, chi2.value


def update2d(st, P, hit, surf):
    """Measurement-model-1 update (2-D, tangent plane at the hit azimuth)."""
    st = np.ascontiguousarray(st, dtype=np.float64).copy()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(36).copy()
    hit = np.ascontiguousarray(hit, dtype=np.float64)
    chi2 = np.zeros(1)
    sarr = surfaces({"surfaces": [surf]})
    rc = lib().or_update2d(_p(st, C.c_double), _p(P, C.c_double), _p(hit, C.c_double), sarr, _p(chi2, C.c_double))
    return rc, st, P.reshape(6, 6), float(chi2[0])


def transport(J, P):
    J = np.ascontiguousarray(J, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64).copy()
    lib().or_transport(_p(J, C.c_double), _p(P, C.c_double))
    return P


def seed(h1, h2, h3, bz):
    h1, h2, h3 = (np.ascontiguousarray(h, dtype=np.float64) for h in (h1, h2, h3))
    st = np.zeros(6)
    q = C.c_int(0)
    lib().or_seed(_p(h1, C.c_double), _p(h2, C.c_double), _p(h3, C.c_double), float(bz), _p(st, C.c_double),
                  C.byref(q))
    return st, q.value


def seed_hits(hx, hy):
    hx, hy = (np.ascontiguousarray(a, dtype=np.float32) for a in (hx, hy))
    a, b = C.c_int(0), C.c_int(0)
    lib().or_seed_hits(len(hx), _p(hx, C.c_float), _p(hy, C.c_float), C.byref(a), C.byref(b))
    return 0, a.value, b.value


def fit_one(geom, layer, hx, hy, hz, seed_state, q, seed_cov=1e4, ms_on=True, lin_ref=None):
    cfg = fit_cfg(geom, seed_cov, ms_on)
    sarr = surfaces(geom)
    layer = np.ascontiguousarray(layer, dtype=np.uint8)
    hx, hy, hz = (np.ascontiguousarray(a, dtype=np.float32) for a in (hx, hy, hz))
    seed_state = np.ascontiguousarray(seed_state, dtype=np.float64)
    st = np.zeros(6)
    P = np.zeros(36)
    chi2 = C.c_double(0.0)
    ndof = C.c_int(0)
    nu = C.c_int(0)
    each = np.zeros(len(hx))
    ref = None
    if lin_ref is not None:
        ref = np.ascontiguousarray(lin_ref, dtype=np.float64)
    status = lib().or_fit_one(C.byref(cfg), sarr, len(hx), _p(layer, C.c_uint8), _p(hx, C.c_float),
                              _p(hy, C.c_float), _p(hz, C.c_float), _p(seed_state, C.c_double), int(q),
                              _p(ref, C.c_double) if ref is not None else None, _p(st, C.c_double),
                              _p(P, C.c_double), C.byref(chi2), C.byref(ndof), C.byref(nu), _p(each, C.c_double))
    return dict(status=status, state=st, cov=P.reshape(6, 6), chi2=chi2.value, ndof=ndof.value,
                n_used=nu.value, chi2_each=each)


# ---------------------------------------------------------------- batched entry points

def fit(geom, hits, seeds=None, q=None, seed_cov=1e4, ms_on=True, t0=0, t1=None, threads=1, meas_model=0):
    """Fit every track of a CSR hit set.  hits: dict offsets (n+1,), layer, x, y, z.
    meas_model 1: barrel hits after the first reached on their own radius, 2-D update there
    (non-ideal geometry); the first hit, where the state starts, takes the 3-D update.
    Returns dict with seed, q, state (n,6), cov (n,6,6), chi2, ndof, status."""
    cfg = fit_cfg(geom, seed_cov, ms_on, meas_model)
    sarr = surfaces(geom)
    off = np.ascontiguousarray(hits["offsets"], dtype=np.int32)
    n = len(off) - 1
    if t1 is None:
        t1 = n
    layer = np.ascontiguousarray(hits["layer"], dtype=np.uint8)
    x, y, z = (np.ascontiguousarray(hits[k], dtype=np.float32) for k in ("x", "y", "z"))
    sd = None
    qi = None
    if seeds is not None:
        sd = np.ascontiguousarray(seeds, dtype=np.float64)
        qi = np.ascontiguousarray(q, dtype=np.int8)
    out = dict(seed=np.zeros((n, 6)), q=np.zeros(n, np.int8), state=np.zeros((n, 6)),
               cov=np.zeros((n, 6, 6)), chi2=np.zeros(n), ndof=np.zeros(n, np.int32),
               status=np.zeros(n, np.uint32))
    L = lib()

    def run(a, b):
        L.or_fit_tracks(C.byref(cfg), sarr, int(a), int(b), _p(off, C.c_int32),
                        _p(layer, C.c_uint8) if len(layer) else None,
                        _p(x, C.c_float), _p(y, C.c_float), _p(z, C.c_float),
                        _p(sd, C.c_double) if sd is not None else None,
                        _p(qi, C.c_int8) if qi is not None else None,
                        _p(out["seed"], C.c_double), _p(out["q"], C.c_int8), _p(out["state"], C.c_double),
                        _p(out["cov"], C.c_double), _p(out["chi2"], C.c_double), _p(out["ndof"], C.c_int32),
                        _p(out["status"], C.c_uint32))

    _run_ranges(run, t0, t1, threads)
    return out


def _run_ranges(fn, t0, t1, threads):
    if threads <= 1 or t1 - t0 < 2 * threads:
        fn(t0, t1)
        return
    edges = np.linspace(t0, t1, threads + 1).astype(int)
    ths = [threading.Thread(target=fn, args=(int(edges[i]), int(edges[i + 1]))) for i in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()


def bin_key(x, y, z, half_len):
    return lib().or_bin_key(float(np.float32(x)), float(np.float32(y)), float(np.float32(z)), float(half_len))


def bin_layer(x, y, z, half_len):
    """Stable counting sort of one layer's hits by (z_bin * 1024 + phi_bin)."""
    x, y, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
    n = len(x)
    perm = np.zeros(max(n, 1), np.int32)
    offsets = np.zeros(1024 * 64 + 1, np.int32)
    lib().or_bin_layer(n, _p(x, C.c_float), _p(y, C.c_float), _p(z, C.c_float), float(half_len),
                       _p(perm, C.c_int32), _p(offsets, C.c_int32))
    return perm[:n], offsets


def build_besthit(geom, event, nsigma=3.0, chi2_cut=30.0, max_cand=32, seed_cov=1e4, ms_on=True, t0=0, t1=None,
          record=False, threads=1, meas_model=0):
    """Best-hit building of one event.  event: dict with 'layers' (list of dicts x, y, z, perm, offsets,
    surf), 'seed_hits' (n,3,3) float32, 'seed_idx' (n,3) int32.  meas_model 1: two-step
    propagation (layer average cylinder, then each candidate's own) and 2-D updates."""
    fc = fit_cfg(geom, seed_cov, ms_on, meas_model)
    bc = BuildCfg(nsigma=float(nsigma), chi2_cut=float(chi2_cut), max_cand=int(min(max_cand, 1024)))
    sarr = surfaces(geom)
    lays = event["layers"]
    nlay = len(lays)
    keep = []
    larr = (Layer * nlay)()
    for i, ly in enumerate(lays):
        arrs = [np.ascontiguousarray(ly[k], dtype=np.float32) for k in ("x", "y", "z")]
        perm = np.ascontiguousarray(ly["perm"], dtype=np.int32) if ly.get("perm") is not None else None
        offs = np.ascontiguousarray(ly["offsets"], dtype=np.int32) if ly.get("offsets") is not None else None
        keep += arrs + [perm, offs]
        larr[i].n = len(arrs[0])
        larr[i].surf = int(ly["surf"])
        larr[i].x = _p(arrs[0], C.c_float)
        larr[i].y = _p(arrs[1], C.c_float)
        larr[i].z = _p(arrs[2], C.c_float)
        larr[i].perm = _p(perm, C.c_int32) if perm is not None else None
        larr[i].offsets = _p(offs, C.c_int32) if offs is not None else None
    sh = np.ascontiguousarray(event["seed_hits"], dtype=np.float32).reshape(-1, 9)
    si = np.ascontiguousarray(event["seed_idx"], dtype=np.int32).reshape(-1, 3)
    n = sh.shape[0]
    if t1 is None:
        t1 = n
    out = dict(idx=np.full((n, nlay), -1, np.int32), state=np.zeros((n, 6)), cov=np.zeros((n, 6, 6)),
               chi2=np.zeros(n), ndof=np.zeros(n, np.int32), status=np.zeros(n, np.uint32))
    rec = np.zeros((n, nlay), STEP_DTYPE) if record else None
    L = lib()

    def run(a, b):
        L.or_build_tracks(C.byref(fc), C.byref(bc), sarr, nlay, larr, int(a), int(b), _p(sh, C.c_float),
                          _p(si, C.c_int32), _p(out["idx"], C.c_int32), _p(out["state"], C.c_double),
                          _p(out["cov"], C.c_double), _p(out["chi2"], C.c_double), _p(out["ndof"], C.c_int32),
                          _p(out["status"], C.c_uint32), rec.ctypes.data if rec is not None else None)

    _run_ranges(run, t0, t1, threads)
    if record:
        out["rec"] = rec
    return out


def besthit_step(geom, layer, st, P, q, nsigma=3.0, chi2_cut=30.0, max_cand=32, meas_model=0, seed_cov=1e4,
                 ms_on=True):
    """One best-hit step (window, candidates, chi2, best) on one binned layer (dict x, y, z, perm,
    offsets, surf) from the predicted state st (6) and covariance P (6x6) given in FP64.
    Returns the step record (STEP_DTYPE fields) with 'best' the best hit (no chi2 cut)."""
    fc = fit_cfg(geom, seed_cov, ms_on, meas_model)
    bc = BuildCfg(nsigma=float(nsigma), chi2_cut=float(chi2_cut), max_cand=int(min(max_cand, 1024)))
    surf = surfaces(geom)
    arrs = [np.ascontiguousarray(layer[k], dtype=np.float32) for k in ("x", "y", "z")]
    perm = np.ascontiguousarray(layer["perm"], dtype=np.int32)
    offs = np.ascontiguousarray(layer["offsets"], dtype=np.int32)
    ly = Layer(n=len(arrs[0]), surf=int(layer["surf"]), x=_p(arrs[0], C.c_float), y=_p(arrs[1], C.c_float),
               z=_p(arrs[2], C.c_float), perm=_p(perm, C.c_int32), offsets=_p(offs, C.c_int32))
    st = np.ascontiguousarray(st, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(36)
    rec = StepRec()
    c2 = C.c_double(0.0)
    best = lib().or_besthit_step(C.byref(fc), C.byref(bc), C.byref(surf[int(layer["surf"])]), C.byref(ly),
                                 _p(st, C.c_double), _p(P, C.c_double), int(q), C.byref(c2), C.byref(rec))
    out = {name: getattr(rec, name) for name, _ in StepRec._fields_}
    out["pred"] = np.array(rec.pred)
    out["best"] = int(best)
    return out


def _layers_array(event):
    lays = event["layers"]
    keep = []
    larr = (Layer * len(lays))()
    for i, ly in enumerate(lays):
        arrs = [np.ascontiguousarray(ly[k], dtype=np.float32) for k in ("x", "y", "z")]
        perm = np.ascontiguousarray(ly["perm"], dtype=np.int32) if ly.get("perm") is not None else None
        offs = np.ascontiguousarray(ly["offsets"], dtype=np.int32) if ly.get("offsets") is not None else None
        keep += arrs + [perm, offs]
        larr[i].n = len(arrs[0])
        larr[i].surf = int(ly["surf"])
        larr[i].x = _p(arrs[0], C.c_float)
        larr[i].y = _p(arrs[1], C.c_float)
        larr[i].z = _p(arrs[2], C.c_float)
        larr[i].perm = _p(perm, C.c_int32) if perm is not None else None
        larr[i].offsets = _p(offs, C.c_int32) if offs is not None else None
    return larr, keep


def build_ckf(geom, event, n_slots=4, nsigma=3.0, chi2_cut=30.0, max_cand=32, seed_cov=1e4, ms_on=True, t0=0,
              t1=None, threads=1):
    """Combinatorial building of one event (n_slots candidates per seed); event as build_besthit.
    Returns idx (n, nlay), state, cov, chi2, ndof, status and margin (n, CKF_MARGIN_DTYPE)."""
    fc = fit_cfg(geom, seed_cov, ms_on)
    cc = CkfCfg(nsigma=float(nsigma), chi2_cut=float(chi2_cut), max_cand=int(min(max_cand, 1024)),
                n_slots=int(n_slots))
    sarr = surfaces(geom)
    larr, keep = _layers_array(event)
    nlay = len(event["layers"])
    sh = np.ascontiguousarray(event["seed_hits"], dtype=np.float32).reshape(-1, 9)
    si = np.ascontiguousarray(event["seed_idx"], dtype=np.int32).reshape(-1, 3)
    n = sh.shape[0]
    if t1 is None:
        t1 = n
    out = dict(idx=np.full((n, nlay), -1, np.int32), state=np.zeros((n, 6)), cov=np.zeros((n, 6, 6)),
               chi2=np.zeros(n), ndof=np.zeros(n, np.int32), status=np.zeros(n, np.uint32),
               margin=np.zeros(n, CKF_MARGIN_DTYPE))
    L = lib()

    def run(a, b):
        L.or_ckf_tracks(C.byref(fc), C.byref(cc), sarr, nlay, larr, int(a), int(b), _p(sh, C.c_float),
                        _p(si, C.c_int32), _p(out["idx"], C.c_int32), _p(out["state"], C.c_double),
                        _p(out["cov"], C.c_double), _p(out["chi2"], C.c_double), _p(out["ndof"], C.c_int32),
                        _p(out["status"], C.c_uint32), out["margin"].ctypes.data)

    _run_ranges(run, t0, t1, threads)
    del keep
    return out


def refit_inward(geom, hits, fwd_state, fwd_cov, q, fwd_ndof, cov_scale=100.0, seed_cov=1e4, ms_on=True, t0=0,
                 t1=None, threads=1, meas_model=0):
    """Outward-inward refit: the hits each forward fit used ((ndof + 5) / 2 of them) fitted
    again from the last back to the first, starting from the forward state at the last used
    hit with the forward covariance times cov_scale (fwd_state (n, 6), fwd_cov (n, 6, 6),
    q (n,), fwd_ndof (n,)).  Returns the state (n, 6) and cov (n, 6, 6) at the first hit,
    chi2, ndof, status."""
    cfg = fit_cfg(geom, seed_cov, ms_on, meas_model)
    sarr = surfaces(geom)
    off = np.ascontiguousarray(hits["offsets"], dtype=np.int32)
    n = len(off) - 1
    if t1 is None:
        t1 = n
    layer = np.ascontiguousarray(hits["layer"], dtype=np.uint8)
    x, y, z = (np.ascontiguousarray(hits[k], dtype=np.float32) for k in ("x", "y", "z"))
    fwd = np.ascontiguousarray(fwd_state, dtype=np.float64).reshape(n, 6)
    fcv = np.ascontiguousarray(fwd_cov, dtype=np.float64).reshape(n, 36)
    qi = np.ascontiguousarray(q, dtype=np.int8)
    nd = np.ascontiguousarray(fwd_ndof, dtype=np.int32)
    out = dict(state=np.zeros((n, 6)), cov=np.zeros((n, 6, 6)), chi2=np.zeros(n), ndof=np.zeros(n, np.int32),
               status=np.zeros(n, np.uint32))
    L = lib()

    def run(a, b):
        L.or_refit_tracks(C.byref(cfg), sarr, int(a), int(b), _p(off, C.c_int32),
                          layer.ctypes.data if len(layer) else None, _p(x, C.c_float), _p(y, C.c_float),
                          _p(z, C.c_float), _p(fwd, C.c_double), _p(fcv, C.c_double), float(cov_scale),
                          _p(qi, C.c_int8), _p(nd, C.c_int32),
                          _p(out["state"], C.c_double),
                          _p(out["cov"], C.c_double), _p(out["chi2"], C.c_double), _p(out["ndof"], C.c_int32),
                          _p(out["status"], C.c_uint32))

    _run_ranges(run, t0, t1, threads)
    return out
