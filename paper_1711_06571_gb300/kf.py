"""Thin Python binding of libkf.so (include/kf.h): ctypes structures with the
same layout and functions with the same names, taking torch CUDA tensors.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing works without a GPU; any call raises if the library has
not been built (no fallback of any kind).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkf.so")

KF_OK = 0
KF_EINVAL = -1
KF_ENOMEM = -2
KF_ECUDA = -3
KF_ETIMEOUT = -4
KF_EAGAIN = -5
KF_EBUSY = -6
KF_ESIZE = -7
KF_STATIC_MAX_HITS = 262144
KF_EVENT_ZERO_COPY = 1

KF_ST_NO_INTERSECT = 1
KF_ST_CHOL_FAIL = 2
KF_ST_NONFINITE = 4
KF_ST_CAND_CAPPED = 8
KF_ST_GRAZING = 16
KF_ST_THETA_RANGE = 32
KF_ST_FP64_TRACK = 64

KF_PREC_MIXED = 0
KF_PREC_FP64 = 1
KF_SCHED_GRID = 0
KF_SCHED_PERSISTENT = 1
KF_MEAS_LAYER = 0
KF_MEAS_HIT_2D = 1
KF_SEED_UD_DF = 0
KF_SEED_JOSEPH_FP64 = 1
KF_MAX_SURFACES = 64
KF_NPHI = 1024
KF_NZ = 64
KF_NBINS = KF_NPHI * KF_NZ


class KfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libkf error {code}: {msg}")
        self.code = code


class kf_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("pos", C.c_double), ("half_or_rin", C.c_double),
                ("r_out", C.c_double), ("x_x0", C.c_double), ("sig_n", C.c_double), ("sig_rphi", C.c_double),
                ("sig_3", C.c_double), ("dr", C.c_double)]


class kf_geometry(C.Structure):
    _fields_ = [("bz", C.c_double), ("mass", C.c_double), ("n_surfaces", C.c_int32), ("pad_", C.c_int32),
                ("surfaces", C.POINTER(kf_surface))]


class kf_fit_params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_fp64_updates", C.c_int32), ("seed_cov", C.c_double),
                ("ms_on", C.c_int32), ("schedule", C.c_int32), ("meas_model", C.c_int32),
                ("seed_update", C.c_int32)]


class kf_seeds(C.Structure):
    _fields_ = [("state", C.c_void_p), ("q", C.c_void_p)]


class kf_track_hits(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("layer", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p),
                ("z", C.c_void_p)]


class kf_tracks_out(C.Structure):
    _fields_ = [("state", C.c_void_p), ("cov", C.c_void_p), ("chi2", C.c_void_p), ("ndof", C.c_void_p),
                ("status", C.c_void_p), ("cov_f32", C.c_void_p)]


class kf_binned_layer(C.Structure):
    _fields_ = [("n_hits", C.c_int32), ("surface", C.c_int32), ("packed", C.c_void_p), ("offsets", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p)]


class kf_build_params(C.Structure):
    _fields_ = [("nsigma", C.c_double), ("chi2_cut", C.c_double), ("max_cand", C.c_int32),
                ("warp_coop", C.c_int32), ("debug_pred", C.c_void_p)]


class kf_server_params(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("host_staging_bytes", C.c_size_t), ("max_batches", C.c_int32),
                ("max_batch_events", C.c_int32), ("fit", kf_fit_params), ("build", kf_build_params),
                ("batch_window_ms", C.c_double)]


class kf_event(C.Structure):
    _fields_ = [("n_tracks", C.c_int32), ("n_layers", C.c_int32), ("surface", C.POINTER(C.c_int32)),
                ("n_hits", C.POINTER(C.c_int32)), ("x", C.POINTER(C.c_void_p)), ("y", C.POINTER(C.c_void_p)),
                ("z", C.POINTER(C.c_void_p)), ("seed_hits", C.c_void_p), ("flags", C.c_int32),
                ("pad_", C.c_int32)]


class kf_event_result(C.Structure):
    _fields_ = [("hit_idx", C.c_void_p), ("state", C.c_void_p), ("cov", C.c_void_p), ("chi2", C.c_void_p),
                ("ndof", C.c_void_p), ("status", C.c_void_p)]


class kf_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("batches", C.c_uint64), ("queued", C.c_int32), ("in_flight_events", C.c_int32),
                ("in_flight_batches", C.c_int32), ("pad_", C.c_int32), ("bytes_in_use", C.c_size_t),
                ("peak_bytes_in_use", C.c_size_t), ("mean_batch_events", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("mean_ms", C.c_double),
                ("events_per_s", C.c_double), ("tracks_per_s", C.c_double), ("batch_device_ms", C.c_double),
                ("copy_out_ms", C.c_double), ("stage_ms", C.c_double)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); every symbol of include/kf.h
_SIGS = {
    "kf_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]),
    "kf_ctx_destroy": (None, [C.c_void_p]),
    "kf_ctx_last_error": (C.c_char_p, [C.c_void_p]),
    "kf_version": (C.c_char_p, []),
    "kf_make_seeds": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.c_int32, C.POINTER(kf_track_hits),
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "kf_fit": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params), C.c_int32,
                         C.POINTER(kf_seeds), C.POINTER(kf_track_hits), C.POINTER(kf_tracks_out), C.c_void_p]),
    "kf_refit_inward": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params), C.c_int32,
                                  C.POINTER(kf_track_hits), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_double, C.POINTER(kf_tracks_out), C.c_void_p]),
    "kf_fit_host": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params), C.c_int32,
                              C.POINTER(kf_track_hits), C.POINTER(kf_tracks_out), C.c_int32]),
    "kf_fit_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "kf_fit_phase_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    "kf_autotune_fit": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params), C.c_int32,
                                  C.POINTER(kf_seeds), C.POINTER(kf_track_hits), C.POINTER(kf_tracks_out),
                                  C.c_void_p, C.c_char_p, C.c_size_t]),
    "kf_bin_hits": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "kf_build_besthit": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params),
                                   C.POINTER(kf_build_params), C.c_int32, C.c_int32, C.POINTER(kf_binned_layer),
                                   C.POINTER(C.c_int32), C.POINTER(kf_seeds), C.c_void_p, C.c_void_p,
                                   C.POINTER(kf_tracks_out), C.c_void_p]),
    "kf_bin_hits_batched": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "kf_build_ckf": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_fit_params),
                               C.POINTER(kf_build_params), C.c_int32, C.c_int32, C.c_int32, C.POINTER(kf_binned_layer),
                               C.POINTER(C.c_int32), C.POINTER(kf_seeds), C.c_void_p, C.c_void_p,
                               C.POINTER(kf_tracks_out), C.c_void_p]),
    "kf_bin_hits_static": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "kf_measure_peak": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "kf_layout_transport": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "kf_gather_hits": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(kf_binned_layer),
                                 C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "kf_server_create": (C.c_int, [C.c_void_p, C.POINTER(kf_geometry), C.POINTER(kf_server_params),
                                   C.POINTER(C.c_void_p)]),
    "kf_server_submit": (C.c_int, [C.c_void_p, C.POINTER(kf_event), C.POINTER(kf_event_result),
                                   C.POINTER(C.c_uint64)]),
    "kf_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double)]),
    "kf_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(C.c_double)]),
    "kf_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(kf_server_stats), C.c_int]),
    "kf_server_destroy": (None, [C.c_void_p]),
}


def load(path: str = LIB_PATH):
    """Load libkf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libkf.so not found at {path}: build it with "
                                   "paper_1711_06571_gb300.build.build() (there is no CPU fallback)")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(ctx, rc):
    if rc != KF_OK:
        msg = load().kf_ctx_last_error(ctx)
        raise KfError(rc, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_geometry(geom: dict):
    """kf_geometry from a geometry dict (synth.geometry); keeps the surface array alive."""
    surfs = geom["surfaces"]
    arr = (kf_surface * len(surfs))()
    for i, s in enumerate(surfs):
        arr[i].kind = int(s["kind"])
        arr[i].pos = float(s["pos"])
        arr[i].half_or_rin = float(s["half_or_rin"])
        arr[i].r_out = float(s.get("r_out", 0.0))
        arr[i].x_x0 = float(s["x_x0"])
        arr[i].sig_n = float(s["sig_n"])
        arr[i].sig_rphi = float(s["sig_rphi"])
        arr[i].sig_3 = float(s["sig_3"])
        arr[i].dr = float(s.get("dr", 0.0))
    g = kf_geometry(bz=float(geom["bz"]), mass=float(geom["mass"]), n_surfaces=len(surfs),
                    surfaces=C.cast(arr, C.POINTER(kf_surface)))
    g._keep = arr
    return g


def fit_params(precision=KF_PREC_MIXED, n_fp64_updates=3, seed_cov=1e4, ms_on=True, schedule=KF_SCHED_GRID,
               meas_model=KF_MEAS_LAYER, seed_update=KF_SEED_UD_DF):
    return kf_fit_params(precision=int(precision), n_fp64_updates=int(n_fp64_updates), seed_cov=float(seed_cov),
                         ms_on=int(bool(ms_on)), schedule=int(schedule), meas_model=int(meas_model),
                         seed_update=int(seed_update))


# ---------------------------------------------------------------- entry points (same names as kf.h)

def kf_version() -> str:
    return load().kf_version().decode()


def kf_ctx_create(device: int = 0, budget: int = 0):
    h = C.c_void_p()
    rc = load().kf_ctx_create(C.byref(h), int(device), C.c_size_t(int(budget)))
    if rc != KF_OK:
        raise KfError(rc, "kf_ctx_create failed")
    return h


def kf_ctx_destroy(ctx):
    load().kf_ctx_destroy(ctx)


def kf_ctx_last_error(ctx) -> str:
    m = load().kf_ctx_last_error(ctx)
    return m.decode() if m else ""


def kf_make_seeds(ctx, geom, n, offsets, x, y, z, state_out, q_out, stream=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    h = kf_track_hits(_ptr(offsets), None, _ptr(x), _ptr(y), _ptr(z))
    _check(ctx, load().kf_make_seeds(ctx, C.byref(g), int(n), C.byref(h), _ptr(state_out), _ptr(q_out),
                                     _stream(stream)))


def kf_fit(ctx, geom, params, n, seed_state, seed_q, offsets, layer, x, y, z, out_state=None, out_cov=None,
           out_chi2=None, out_ndof=None, out_status=None, stream=None,
           out_cov_f32=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    p = params if params is not None else fit_params()
    s = kf_seeds(_ptr(seed_state), _ptr(seed_q))
    h = kf_track_hits(_ptr(offsets), _ptr(layer), _ptr(x), _ptr(y), _ptr(z))
    o = kf_tracks_out(_ptr(out_state), _ptr(out_cov), _ptr(out_chi2), _ptr(out_ndof), _ptr(out_status),
                      _ptr(out_cov_f32))
    _check(ctx, load().kf_fit(ctx, C.byref(g), C.byref(p), int(n), C.byref(s), C.byref(h), C.byref(o),
                              _stream(stream)))


def kf_refit_inward(ctx, geom, params, n, offsets, layer, x, y, z, fwd_state, fwd_cov, q, fwd_ndof, cov_scale=100.0,
                    out_state=None, out_cov=None, out_chi2=None, out_ndof=None, out_status=None, stream=None,
                    out_cov_f32=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    p = params if params is not None else fit_params()
    h = kf_track_hits(_ptr(offsets), _ptr(layer), _ptr(x), _ptr(y), _ptr(z))
    o = kf_tracks_out(_ptr(out_state), _ptr(out_cov), _ptr(out_chi2), _ptr(out_ndof), _ptr(out_status),
                      _ptr(out_cov_f32))
    _check(ctx, load().kf_refit_inward(ctx, C.byref(g), C.byref(p), int(n), C.byref(h), _ptr(fwd_state),
                                       _ptr(fwd_cov), _ptr(q), _ptr(fwd_ndof), float(cov_scale), C.byref(o),
                                       _stream(stream)))


def _hptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.is_cuda:
            raise ValueError("kf_fit_host takes host tensors")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)  # numpy


def kf_fit_host(ctx, geom, params, n, offsets, layer, x, y, z, out_state=None, out_cov=None, out_chi2=None,
                out_ndof=None, out_status=None, n_chunks=0, out_cov_f32=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    p = params if params is not None else fit_params()
    h = kf_track_hits(_hptr(offsets), _hptr(layer), _hptr(x), _hptr(y), _hptr(z))
    o = kf_tracks_out(_hptr(out_state), _hptr(out_cov), _hptr(out_chi2), _hptr(out_ndof), _hptr(out_status),
                      _hptr(out_cov_f32))
    _check(ctx, load().kf_fit_host(ctx, C.byref(g), C.byref(p), int(n), C.byref(h), C.byref(o), int(n_chunks)))


def kf_fit_timing(ctx, enable=True):
    _check(ctx, load().kf_fit_timing(ctx, int(bool(enable))))


def kf_fit_phase_times(ctx):
    """(timed calls, mean phase-1 ms, mean phase-2 ms) of the grid-schedule kf_fit calls
    timed on ctx since kf_fit_timing(ctx, True)."""
    m, a, b = C.c_int32(0), C.c_double(0.0), C.c_double(0.0)
    _check(ctx, load().kf_fit_phase_times(ctx, C.byref(m), C.byref(a), C.byref(b)))
    return m.value, a.value, b.value


def kf_autotune_fit(ctx, geom, params, n, seed_state, seed_q, offsets, layer, x, y, z, out_state=None,
                    out_cov=None, out_chi2=None, out_ndof=None, out_status=None, stream=None,
                    out_cov_f32=None) -> str:
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    p = params if params is not None else fit_params()
    s = kf_seeds(_ptr(seed_state), _ptr(seed_q))
    h = kf_track_hits(_ptr(offsets), _ptr(layer), _ptr(x), _ptr(y), _ptr(z))
    o = kf_tracks_out(_ptr(out_state), _ptr(out_cov), _ptr(out_chi2), _ptr(out_ndof), _ptr(out_status),
                      _ptr(out_cov_f32))
    buf = C.create_string_buffer(128)
    _check(ctx, load().kf_autotune_fit(ctx, C.byref(g), C.byref(p), int(n), C.byref(s), C.byref(h), C.byref(o),
                                       _stream(stream), buf, 128))
    return buf.value.decode()


def kf_bin_hits(ctx, n_hits, x, y, z, half_len, perm_out, offsets_out, packed_out=None, stream=None):
    _check(ctx, load().kf_bin_hits(ctx, int(n_hits), _ptr(x), _ptr(y), _ptr(z), float(half_len), _ptr(perm_out),
                                   _ptr(offsets_out), _ptr(packed_out), _stream(stream)))


def kf_bin_hits_batched(ctx, segment_offsets, half_len, x, y, z, perm_out, offsets_out, packed_out=None,
                        stream=None):
    """Bin many layers in one pass: segment_offsets (n_segments + 1) and half_len (n_segments) are host
    sequences; x, y, z the concatenated device coordinates."""
    ns = len(half_len)
    so = (C.c_int32 * (ns + 1))(*[int(v) for v in segment_offsets])
    hl = (C.c_double * ns)(*[float(v) for v in half_len])
    _check(ctx, load().kf_bin_hits_batched(ctx, ns, so, hl, _ptr(x), _ptr(y), _ptr(z), _ptr(perm_out),
                                           _ptr(offsets_out), _ptr(packed_out), _stream(stream)))


def kf_bin_hits_static(n_hits, x, y, z, half_len, perm_out, offsets_out, packed_out=None, stream=None) -> int:
    """Allocation-free binning (no context); returns the library's status code."""
    return load().kf_bin_hits_static(int(n_hits), _ptr(x), _ptr(y), _ptr(z), float(half_len), _ptr(perm_out),
                                     _ptr(offsets_out), _ptr(packed_out), _stream(stream))


def binned_layers(layer_dicts):
    """kf_binned_layer array from dicts with n_hits, surface and tensors packed, offsets (and x, y, z)."""
    arr = (kf_binned_layer * len(layer_dicts))()
    for i, d in enumerate(layer_dicts):
        arr[i].n_hits = int(d["n_hits"])
        arr[i].surface = int(d["surface"])
        arr[i].packed = _ptr(d.get("packed"))
        arr[i].offsets = _ptr(d.get("offsets"))
        arr[i].x = _ptr(d.get("x"))
        arr[i].y = _ptr(d.get("y"))
        arr[i].z = _ptr(d.get("z"))
    return arr


def build_params(nsigma=3.0, chi2_cut=30.0, max_cand=32, warp_coop=False, debug_pred=None):
    """debug_pred: None, or a CUDA FP64 tensor of n_layers * 27 * n values (kf_build_besthit
    writes each track's predicted state and covariance per build layer into it)."""
    return kf_build_params(nsigma=float(nsigma), chi2_cut=float(chi2_cut), max_cand=int(max_cand),
                           warp_coop=int(bool(warp_coop)),
                           debug_pred=None if debug_pred is None else debug_pred.data_ptr())


def kf_build_besthit(ctx, geom, fit, bp, n_events, n_layers, layers, event_offsets, seed_state, seed_q, seed_hits,
                     hit_idx_out, out_state=None, out_cov=None, out_chi2=None, out_ndof=None, out_status=None,
                     stream=None, out_cov_f32=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    f = fit if fit is not None else fit_params()
    b = bp if bp is not None else build_params()
    eo = (C.c_int32 * (n_events + 1))(*[int(v) for v in event_offsets])
    s = kf_seeds(_ptr(seed_state), _ptr(seed_q))
    o = kf_tracks_out(_ptr(out_state), _ptr(out_cov), _ptr(out_chi2), _ptr(out_ndof), _ptr(out_status),
                      _ptr(out_cov_f32))
    _check(ctx, load().kf_build_besthit(ctx, C.byref(g), C.byref(f), C.byref(b), int(n_events), int(n_layers),
                                        layers, eo, C.byref(s), _ptr(seed_hits), _ptr(hit_idx_out), C.byref(o),
                                        _stream(stream)))


def kf_build_ckf(ctx, geom, fit, bp, n_slots, n_events, n_layers, layers, event_offsets, seed_state, seed_q,
                 seed_hits, hit_idx_out, out_state=None, out_cov=None, out_chi2=None, out_ndof=None, out_status=None,
                 stream=None, out_cov_f32=None):
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    f = fit if fit is not None else fit_params()
    b = bp if bp is not None else build_params()
    eo = (C.c_int32 * (n_events + 1))(*[int(v) for v in event_offsets])
    s = kf_seeds(_ptr(seed_state), _ptr(seed_q))
    o = kf_tracks_out(_ptr(out_state), _ptr(out_cov), _ptr(out_chi2), _ptr(out_ndof), _ptr(out_status),
                      _ptr(out_cov_f32))
    _check(ctx, load().kf_build_ckf(ctx, C.byref(g), C.byref(f), C.byref(b), int(n_slots), int(n_events),
                                    int(n_layers), layers, eo, C.byref(s), _ptr(seed_hits), _ptr(hit_idx_out),
                                    C.byref(o), _stream(stream)))


def kf_gather_hits(ctx, n_events, n_layers, layers, event_offsets, seed_hits, hit_idx, offsets_out, layer_out,
                   x_out, y_out, z_out, stream=None):
    eo = (C.c_int32 * (n_events + 1))(*[int(v) for v in event_offsets])
    _check(ctx, load().kf_gather_hits(ctx, int(n_events), int(n_layers), layers, eo, _ptr(seed_hits),
                                      _ptr(hit_idx), _ptr(offsets_out), _ptr(layer_out), _ptr(x_out), _ptr(y_out),
                                      _ptr(z_out), _stream(stream)))


KF_LAYOUT_AOS = 0
KF_LAYOUT_SOA = 1
KF_LAYOUT_BLOCK = 2


def kf_layout_transport(ctx, layout, n, J, P, P_out, stream=None):
    _check(ctx, load().kf_layout_transport(ctx, int(layout), int(n), _ptr(J), _ptr(P), _ptr(P_out), _stream(stream)))


def kf_measure_peak(ctx, which: int) -> float:
    """Measured FMA throughput (FLOP/s): which = 0 FP64, 1 FP32."""
    v = C.c_double(0.0)
    _check(ctx, load().kf_measure_peak(ctx, int(which), C.byref(v)))
    return v.value


# ---------------------------------------------------------------- serving

class Server:
    """Handle of a kf_server: the raw pointer plus the result arrays of the
    tickets not yet reported (the dispatcher thread writes into them)."""

    def __init__(self, ptr, ctx):
        self.ptr = ptr
        self.ctx = ctx
        self.results = {}


def server_params(mem_budget_bytes=0, host_staging_bytes=0, max_batches=0, max_batch_events=0, fit=None,
                  build=None, batch_window_ms=0.0):
    p = kf_server_params(mem_budget_bytes=int(mem_budget_bytes), host_staging_bytes=int(host_staging_bytes),
                         max_batches=int(max_batches), max_batch_events=int(max_batch_events),
                         batch_window_ms=float(batch_window_ms))
    if fit is not None:
        p.fit = fit
    if build is not None:
        p.build = build
    return p


def kf_server_create(ctx, geom, params=None) -> Server:
    g = geom if isinstance(geom, kf_geometry) else make_geometry(geom)
    p = params if params is not None else server_params()
    out = C.c_void_p()
    _check(ctx, load().kf_server_create(ctx, C.byref(g), C.byref(p), C.byref(out)))
    return Server(out, ctx)


def _np_ptr(a, dtype):
    import numpy as np
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise ValueError(f"expected a C-contiguous numpy array of {dtype}")
    return C.c_void_p(a.ctypes.data)


def kf_server_submit(srv: Server, n_tracks, surfaces, x, y, z, seed_hits, hit_idx=None, state=None, cov=None,
                     chi2=None, ndof=None, status=None, zero_copy=False):
    """Queue one event.  surfaces: list of geometry indices (first three = seed
    layers); x, y, z: per layer numpy float32 arrays (layers 0..2 may be None);
    seed_hits: float32 [n_tracks, 3, 3]; result arrays: numpy, shapes as in the
    C header.  zero_copy: the input arrays stay alive and unchanged until the
    ticket completes (the handle keeps references to them until it is reported).
    Returns (code, ticket): code KF_OK, KF_EBUSY or KF_EAGAIN."""
    import numpy as np
    L = len(surfaces)
    sf = (C.c_int32 * L)(*[int(v) for v in surfaces])
    nh = (C.c_int32 * L)(*[0 if x[l] is None else int(len(x[l])) for l in range(L)])
    xs = (C.c_void_p * L)(*[None if x[l] is None else _np_ptr(x[l], np.float32).value for l in range(L)])
    ys = (C.c_void_p * L)(*[None if y[l] is None else _np_ptr(y[l], np.float32).value for l in range(L)])
    zs = (C.c_void_p * L)(*[None if z[l] is None else _np_ptr(z[l], np.float32).value for l in range(L)])
    ev = kf_event(n_tracks=int(n_tracks), n_layers=L, surface=sf, n_hits=nh,
                  x=C.cast(xs, C.POINTER(C.c_void_p)), y=C.cast(ys, C.POINTER(C.c_void_p)),
                  z=C.cast(zs, C.POINTER(C.c_void_p)), seed_hits=_np_ptr(seed_hits, np.float32),
                  flags=KF_EVENT_ZERO_COPY if zero_copy else 0)
    res = kf_event_result(_np_ptr(hit_idx, np.int32), _np_ptr(state, np.float64), _np_ptr(cov, np.float64),
                          _np_ptr(chi2, np.float64), _np_ptr(ndof, np.int32), _np_ptr(status, np.uint32))
    t = C.c_uint64(0)
    rc = load().kf_server_submit(srv.ptr, C.byref(ev), C.byref(res), C.byref(t))
    if rc == KF_OK:
        srv.results[t.value] = (hit_idx, state, cov, chi2, ndof, status) + ((x, y, z, seed_hits) if zero_copy else ())
    elif rc == KF_EINVAL:
        raise KfError(rc, "kf_server_submit: malformed event")
    return rc, t.value


def kf_server_poll(srv: Server, ticket):
    """(code, latency_ms); KF_EAGAIN while pending."""
    lat = C.c_double(0.0)
    rc = load().kf_server_poll(srv.ptr, int(ticket), C.byref(lat))
    if rc != KF_EAGAIN:
        srv.results.pop(int(ticket), None)
    return rc, lat.value


def kf_server_wait(srv: Server, ticket, timeout_ms=60000.0):
    lat = C.c_double(0.0)
    rc = load().kf_server_wait(srv.ptr, int(ticket), float(timeout_ms), C.byref(lat))
    if rc != KF_ETIMEOUT:
        srv.results.pop(int(ticket), None)
    return rc, lat.value


def kf_server_stats_get(srv: Server, reset=False) -> dict:
    st = kf_server_stats()
    rc = load().kf_server_stats_get(srv.ptr, C.byref(st), int(bool(reset)))
    d = {name: getattr(st, name) for name, _ in kf_server_stats._fields_ if name != "pad_"}
    d["rc"] = rc
    return d


def kf_server_destroy(srv: Server):
    if srv is not None and srv.ptr:
        load().kf_server_destroy(srv.ptr)
        srv.ptr = None
        srv.results.clear()
