"""Device plumbing around the binding: move synthetic inputs into torch CUDA
tensors, allocate outputs, call the libkf entry points, bring results back.

Nothing here computes any step of the method; it only allocates and copies.
"""
from __future__ import annotations

import numpy as np
import torch

from . import kf

_ctx_cache = {}


def context(device: int = 0, budget: int = 0):
    """One libkf context per device for the life of the process."""
    key = (device, budget)
    if key not in _ctx_cache:
        _ctx_cache[key] = kf.kf_ctx_create(device, budget)
    return _ctx_cache[key]


def hits_to_device(tk: dict, device="cuda"):
    """CSR hits (numpy) -> dict of contiguous CUDA tensors."""
    dev = torch.device(device)
    return dict(
        offsets=torch.from_numpy(np.ascontiguousarray(tk["offsets"], np.int32)).to(dev),
        layer=torch.from_numpy(np.ascontiguousarray(tk["layer"], np.uint8)).to(dev),
        x=torch.from_numpy(np.ascontiguousarray(tk["x"], np.float32)).to(dev),
        y=torch.from_numpy(np.ascontiguousarray(tk["y"], np.float32)).to(dev),
        z=torch.from_numpy(np.ascontiguousarray(tk["z"], np.float32)).to(dev),
        n=int(len(tk["offsets"]) - 1),
    )


def alloc_fit_out(n: int, device="cuda"):
    dev = torch.device(device)
    return dict(state=torch.empty((6, n), dtype=torch.float64, device=dev),
                cov=torch.empty((21, n), dtype=torch.float64, device=dev),
                chi2=torch.empty(n, dtype=torch.float64, device=dev),
                ndof=torch.empty(n, dtype=torch.int32, device=dev),
                status=torch.empty(n, dtype=torch.int32, device=dev))


def make_seeds(ctx, geom, dh, stream=None):
    n = dh["n"]
    st = torch.empty((6, n), dtype=torch.float32, device=dh["x"].device)
    q = torch.empty(n, dtype=torch.int8, device=dh["x"].device)
    kf.kf_make_seeds(ctx, geom, n, dh["offsets"], dh["x"], dh["y"], dh["z"], st, q, stream=stream)
    return st, q


def fit(ctx, geom, dh, seeds, out, precision=kf.KF_PREC_MIXED, n_fp64=3, ms_on=True,
        schedule=kf.KF_SCHED_GRID, stream=None, meas_model=kf.KF_MEAS_LAYER, seed_update=kf.KF_SEED_UD_DF):
    p = kf.fit_params(precision=precision, n_fp64_updates=n_fp64, ms_on=ms_on, schedule=schedule,
                      meas_model=meas_model, seed_update=seed_update)
    kf.kf_fit(ctx, geom, p, dh["n"], seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
              out["state"], out["cov"], out["chi2"], out["ndof"], out["status"], stream=stream)


def unpack_cov(cov21: np.ndarray) -> np.ndarray:
    """[21][n] packed lower triangles -> (n, 6, 6)."""
    n = cov21.shape[1]
    C = np.zeros((n, 6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            C[:, i, j] = cov21[k]
            C[:, j, i] = cov21[k]
            k += 1
    return C


def fit_numpy(ctx, geom, tk, precision=kf.KF_PREC_MIXED, n_fp64=3, ms_on=True, schedule=kf.KF_SCHED_GRID,
              meas_model=kf.KF_MEAS_LAYER, seed_update=kf.KF_SEED_UD_DF):
    """End to end on numpy CSR hits: seeds + fit on the GPU; numpy results (track-major)."""
    g = kf.make_geometry(geom)
    dh = hits_to_device(tk)
    seeds = make_seeds(ctx, g, dh)
    out = alloc_fit_out(dh["n"])
    fit(ctx, g, dh, seeds, out, precision=precision, n_fp64=n_fp64, ms_on=ms_on, schedule=schedule,
        meas_model=meas_model, seed_update=seed_update)
    torch.cuda.synchronize()
    return dict(seed=seeds[0].t().double().cpu().numpy(), q=seeds[1].cpu().numpy(),
                state=out["state"].t().cpu().numpy(), cov=unpack_cov(out["cov"].cpu().numpy()),
                chi2=out["chi2"].cpu().numpy(), ndof=out["ndof"].cpu().numpy(),
                status=out["status"].cpu().numpy().astype(np.uint32))


def bin_event(ctx, geom, ev, device="cuda", stream=None):
    """Upload one event's layers and bin every layer on the GPU (kf_bin_hits).
    Returns the layer dicts the binding's binned_layers() takes, plus perm."""
    dev = torch.device(device)
    out = []
    for ly in ev["layers"]:
        x = torch.from_numpy(np.ascontiguousarray(ly["x"], np.float32)).to(dev)
        y = torch.from_numpy(np.ascontiguousarray(ly["y"], np.float32)).to(dev)
        z = torch.from_numpy(np.ascontiguousarray(ly["z"], np.float32)).to(dev)
        n = int(x.numel())
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        offsets = torch.empty(kf.KF_NBINS + 1, dtype=torch.int32, device=dev)
        packed = torch.empty((max(n, 1), 4), dtype=torch.float32, device=dev)
        half = float(geom["surfaces"][ly["surf"]]["half_or_rin"])
        kf.kf_bin_hits(ctx, n, x, y, z, half, perm, offsets, packed, stream=stream)
        out.append(dict(n_hits=n, surface=int(ly["surf"]), packed=packed, offsets=offsets, perm=perm, x=x, y=y, z=z))
    return out


def seeds_from_seed_hits(ctx, geom, seed_hits_np, device="cuda", stream=None):
    """Seed estimate (kf_make_seeds) from each track's three seed hits; also returns the
    [9][n] device array of seed-hit coordinates kf_build_besthit takes."""
    sh = np.ascontiguousarray(seed_hits_np, np.float32).reshape(-1, 3, 3)
    n = sh.shape[0]
    tk = dict(offsets=(np.arange(n + 1) * 3).astype(np.int32), layer=np.zeros(3 * n, np.uint8),
              x=sh[:, :, 0].reshape(-1), y=sh[:, :, 1].reshape(-1), z=sh[:, :, 2].reshape(-1))
    dh = hits_to_device(tk, device)
    st, q = make_seeds(ctx, kf.make_geometry(geom), dh, stream=stream)
    sh9 = torch.from_numpy(np.ascontiguousarray(sh.reshape(n, 9).T)).to(torch.device(device))
    return st, q, sh9


def build_numpy(ctx, geom, events, precision=kf.KF_PREC_MIXED, warp_coop=False, nsigma=3.0, chi2_cut=30.0,
                max_cand=32, n_slots=0, meas_model=kf.KF_MEAS_LAYER, record_pred=False, cov_f32=False):
    """Bin every event's layers, seed, and run best-hit building of all events in one
    launch; returns numpy idx (n, n_layers) and fitted tracks (track-major).  record_pred
    (best-hit only): also 'pred' (n, n_layers, 27), each build step's predicted state and
    packed covariance (NaN where a track did not get to the layer).  cov_f32: also
    'cov32' ([21][n]), the FP32 covariance output."""
    g = kf.make_geometry(geom)
    binned = [bin_event(ctx, geom, ev) for ev in events]
    n_layers = len(events[0]["layers"])
    layers = kf.binned_layers([ly for b in binned for ly in b])
    counts = [ev["seed_hits"].shape[0] for ev in events]
    eoff = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    sh = np.concatenate([ev["seed_hits"].reshape(-1, 9) for ev in events])
    st, q, sh9 = seeds_from_seed_hits(ctx, geom, sh)
    n = int(eoff[-1])
    idx = torch.empty((n_layers, n), dtype=torch.int32, device="cuda")
    out = alloc_fit_out(n)
    c32 = torch.full((21, n), float("nan"), dtype=torch.float32, device="cuda") if cov_f32 else None
    if n_slots:  # combinatorial building with n_slots candidates per seed
        kf.kf_build_ckf(ctx, g, kf.fit_params(precision=precision, meas_model=meas_model),
                        kf.build_params(nsigma, chi2_cut, max_cand),
                        n_slots, len(events), n_layers, layers, eoff, st, q, sh9, idx, out["state"], out["cov"],
                        out["chi2"], out["ndof"], out["status"], out_cov_f32=c32)
    else:
        pred = torch.full((n_layers * 27 * n,), float("nan"), dtype=torch.float64, device="cuda") \
            if record_pred else None
        kf.kf_build_besthit(ctx, g, kf.fit_params(precision=precision, meas_model=meas_model),
                            kf.build_params(nsigma, chi2_cut, max_cand, warp_coop, debug_pred=pred),
                            len(events), n_layers, layers, eoff, st, q, sh9, idx, out["state"], out["cov"],
                            out["chi2"], out["ndof"], out["status"], out_cov_f32=c32)
    torch.cuda.synchronize()
    extra = {}
    if not n_slots and record_pred:
        extra["pred"] = pred.view(n_layers, 27, n).permute(2, 0, 1).cpu().numpy()
    if cov_f32:
        extra["cov32"], extra["cov64"] = c32.cpu().numpy(), out["cov"].cpu().numpy()
    return dict(extra, idx=idx.t().cpu().numpy(), state=out["state"].t().cpu().numpy(),
                cov=unpack_cov(out["cov"].cpu().numpy()), chi2=out["chi2"].cpu().numpy(),
                ndof=out["ndof"].cpu().numpy(), status=out["status"].cpu().numpy().astype(np.uint32),
                q=q.cpu().numpy(), binned=binned, layers=layers, eoff=eoff, sh9=sh9, idx_dev=idx)
