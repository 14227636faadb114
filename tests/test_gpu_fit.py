"""GPU parity of seeding and the Kalman-filter fit against the FP64 oracle, called
through the C ABI (libkf.so via the ctypes binding)."""
import numpy as np
import pytest
import torch

import parity
from paper_1711_06571_gb300 import kf, run, synth

pytestmark = pytest.mark.gpu

ST_BAD = kf.KF_ST_NO_INTERSECT | kf.KF_ST_CHOL_FAIL | kf.KF_ST_NONFINITE


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1711_06571_gb300 import build
    build.build()
    return run.context(0)


def _check_fit(tk, orc, gpu, geom, tol=parity.TOL_PARAM_SIGMA, label="", noise=None):
    np.testing.assert_array_equal(gpu["status"] & ST_BAD, orc["status"] & ST_BAD)
    np.testing.assert_array_equal(gpu["ndof"], orc["ndof"])
    ok = (orc["status"] & ST_BAD) == 0
    kinds = np.array([geom["surfaces"][s]["kind"] for s in parity.last_surface(tk, orc["ndof"])])
    res = parity.compare_fits(gpu, orc, kinds, ok)
    print(label, parity.summary(res))
    if noise is None:
        assert res["max_pull"].max() <= tol, parity.summary(res)
    else:
        # per-track bound: the stated tolerance, or 3x the oracle's own resolution where
        # that is coarser (reported)
        lim = np.maximum(tol, 3.0 * noise[ok])
        coarse = int(np.sum(3.0 * noise[ok] > tol))
        print(f"{label}: {coarse} of {ok.sum()} tracks where the oracle resolves the fit coarser than {tol}")
        assert coarse <= max(2, 0.002 * ok.sum())
        assert np.all(res["max_pull"] <= lim), parity.summary(res)
    assert res["chi2rel"].max() <= parity.TOL_CHI2_REL, parity.summary(res)
    assert res["dcov"].max() <= parity.TOL_COV_NORM, parity.summary(res)
    return res


def test_seed_parity(ctx, oracle_mod):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 1000, synth.BASE_SEED + 1)
    orc = oracle_mod.fit(g, tk)
    gg = kf.make_geometry(g)
    dh = run.hits_to_device(tk)
    st, q = run.make_seeds(ctx, gg, dh)
    torch.cuda.synchronize()
    st = st.t().double().cpu().numpy()
    q = q.cpu().numpy()
    so = orc["seed"]
    # FP32 closed form on FP32 inputs: position exact, angles to a few ulp of the
    # 3-point geometry; the curvature carries the conditioning of a 3-point circle
    # (sagitta ~ 1e-2 cm over 8 cm at 10 GeV), so compare q/pT absolutely, scaled
    np.testing.assert_array_equal(st[:, :3], so[:, :3])
    dphi = (st[:, 4] - so[:, 4] + np.pi) % (2 * np.pi) - np.pi
    assert np.abs(dphi).max() < 2e-5
    assert np.abs(st[:, 5] - so[:, 5]).max() < 2e-5
    qip_g, qip_o = q * st[:, 3], orc["q"] * so[:, 3]
    assert np.abs(qip_g - qip_o).max() < 2e-3 * np.maximum(1.0, np.abs(qip_o)).max()
    same_q = q == orc["q"]
    assert same_q.mean() > 0.99


def test_seed_hit_choice_at_the_2cm_threshold(ctx, oracle_mod):
    """The seed-hit rule (hits at least 2 cm apart, transverse) decided exactly as
    the oracle's FP64 test decides it, also for hits whose distance is within a
    few ulp of 2 cm (where the kernel's single-precision pre-test defers to FP64).
    The kernel's seeds from the whole track must equal its seeds from the three
    hits the oracle picks."""
    rng = np.random.default_rng(synth.BASE_SEED + 77)
    n, nh = 4096, 6
    x0, y0 = rng.uniform(-50, 50, n), rng.uniform(-50, 50, n)
    hx, hy, hz = np.zeros((n, nh), np.float32), np.zeros((n, nh), np.float32), np.zeros((n, nh), np.float32)
    hx[:, 0], hy[:, 0] = x0, y0
    for j in range(1, nh):
        # distances 2 cm * (1 + k * 2^-24), |k| <= 12: the float grid around the threshold
        d = 2.0 * (1.0 + rng.integers(-12, 13, n) * 2.0 ** -24)
        a = rng.uniform(-np.pi, np.pi, n)
        hx[:, j], hy[:, j] = x0 + d * np.cos(a), y0 + d * np.sin(a)
    hz[:] = 0.7 * np.arange(nh, dtype=np.float32)
    d2 = (hx[:, 1].astype(np.float64) - hx[:, 0]) ** 2 + (hy[:, 1].astype(np.float64) - hy[:, 0]) ** 2
    assert np.sum(np.abs(d2 / 4.0 - 1.0) < 1e-6) > n // 2  # most first distances are in the FP64 band
    picks = np.array([oracle_mod.seed_hits(hx[t], hy[t]) for t in range(n)])
    assert len(set(map(tuple, picks[:, 1:]))) > 3  # the rule picks several different hit pairs
    g = kf.make_geometry(synth.geometry("barrel10"))
    full = run.hits_to_device(dict(offsets=(np.arange(n + 1) * nh).astype(np.int32), layer=np.zeros(n * nh, np.uint8),
                                   x=hx.reshape(-1), y=hy.reshape(-1), z=hz.reshape(-1)))
    rows = np.arange(n)[:, None]
    three = run.hits_to_device(dict(offsets=(np.arange(n + 1) * 3).astype(np.int32), layer=np.zeros(n * 3, np.uint8),
                                    x=hx[rows, picks].reshape(-1), y=hy[rows, picks].reshape(-1),
                                    z=hz[rows, picks].reshape(-1)))
    st_a, q_a = run.make_seeds(ctx, g, full)
    st_b, q_b = run.make_seeds(ctx, g, three)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st_a.cpu().numpy(), st_b.cpu().numpy())
    np.testing.assert_array_equal(q_a.cpu().numpy(), q_b.cpu().numpy())


@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
def test_fit_parity_1000_tracks_10_layers(ctx, oracle_mod, precision):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 1000, synth.BASE_SEED + 1)
    orc = oracle_mod.fit(g, tk)
    gpu = run.fit_numpy(ctx, g, tk, precision=precision)
    res = _check_fit(tk, orc, gpu, g, label=f"barrel10 prec={precision}")
    if precision == kf.KF_PREC_FP64:
        # both GPU paths start from the FP32 seed estimate; the rest is FP64
        assert res["max_pull"].max() < 1e-4


@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
def test_fit_parity_17_layers_ragged(ctx, oracle_mod, precision):
    # 17 layers up to 100 cm: a few percent of tracks curl before the last layers
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 3000, synth.BASE_SEED + 2)
    nh = np.diff(tk["offsets"])
    assert nh.min() < 17 <= nh.max()
    orc = oracle_mod.fit(g, tk)
    gpu = run.fit_numpy(ctx, g, tk, precision=precision)
    _check_fit(tk, orc, gpu, g, label=f"barrel17 prec={precision}")


@pytest.mark.parametrize("precision,seed_update", [(kf.KF_PREC_MIXED, kf.KF_SEED_UD_DF),
                                                   (kf.KF_PREC_MIXED, kf.KF_SEED_JOSEPH_FP64),
                                                   (kf.KF_PREC_FP64, kf.KF_SEED_UD_DF)])
def test_fit_parity_cylinder_with_lids(ctx, oracle_mod, precision, seed_update):
    """The barrel closed by end-cap disks (Sec. 4.1), |eta| < 2.5, 20,000 tracks: every
    track within max(1e-3 sigma, 3 x the oracle's own resolution), tracks that cross a
    layer twice in a row fitted in FP64 (KF_ST_FP64_TRACK), tracks whose theta left
    (0, pi) ended with KF_ST_THETA_RANGE on both sides."""
    g = synth.geometry("lids")
    tk = synth.gen_tracks(g, 20000, synth.BASE_SEED + 4, eta_max=2.5, min_hits=4)
    orc = oracle_mod.fit(g, tk, threads=4)
    kinds = np.array([g["surfaces"][s]["kind"] for s in parity.last_surface(tk, orc["ndof"])])
    noise = parity.oracle_self_noise(oracle_mod, g, tk, orc, kinds)
    gpu = run.fit_numpy(ctx, g, tk, precision=precision, seed_update=seed_update)
    np.testing.assert_array_equal(gpu["status"] & kf.KF_ST_THETA_RANGE, orc["status"] & kf.KF_ST_THETA_RANGE)
    off = tk["offsets"]
    recross = np.array([np.any(tk["layer"][off[t] + 1:off[t + 1]] == tk["layer"][off[t]:off[t + 1] - 1])
                        for t in range(tk["n"])])
    if precision == kf.KF_PREC_MIXED:
        np.testing.assert_array_equal((gpu["status"] & kf.KF_ST_FP64_TRACK) != 0, recross)
    print(f"lids: {recross.sum()} tracks cross a layer twice in a row, "
          f"{np.sum((orc['status'] & kf.KF_ST_THETA_RANGE) != 0)} leave (0, pi)")
    _check_fit(tk, orc, gpu, g, label=f"lids prec={precision} seed={seed_update}", noise=noise)


def test_fit_parity_uneven_batch_persistent_sampled(ctx, oracle_mod):
    """The uneven batch at its own size: 2,000,000 barrel+disk tracks (4 to 26 hits)
    in the autotuned persistent launch replayed as a CUDA graph, as the benchmark
    times it; the oracle checks a sample of 2,000 tracks with the bound of the
    barrel+disk test."""
    g = synth.geometry("lids")
    gg = kf.make_geometry(g)
    tkd = synth.gen_tracks(g, 2_000_000, synth.BASE_SEED + 4, eta_max=2.5, min_hits=4, device="cuda")
    n = tkd["n"]
    dh = run.hits_to_device(tkd)
    seeds = run.make_seeds(ctx, gg, dh)
    out = run.alloc_fit_out(n)
    p = kf.fit_params(schedule=kf.KF_SCHED_PERSISTENT)
    kf.kf_autotune_fit(ctx, gg, p, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                       out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
    for _ in range(2):  # graph capture, then a replay
        kf.kf_fit(ctx, gg, p, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                  out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
    torch.cuda.synchronize()
    tk = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in tkd.items()}
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, 2000, replace=False))
    off = tk["offsets"]
    rows = np.concatenate([np.arange(off[t], off[t + 1]) for t in idx])
    sub = dict(offsets=np.concatenate([[0], np.cumsum(np.diff(off)[idx])]).astype(np.int32),
               layer=tk["layer"][rows], x=tk["x"][rows], y=tk["y"][rows], z=tk["z"][rows], n=len(idx))
    orc = oracle_mod.fit(g, sub, threads=4)
    kinds = np.array([g["surfaces"][s]["kind"] for s in parity.last_surface(sub, orc["ndof"])])
    noise = parity.oracle_self_noise(oracle_mod, g, sub, orc, kinds)
    gpu = dict(seed=seeds[0].t().double().cpu().numpy()[idx], q=seeds[1].cpu().numpy()[idx],
               state=out["state"].t().cpu().numpy()[idx], cov=run.unpack_cov(out["cov"][:, idx].cpu().numpy()),
               chi2=out["chi2"].cpu().numpy()[idx], ndof=out["ndof"].cpu().numpy()[idx],
               status=out["status"].cpu().numpy().astype(np.uint32)[idx])
    _check_fit(sub, orc, gpu, g, label="uneven 2e6 persistent sampled", noise=noise)


@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
def test_fit_parity_hit_2d_staggered(ctx, oracle_mod, precision):
    """Measurement model 1 (Sec. 4.1) on the staggered 17-layer barrel: every
    barrel hit reached on the cylinder through it and updated in 2-D there."""
    g = synth.geometry("barrel17s")
    tk = synth.gen_tracks(g, 3000, synth.BASE_SEED + 21)
    orc = oracle_mod.fit(g, tk, meas_model=1)
    gpu = run.fit_numpy(ctx, g, tk, precision=precision, meas_model=kf.KF_MEAS_HIT_2D)
    _check_fit(tk, orc, gpu, g, label=f"barrel17s model 1 prec={precision}")


def test_hit_2d_rejected_where_unsupported(ctx):
    g = synth.geometry("barrel17s")
    tk = synth.gen_tracks(g, 100, synth.BASE_SEED + 22)
    with pytest.raises(kf.KfError):
        run.fit_numpy(ctx, g, tk, schedule=kf.KF_SCHED_PERSISTENT, meas_model=kf.KF_MEAS_HIT_2D)
    with pytest.raises(kf.KfError):
        run.fit_numpy(ctx, g, tk, meas_model=2)


def _host_fit(ctx, g, tk, n_chunks, pinned, meas_model=kf.KF_MEAS_LAYER):
    n = tk["n"]

    def buf(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.pin_memory() if pinned else t
    hh = {k: buf(tk[k]) for k in ("offsets", "layer", "x", "y", "z")}
    out = dict(state=np.full((6, n), np.nan), cov=np.full((21, n), np.nan), chi2=np.full(n, np.nan),
               ndof=np.full(n, -99, np.int32), status=np.full(n, 0xffff, np.uint32))
    if pinned:
        out = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in out.items()}
    kf.kf_fit_host(ctx, kf.make_geometry(g), kf.fit_params(meas_model=meas_model), n, hh["offsets"], hh["layer"],
                   hh["x"], hh["y"], hh["z"], out["state"], out["cov"], out["chi2"], out["ndof"], out["status"],
                   n_chunks=n_chunks)
    return out


def test_fit_host_matches_device_path(ctx):
    """kf_fit_host (host buffers in and out, the tracks split into ranges on three
    streams, the first and last ranges half size) returns exactly what the device
    path returns, for any number of ranges, page-locked or pageable buffers."""
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 70001, synth.BASE_SEED + 23)
    gg = kf.make_geometry(g)
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, gg, dh)
    ref = run.alloc_fit_out(dh["n"])
    run.fit(ctx, gg, dh, seeds, ref)
    torch.cuda.synchronize()
    ref = dict(state=ref["state"].cpu().numpy(), cov=ref["cov"].cpu().numpy(), chi2=ref["chi2"].cpu().numpy(),
               ndof=ref["ndof"].cpu().numpy(), status=ref["status"].cpu().numpy().astype(np.uint32))
    for n_chunks, pinned in ((0, True), (1, True), (2, False), (3, True), (7, True), (64, False)):
        got = _host_fit(ctx, g, tk, n_chunks, pinned)
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{k} n_chunks={n_chunks} pinned={pinned}")


def test_fp32_covariance_output(ctx):
    """kf_tracks_out.cov_f32: the covariance in FP32 storage, beside or instead of
    the FP64 one, from kf_fit (both precisions, both schedules), kf_fit_host,
    kf_refit_inward and best-hit and combinatorial building -- each entry the FP64
    output rounded to FP32 (the same value rounded once), and the other outputs
    unchanged when only cov_f32 is asked for."""
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 20001, synth.BASE_SEED + 27)
    gg = kf.make_geometry(g)
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, gg, dh)
    n = dh["n"]
    for precision in (kf.KF_PREC_MIXED, kf.KF_PREC_FP64):
        for schedule in (kf.KF_SCHED_GRID, kf.KF_SCHED_PERSISTENT):
            p = kf.fit_params(precision=precision, schedule=schedule)
            ref = run.alloc_fit_out(n)
            c32 = torch.full((21, n), float("nan"), dtype=torch.float32, device="cuda")
            kf.kf_fit(ctx, gg, p, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                      ref["state"], ref["cov"], ref["chi2"], ref["ndof"], ref["status"], out_cov_f32=c32)
            alone = run.alloc_fit_out(n)
            c32b = torch.full((21, n), float("nan"), dtype=torch.float32, device="cuda")
            kf.kf_fit(ctx, gg, p, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                      alone["state"], None, alone["chi2"], alone["ndof"], alone["status"], out_cov_f32=c32b)
            torch.cuda.synchronize()
            want = ref["cov"].cpu().numpy().astype(np.float32)
            np.testing.assert_array_equal(c32.cpu().numpy(), want, err_msg=f"prec={precision} sched={schedule}")
            np.testing.assert_array_equal(c32b.cpu().numpy(), want)
            for k in ("state", "chi2", "ndof", "status"):
                assert torch.equal(alone[k], ref[k]), k
    # host path: FP32 covariance only, and both
    ref = run.alloc_fit_out(n)
    run.fit(ctx, gg, dh, seeds, ref)
    torch.cuda.synchronize()
    want = ref["cov"].cpu().numpy().astype(np.float32)
    hh = {k: torch.from_numpy(np.ascontiguousarray(tk[k])).pin_memory() for k in ("offsets", "layer", "x", "y", "z")}
    for with64 in (False, True):
        c32 = torch.full((21, n), float("nan"), dtype=torch.float32).pin_memory()
        c64 = torch.full((21, n), float("nan"), dtype=torch.float64).pin_memory() if with64 else None
        st = torch.full((6, n), float("nan"), dtype=torch.float64).pin_memory()
        kf.kf_fit_host(ctx, gg, None, n, hh["offsets"], hh["layer"], hh["x"], hh["y"], hh["z"], st, c64,
                       out_cov_f32=c32, n_chunks=5)
        np.testing.assert_array_equal(c32.numpy(), want)
        np.testing.assert_array_equal(st.numpy(), ref["state"].cpu().numpy())
        if with64:
            np.testing.assert_array_equal(c64.numpy(), ref["cov"].cpu().numpy())
    # refit (its output turned back to the outward direction in both planes)
    bw = run.alloc_fit_out(n)
    c32 = torch.full((21, n), float("nan"), dtype=torch.float32, device="cuda")
    kf.kf_refit_inward(ctx, gg, None, n, dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"], ref["state"],
                       ref["cov"], seeds[1], ref["ndof"], 100.0, bw["state"], bw["cov"], bw["chi2"], bw["ndof"],
                       bw["status"], out_cov_f32=c32)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c32.cpu().numpy(), bw["cov"].cpu().numpy().astype(np.float32))
    # building
    ev = synth.gen_event(g, 2000, synth.BASE_SEED + 28)
    for n_slots in (0, 4):
        b = run.build_numpy(ctx, g, [ev], n_slots=n_slots, cov_f32=True)
        np.testing.assert_array_equal(b["cov32"], b["cov64"].astype(np.float32), err_msg=f"n_slots={n_slots}")


def test_fit_host_concurrent_calls_on_one_context(ctx):
    """kf_fit_host from two host threads on one context: the calls share the
    context's device buffers and streams, so the library runs them one at a time,
    and each returns what it returns alone (the larger batch regrows the buffers
    in between)."""
    import threading
    g = synth.geometry("barrel17")
    tks = [synth.gen_tracks(g, n, synth.BASE_SEED + 25 + i) for i, n in enumerate((40000, 65537))]
    alone = [_host_fit(ctx, g, tk, 0, True) for tk in tks]
    got = [[None] * 3 for _ in tks]
    errors = []

    def worker(i):
        try:
            for r in range(3):
                got[i][r] = _host_fit(ctx, g, tks[i], 0, True)
        except Exception as e:  # reported below, in the test's own thread
            errors.append(e)
    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(tks))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    assert not any(t.is_alive() for t in threads)
    for i in range(len(tks)):
        for r in range(3):
            for k in alone[i]:
                np.testing.assert_array_equal(got[i][r][k], alone[i][k], err_msg=f"{k} thread {i} call {r}")


def test_fit_host_small_and_bad_arguments(ctx):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 5, synth.BASE_SEED + 24)
    a = _host_fit(ctx, g, tk, 0, False)
    b = _host_fit(ctx, g, tk, 64, False)  # more ranges than tracks: one track per range
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert np.all(a["ndof"] > 0)
    with pytest.raises(kf.KfError):
        _host_fit(ctx, g, tk, 65, False)
    dh = run.hits_to_device(tk)
    with pytest.raises(ValueError):  # device memory where host memory is required
        kf.kf_fit_host(ctx, kf.make_geometry(g), None, tk["n"], dh["offsets"], dh["layer"], dh["x"], dh["y"],
                       dh["z"])


def test_persistent_schedule_matches_grid(ctx):
    g = synth.geometry("lids")
    tk = synth.gen_tracks(g, 20000, synth.BASE_SEED + 5, eta_max=2.5, min_hits=4)
    a = run.fit_numpy(ctx, g, tk, schedule=kf.KF_SCHED_GRID)
    b = run.fit_numpy(ctx, g, tk, schedule=kf.KF_SCHED_PERSISTENT)
    c = run.fit_numpy(ctx, g, tk, schedule=kf.KF_SCHED_PERSISTENT)  # graph replay
    for k in ("state", "cov", "chi2", "ndof", "status"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])


def test_fit_edge_cases(ctx, oracle_mod):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 64, synth.BASE_SEED + 6)
    # ragged: cut tracks to 0, 1, 2, 3 hits and keep the rest whole
    off = tk["offsets"]
    keep = []
    newoff = [0]
    for t in range(tk["n"]):
        nh = off[t + 1] - off[t]
        m = [0, 1, 2, 3, nh][t % 5]
        keep.extend(range(off[t], off[t] + m))
        newoff.append(newoff[-1] + m)
    keep = np.array(keep, int)
    tk2 = dict(offsets=np.array(newoff, np.int32), layer=tk["layer"][keep], x=tk["x"][keep], y=tk["y"][keep],
               z=tk["z"][keep], n=tk["n"])
    gpu = run.fit_numpy(ctx, g, tk2)
    nh = np.diff(tk2["offsets"])
    # tracks with >= 3 hits: parity with the oracle fed the GPU path's own inputs rule
    orc = oracle_mod.fit(g, tk2)
    sel = nh >= 3
    assert np.all(gpu["ndof"][sel] == 2 * nh[sel] - 5)
    np.testing.assert_array_equal(gpu["ndof"][sel], orc["ndof"][sel])
    # tracks with no hit: the seed comes back untouched with its covariance
    z0 = nh == 0
    assert np.all(gpu["ndof"][z0] == -5)
    assert np.allclose(gpu["cov"][z0][:, np.arange(6), np.arange(6)], 1e4)
    # n = 0 is a no-op
    e = run.alloc_fit_out(0)
    empty = run.hits_to_device(dict(offsets=np.zeros(1, np.int32), layer=np.zeros(0, np.uint8),
                                    x=np.zeros(0, np.float32), y=np.zeros(0, np.float32), z=np.zeros(0, np.float32)))
    kf.kf_fit(ctx, kf.make_geometry(g), None, 0, torch.empty((6, 0), device="cuda"),
              torch.empty(0, dtype=torch.int8, device="cuda"), empty["offsets"], empty["layer"], empty["x"],
              empty["y"], empty["z"], e["state"], e["cov"], e["chi2"], e["ndof"], e["status"])


def test_fit_rejects_host_pointers(ctx):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 10, 1)
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, kf.make_geometry(g), dh)
    out = run.alloc_fit_out(dh["n"])
    host_x = dh["x"].cpu()
    with pytest.raises(kf.KfError) as ei:
        kf.kf_fit(ctx, kf.make_geometry(g), None, dh["n"], seeds[0], seeds[1], dh["offsets"], dh["layer"], host_x,
                  dh["y"], dh["z"], out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
    assert ei.value.code == kf.KF_EINVAL
    with pytest.raises(kf.KfError):
        kf.kf_fit(ctx, kf.make_geometry(g), kf.fit_params(precision=7), dh["n"], seeds[0], seeds[1],
                  dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"])


def test_fit_rejects_misaligned_device_pointers(ctx):
    """Device arrays must sit at a multiple of their element size (the kernels
    load and store whole elements, and a misaligned access faults the GPU): the
    entry points refuse them with KF_EINVAL before anything is launched.  The
    misaligned pointers are byte views a few bytes into device buffers."""
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 10, 1)
    dh = run.hits_to_device(tk)
    n = dh["n"]
    seeds = run.make_seeds(ctx, kf.make_geometry(g), dh)
    out = run.alloc_fit_out(n)
    state_buf = torch.empty(48 * n + 8, dtype=torch.uint8, device="cuda")
    x_buf = torch.empty(dh["x"].numel() * 4 + 4, dtype=torch.uint8, device="cuda")
    for bad in (dict(out_state=state_buf[4:4 + 48 * n]), dict(x=x_buf[2:2 + 4 * dh["x"].numel()])):
        args = dict(x=dh["x"], out_state=out["state"])
        args.update(bad)
        with pytest.raises(kf.KfError) as ei:
            kf.kf_fit(ctx, kf.make_geometry(g), None, n, seeds[0], seeds[1], dh["offsets"], dh["layer"],
                      args["x"], dh["y"], dh["z"], args["out_state"], out["cov"], out["chi2"], out["ndof"],
                      out["status"])
        assert ei.value.code == kf.KF_EINVAL and "aligned" in str(ei.value)
    # packed hits are read as 16-byte vectors: an 8-byte aligned packed_out is refused
    h = 64
    hx = torch.zeros(h, device="cuda")
    perm = torch.empty(h, dtype=torch.int32, device="cuda")
    offs = torch.empty(kf.KF_NBINS + 1, dtype=torch.int32, device="cuda")
    pk_buf = torch.empty(16 * h + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(kf.KfError) as ei:
        kf.kf_bin_hits(ctx, h, hx, hx, hx, 40.0, perm, offs, pk_buf[8:8 + 16 * h])
    assert ei.value.code == kf.KF_EINVAL
    # the same calls with aligned arrays still run
    kf.kf_fit(ctx, kf.make_geometry(g), None, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"],
              dh["y"], dh["z"], out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
    kf.kf_bin_hits(ctx, h, hx, hx, hx, 40.0, perm, offs, pk_buf[:16 * h])
    torch.cuda.synchronize()
    assert torch.isfinite(out["state"]).all()


def test_fit_parity_million_tracks_sampled(ctx, oracle_mod):
    """The full 1,000,000-track, 17-layer workload on the GPU, in the launch the
    benchmark times; the oracle checks a sample of 2,000 tracks."""
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 1_000_000, synth.BASE_SEED + 2)
    gpu = run.fit_numpy(ctx, g, tk)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(tk["n"], 2000, replace=False))
    off = tk["offsets"]
    rows = np.concatenate([np.arange(off[t], off[t + 1]) for t in idx])
    sub = dict(offsets=np.concatenate([[0], np.cumsum(np.diff(off)[idx])]).astype(np.int32),
               layer=tk["layer"][rows], x=tk["x"][rows], y=tk["y"][rows], z=tk["z"][rows], n=len(idx))
    orc = oracle_mod.fit(g, sub)
    gsub = {k: (v[idx] if isinstance(v, np.ndarray) and len(v) == tk["n"] else v) for k, v in gpu.items()}
    _check_fit(sub, orc, gsub, g, label="1e6 sampled")
    # every track: finite, status clean except the documented ones
    bad = (gpu["status"] & ST_BAD) != 0
    assert bad.mean() < 1e-3


def _gpu_fit_and_refit(ctx, g, tk, precision, meas_model=kf.KF_MEAS_LAYER):
    gg = kf.make_geometry(g)
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, gg, dh)
    fw = run.alloc_fit_out(dh["n"])
    run.fit(ctx, gg, dh, seeds, fw, precision=precision, meas_model=meas_model)
    bw = run.alloc_fit_out(dh["n"])
    kf.kf_refit_inward(ctx, gg, kf.fit_params(precision=precision, meas_model=meas_model), dh["n"], dh["offsets"], dh["layer"], dh["x"],
                       dh["y"], dh["z"], fw["state"], fw["cov"], seeds[1], fw["ndof"], 100.0, bw["state"],
                       bw["cov"], bw["chi2"], bw["ndof"], bw["status"])
    torch.cuda.synchronize()
    return dict(state=bw["state"].t().cpu().numpy(), cov=run.unpack_cov(bw["cov"].cpu().numpy()),
                chi2=bw["chi2"].cpu().numpy(), ndof=bw["ndof"].cpu().numpy(),
                status=bw["status"].cpu().numpy().astype(np.uint32), q=seeds[1].cpu().numpy())


@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
@pytest.mark.parametrize("name", ["barrel10", "barrel17", "barrel17s"])
def test_refit_inward_parity(ctx, oracle_mod, name, precision):
    """Outward-inward refit: the state and covariance at the first hit, the chi2
    and ndof of the backward pass, against the oracle's refit (each side seeded
    with its own forward fit).  The staggered barrel runs measurement model 1
    both ways."""
    g = synth.geometry(name)
    model = 1 if name == "barrel17s" else 0
    tk = synth.gen_tracks(g, 3000, synth.BASE_SEED + 12)
    fw = oracle_mod.fit(g, tk, meas_model=model)
    orc = oracle_mod.refit_inward(g, tk, fw["state"], fw["cov"], fw["q"], fw["ndof"], meas_model=model)
    orc["q"] = fw["q"]
    gpu = _gpu_fit_and_refit(ctx, g, tk, precision, meas_model=model)
    diff = np.nonzero((gpu["status"] & ST_BAD) != (orc["status"] & ST_BAD))[0]
    assert len(diff) == 0, [(int(t), int(gpu["status"][t]), int(orc["status"][t]), int(gpu["ndof"][t]),
                             int(orc["ndof"][t]), int(fw["ndof"][t]), int(fw["status"][t]),
                             tk["offsets"][t + 1] - tk["offsets"][t], fw["state"][t].tolist()) for t in diff[:4]]
    np.testing.assert_array_equal(gpu["ndof"], orc["ndof"])
    ok = ((orc["status"] & ST_BAD) == 0) & (gpu["q"] == orc["q"])
    res = parity.compare_fits(gpu, orc, np.zeros(tk["n"], int), ok)
    print(f"refit {name} prec={precision}:", parity.summary(res))
    assert ok.mean() > 0.99
    assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
    assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
    assert res["dcov"].max() <= parity.TOL_COV_NORM


def _to_layout(a, layout):
    """(n, K) matrices -> the flat array of a layout (see kf_layout_transport)."""
    n, K = a.shape
    if layout == kf.KF_LAYOUT_AOS:
        return np.ascontiguousarray(a).reshape(-1)
    if layout == kf.KF_LAYOUT_SOA:
        return np.ascontiguousarray(a.T).reshape(-1)
    return np.ascontiguousarray(a.reshape(n // 32, 32, K).transpose(0, 2, 1)).reshape(-1)


def _from_layout(f, n, K, layout):
    if layout == kf.KF_LAYOUT_AOS:
        return f.reshape(n, K)
    if layout == kf.KF_LAYOUT_SOA:
        return f.reshape(K, n).T
    return f.reshape(n // 32, K, 32).transpose(0, 2, 1).reshape(n, K)


def test_layout_transport_matches_oracle(ctx, oracle_mod):
    """The layout study's kernel computes J P J^T in every layout; checked against
    the oracle's dense FP64 transport."""
    rng = np.random.default_rng(5)
    n = 4096
    J = rng.normal(size=(n, 36)).astype(np.float32)
    A = rng.normal(size=(n, 6, 6))
    P6 = A @ A.transpose(0, 2, 1)
    tril = np.tril_indices(6)
    P = P6[:, tril[0], tril[1]].astype(np.float32)
    ref = np.zeros((n, 21))
    for t in range(0, n, 97):
        Pn = oracle_mod.transport(J[t].astype(np.float64), P6[t].astype(np.float32).astype(np.float64).reshape(36))
        ref[t] = Pn.reshape(6, 6)[tril]
    outs = []
    for layout in (kf.KF_LAYOUT_AOS, kf.KF_LAYOUT_SOA, kf.KF_LAYOUT_BLOCK):
        dJ = torch.from_numpy(_to_layout(J, layout)).cuda()
        dP = torch.from_numpy(_to_layout(P, layout)).cuda()
        dO = torch.empty(n * 21, dtype=torch.float32, device="cuda")
        kf.kf_layout_transport(ctx, layout, n, dJ, dP, dO)
        torch.cuda.synchronize()
        outs.append(_from_layout(dO.cpu().numpy(), n, 21, layout))
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    sel = np.arange(0, n, 97)
    scale = np.abs(ref[sel]).max(axis=1, keepdims=True)
    assert np.max(np.abs(outs[0][sel] - ref[sel]) / scale) < 1e-5
