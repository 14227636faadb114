"""GPU parity of hit binning (bit-exact) and best-hit building against the FP64
oracle, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import parity
from paper_1711_06571_gb300 import kf, run, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1711_06571_gb300 import build
    build.build()
    return run.context(0)


def _bin_gpu(ctx, x, y, z, half):
    dev = torch.device("cuda")
    n = len(x)
    xt, yt, zt = (torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in (x, y, z))
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    off = torch.empty(kf.KF_NBINS + 1, dtype=torch.int32, device=dev)
    packed = torch.empty((max(n, 1), 4), dtype=torch.float32, device=dev)
    kf.kf_bin_hits(ctx, n, xt, yt, zt, half, perm, off, packed)
    torch.cuda.synchronize()
    return perm.cpu().numpy()[:n], off.cpu().numpy(), packed.cpu().numpy()[:n]


def _edge_allowed(oracle_mod, x, y, z, half, perm_g, perm_o):
    """Positions where the binned orders differ must be hits whose key lies within a few
    ulps of a bin edge (atan2 differs between libraries by an ulp at most)."""
    bad = np.nonzero(perm_g != perm_o)[0]
    for p in bad:
        for i in (perm_g[p], perm_o[p]):
            u = ((math.atan2(float(y[i]), float(x[i])) + math.pi) * 1024.0) / (2 * math.pi)
            if abs(u - round(u)) > 1e-9:
                return False
    return True


def test_binning_bit_exact_event(ctx, oracle_mod):
    g = synth.geometry("barrel17")
    ev = synth.gen_event(g, 20000, synth.BASE_SEED + 3)
    for ly in ev["layers"]:
        half = g["surfaces"][ly["surf"]]["half_or_rin"]
        pg, og, pk = _bin_gpu(ctx, ly["x"], ly["y"], ly["z"], half)
        po, oo = oracle_mod.bin_layer(ly["x"], ly["y"], ly["z"], half)
        np.testing.assert_array_equal(og, oo)
        if not np.array_equal(pg, po):
            assert _edge_allowed(oracle_mod, ly["x"], ly["y"], ly["z"], half, pg, po)
        # packed records are the hits in binned order with their original index
        np.testing.assert_array_equal(pk[:, 3].view(np.int32), pg)
        np.testing.assert_array_equal(pk[:, 0], ly["x"][pg])


def test_binning_edge_cases(ctx, oracle_mod):
    half = 40.0
    rng = np.random.default_rng(3)
    cases = []
    # empty layer
    cases.append((np.zeros(0, np.float32),) * 3)
    # every hit in one bin (stability over a long run of equal keys), odd size
    n = 5000 + 17
    cases.append((np.full(n, 20.0, np.float32), np.full(n, 0.001, np.float32), np.full(n, 1.0, np.float32)))
    # phi exactly +-pi, on the axes, z outside the layer and on its edges
    x = np.array([-20, -20, 20, 0, 0, -1e-30, 20, 20, 20], np.float32)
    y = np.array([0, -0.0, 0, 20, -20, 0, 1, 1, 1], np.float32)
    z = np.array([0, 0, 0, 0, 0, 0, -half, half, 1e6], np.float32)
    cases.append((x, y, z))
    # many hits, crowded into a few bins
    ph = rng.choice(np.linspace(-3, 3, 7), 70000)
    cases.append(((30 * np.cos(ph)).astype(np.float32), (30 * np.sin(ph)).astype(np.float32),
                  rng.choice([-5.0, 0.0, 5.0], 70000).astype(np.float32)))
    for x, y, z in cases:
        pg, og, _ = _bin_gpu(ctx, x, y, z, half)
        po, oo = oracle_mod.bin_layer(x, y, z, half)
        np.testing.assert_array_equal(og, oo)
        np.testing.assert_array_equal(pg, po)


def test_binning_at_bin_edges(ctx, oracle_mod):
    """Hits placed on and next to phi and z bin edges (where a single-precision
    estimate of the key cannot decide and the FP64 evaluation takes over): keys
    and order equal the oracle's."""
    half = 36.4
    rng = np.random.default_rng(11)
    k = rng.integers(0, 1024, 3000)
    d = rng.choice([0.0, 1e-9, -1e-9, 1e-7, -1e-7, 3e-6, -3e-6, 2e-5, -2e-5, 1e-4, -1e-4, 4e-3, -4e-3], 3000)
    phi = -np.pi + 2 * np.pi * (k + d) / 1024.0
    r = rng.uniform(4.0, 100.0, 3000)
    kz = rng.integers(0, 65, 3000)
    dz = rng.choice([0.0, 1e-6, -1e-6, 1e-4, -1e-4, 2e-3, -2e-3], 3000)
    z = (-half + 2 * half * (kz + dz) / 64.0)
    x, y = (r * np.cos(phi)).astype(np.float32), (r * np.sin(phi)).astype(np.float32)
    z = z.astype(np.float32)
    pg, og, _ = _bin_gpu(ctx, x, y, z, half)
    po, oo = oracle_mod.bin_layer(x, y, z, half)
    if not np.array_equal(og, oo) or not np.array_equal(pg, po):
        # only an atan2 ulp at an exact phi edge may differ between libraries
        assert _edge_allowed(oracle_mod, x, y, z, half, pg, po)


def test_batched_binning_equals_per_layer(ctx, oracle_mod):
    """kf_bin_hits_batched over every layer of two events plus the edge cases
    (empty segments included) gives, per segment, exactly the per-layer call's
    results, and the per-layer call equals the oracle on these inputs."""
    g = synth.geometry("barrel17")
    segs = []
    for e in range(2):
        ev = synth.gen_event(g, 3000 + 1700 * e, synth.BASE_SEED + 13 + e)
        segs += [(ly["x"], ly["y"], ly["z"], g["surfaces"][ly["surf"]]["half_or_rin"]) for ly in ev["layers"]]
    z0 = np.zeros(0, np.float32)
    segs.insert(5, (z0, z0, z0, 12.5))
    segs.append((np.full(999, 20.0, np.float32), np.full(999, 0.001, np.float32), np.ones(999, np.float32), 40.0))
    segs.append((z0, z0, z0, 3.0))
    sizes = [len(s[0]) for s in segs]
    so = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    H, ns = int(so[-1]), len(segs)
    dev = torch.device("cuda")
    xt, yt, zt = (torch.from_numpy(np.concatenate([s[k] for s in segs]).astype(np.float32)).to(dev) for k in range(3))
    perm = torch.empty(H, dtype=torch.int32, device=dev)
    off = torch.full((ns, kf.KF_NBINS + 1), -5, dtype=torch.int32, device=dev)
    packed = torch.empty((H, 4), dtype=torch.float32, device=dev)
    kf.kf_bin_hits_batched(ctx, so, [s[3] for s in segs], xt, yt, zt, perm, off, packed)
    torch.cuda.synchronize()
    perm_h, off_h, pk_h = perm.cpu().numpy(), off.cpu().numpy(), packed.cpu().numpy()
    for i, (x, y, z, half) in enumerate(segs):
        a, b = so[i], so[i + 1]
        pg, og, pkg = _bin_gpu(ctx, x, y, z, half)
        np.testing.assert_array_equal(off_h[i], og)
        np.testing.assert_array_equal(perm_h[a:b], pg)
        np.testing.assert_array_equal(pk_h[a:b].view(np.int32), pkg.view(np.int32))
        if i in (0, 5, ns - 2):
            po, oo = oracle_mod.bin_layer(x, y, z, half)
            np.testing.assert_array_equal(og, oo)
    with pytest.raises(kf.KfError):
        kf.kf_bin_hits_batched(ctx, [0, 3, 2], [1.0, 1.0], xt, yt, zt, perm, off, packed)
    with pytest.raises(kf.KfError):
        kf.kf_bin_hits_batched(ctx, [0, 3], [0.0], xt, yt, zt, perm, off, packed)


# ------------------------------------------------------------------ building

def _binned_oracle_event(oracle_mod, g, ev):
    for ly in ev["layers"]:
        half = g["surfaces"][ly["surf"]]["half_or_rin"]
        ly["perm"], ly["offsets"] = oracle_mod.bin_layer(ly["x"], ly["y"], ly["z"], half)
    return ev


def _unpack21(v):
    P = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            P[i, j] = P[j, i] = v[k]
            k += 1
    return P


def _window_bins(r):
    """(phi bin, z bin) set of a step record's window"""
    phis = {(r["phi_lo"] + k) % 1024 for k in range(r["phi_n"])}
    return {(pb, zb) for zb in range(r["z_lo"], r["z_hi"] + 1) for pb in phis}


def classify_build(oracle_mod, g, ev, orc, gidx, gpred, gq, t_sel=None, meas_model=0, cut=30.0):
    """Per track, compare hit indices layer by layer up to the first difference.  The GPU
    predicts in FP32 and the oracle in FP64, so a decision that sits on a discontinuity can
    flip.  A difference is allowed when
      (i)  tie: the oracle's two best chi2 differ by < 1e-4 relative (the GPU chose the
           other one), or
      (ii) replayed: the oracle's own best-hit step, run from the GPU's predicted state and
           covariance at that step (gpred: what the GPU opened its window around and scored
           against), reproduces the GPU's choice, and the decision sits on a discontinuity --
           the two windows differ (an edge bin), one of the lists was capped, or a best chi2
           lies within 1e-4 relative of the cut.
    The rest of an allowed track is excluded.  Returns (steps compared, allowed by kind,
    unexplained list)."""
    rec = orc["rec"]
    n, nl = orc["idx"].shape
    steps = 0
    allowed = dict(tie=0, edge=0, capped=0, cut=0)
    unexplained = []
    sel = range(n) if t_sel is None else t_sel
    for t in sel:
        for L in range(3, nl):
            a, b = orc["idx"][t, L], gidx[t, L]
            steps += 1
            if a == b:
                continue
            r = rec[t, L]
            kind = None
            if r["chi2_best"] >= 0 and r["chi2_second"] >= 0 and \
                    abs(r["chi2_second"] - r["chi2_best"]) <= 1e-4 * max(r["chi2_best"], 1e-30):
                kind = "tie"
            elif np.all(np.isfinite(gpred[t, L])):
                rp = oracle_mod.besthit_step(g, ev["layers"][L], gpred[t, L, :6], _unpack21(gpred[t, L, 6:]),
                                             int(gq[t]), meas_model=meas_model, chi2_cut=cut)
                choice = rp["best"] if rp["best"] >= 0 and rp["chi2_best"] < cut else -1
                if choice == b:
                    near_cut = any(c >= 0 and abs(c - cut) <= 1e-4 * cut for c in (r["chi2_best"], rp["chi2_best"]))
                    if _window_bins(r) != _window_bins(rp):
                        kind = "edge"
                    elif r["capped"] or rp["capped"]:
                        kind = "capped"
                    elif near_cut:
                        kind = "cut"
            if kind:
                allowed[kind] += 1
            else:
                unexplained.append((t, L, int(a), int(b), float(r["chi2_best"]), float(r["chi2_second"])))
            break
    return steps, allowed, unexplained


def _check_build_cov(res, status, mask):
    """The covariance tolerance of the fits, for built tracks: 1e-3 of sqrt(C_ii C_jj);
    tracks that met a crossing within a few degrees of tangent (KF_ST_GRAZING) are
    held to 1e-2 (the mixed build's double-float step with an FP32 Jacobian leaves up
    to 7.3e-3 there; an FP64 step for such crossings cost 17% of the build)."""
    graz = (status[mask].astype(np.uint32) & kf.KF_ST_GRAZING) != 0
    assert res["dcov"][~graz].max(initial=0.0) <= parity.TOL_COV_NORM, res["dcov"][~graz].max()
    assert res["dcov"][graz].max(initial=0.0) <= 10 * parity.TOL_COV_NORM, res["dcov"][graz].max()


@pytest.mark.parametrize("warp_coop", [True, False])
@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
def test_build_parity(ctx, oracle_mod, warp_coop, precision):
    g = synth.geometry("barrel17")
    events = [synth.gen_event(g, 3000, synth.BASE_SEED + 3 + i) for i in range(2)]
    gpu = run.build_numpy(ctx, g, events, precision=precision, warp_coop=warp_coop, record_pred=True)
    t0 = 0
    tot_steps = tot_allowed = 0
    for ev in events:
        n = ev["n"]
        orc = oracle_mod.build_besthit(g, _binned_oracle_event(oracle_mod, g, ev), record=True)
        gidx = gpu["idx"][t0:t0 + n]
        steps, allowed, bad = classify_build(oracle_mod, g, ev, orc, gidx, gpu["pred"][t0:t0 + n],
                                             gpu["q"][t0:t0 + n])
        assert not bad, bad[:5]
        print(f"build prec={precision} coop={warp_coop}: allowed differences {allowed}")
        tot_steps += steps
        tot_allowed += sum(allowed.values())
        # tracks whose hit lists agree: fitted state within the fit tolerance
        same = np.all(gidx[:, 3:] == orc["idx"][:, 3:], axis=1)
        bad_st = 7
        same &= (orc["status"] & bad_st) == 0
        g_slice = {k: gpu[k][t0:t0 + n] for k in ("state", "cov", "chi2", "ndof", "status", "q")}
        kinds = np.zeros(n, int)
        res = parity.compare_fits(g_slice, _with_oracle_q(oracle_mod, g, ev, orc), kinds, same)
        print(f"build prec={precision} coop={warp_coop}: {same.mean():.4f} identical tracks,",
              parity.summary(res))
        assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
        assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
        _check_build_cov(res, orc["status"], same)
        t0 += n
    print(f"build prec={precision} coop={warp_coop}: {tot_allowed} allowed differences in {tot_steps} steps")
    assert tot_allowed <= 2e-3 * tot_steps


@pytest.mark.parametrize("precision", [kf.KF_PREC_MIXED, kf.KF_PREC_FP64])
def test_build_parity_hit_2d_staggered(ctx, oracle_mod, precision):
    """Best-hit building under measurement model 1 (Sec. 4.1) on the staggered
    barrel: two propagation steps per layer (the average cylinder, then each
    candidate's own), windows widened by the layers' dr, 2-D scoring and updates."""
    g = synth.geometry("barrel17s")
    events = [synth.gen_event(g, 3000, synth.BASE_SEED + 31 + i) for i in range(2)]
    gpu = run.build_numpy(ctx, g, events, precision=precision, meas_model=kf.KF_MEAS_HIT_2D, record_pred=True)
    t0 = 0
    tot_steps = tot_allowed = 0
    effs = []
    for ev in events:
        n = ev["n"]
        orc = oracle_mod.build_besthit(g, _binned_oracle_event(oracle_mod, g, ev), record=True, meas_model=1)
        gidx = gpu["idx"][t0:t0 + n]
        steps, allowed, bad = classify_build(oracle_mod, g, ev, orc, gidx, gpu["pred"][t0:t0 + n],
                                             gpu["q"][t0:t0 + n], meas_model=1)
        assert not bad, bad[:5]
        print(f"model-1 build prec={precision}: allowed differences {allowed}")
        tot_steps += steps
        tot_allowed += sum(allowed.values())
        same = np.all(gidx[:, 3:] == orc["idx"][:, 3:], axis=1) & ((orc["status"] & 7) == 0)
        g_slice = {k: gpu[k][t0:t0 + n] for k in ("state", "cov", "chi2", "ndof", "status", "q")}
        res = parity.compare_fits(g_slice, _with_oracle_q(oracle_mod, g, ev, orc), np.zeros(n, int), same)
        print(f"model-1 build prec={precision}: {same.mean():.4f} identical tracks,", parity.summary(res))
        ids = np.nonzero(same)[0]
        for j in np.argsort(res["max_pull"])[-3:]:
            t = ids[j]
            print("  worst", int(t), res["pull"][j].round(5).tolist(), "ndof", int(orc["ndof"][t]),
                  "oracle", orc["state"][t].tolist(), "gpu", g_slice["state"][t].tolist())
        assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
        assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
        _check_build_cov(res, orc["status"], same)
        where = ev["truth_where"][:, 3:]
        has = where >= 0
        effs.append(np.mean(gidx[:, 3:][has] == where[has]))
        t0 += n
    print(f"model-1 build prec={precision}: {tot_allowed} allowed differences in {tot_steps} steps; "
          f"true-hit efficiency {np.mean(effs):.4f}")
    assert tot_allowed <= 2e-3 * tot_steps
    assert np.mean(effs) > 0.85


def test_build_hit_2d_ignores_warp_coop(ctx):
    """Measurement model 1 always scores one thread per track: asking for the
    warp-cooperative scheme changes nothing."""
    g = synth.geometry("barrel17s")
    events = [synth.gen_event(g, 2000, synth.BASE_SEED + 51)]
    a = run.build_numpy(ctx, g, events, meas_model=kf.KF_MEAS_HIT_2D, warp_coop=False)
    b = run.build_numpy(ctx, g, events, meas_model=kf.KF_MEAS_HIT_2D, warp_coop=True)
    for k in ("idx", "state", "cov", "chi2", "ndof", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def _with_oracle_q(oracle_mod, g, ev, orc):
    q = np.array([oracle_mod.seed(ev["seed_hits"][t, 0], ev["seed_hits"][t, 1], ev["seed_hits"][t, 2], g["bz"])[1]
                  for t in range(ev["n"])], np.int8)
    return dict(orc, q=q)


@pytest.mark.parametrize("name,model", [("barrel17", 0), ("barrel17s", 1)])
def test_build_full_size_sampled(ctx, oracle_mod, name, model):
    """Ten events of 20,000 tracks with 20% noise in one launch; the oracle checks 300
    tracks of each event against the same binned layers.  The staggered barrel runs
    measurement model 1."""
    g = synth.geometry(name)
    events = [synth.gen_event(g, 20000, synth.BASE_SEED + 3 + i) for i in range(10)]
    gpu = run.build_numpy(ctx, g, events, meas_model=model, record_pred=True)
    t0 = 0
    tot = [0, 0]
    kinds = dict(tie=0, edge=0, capped=0, cut=0)
    eff = []
    for ev in events:
        n = ev["n"]
        ev = _binned_oracle_event(oracle_mod, g, ev)
        sel = np.sort(np.random.default_rng(t0).choice(n, 300, replace=False))
        orc = oracle_mod.build_besthit(g, ev, record=True, meas_model=model)  # all tracks: fast enough
        steps, allowed, bad = classify_build(oracle_mod, g, ev, orc, gpu["idx"][t0:t0 + n], gpu["pred"][t0:t0 + n],
                                             gpu["q"][t0:t0 + n], sel, meas_model=model)
        assert not bad, bad[:5]
        tot[0] += steps
        tot[1] += sum(allowed.values())
        for k, v in allowed.items():
            kinds[k] += v
        # efficiency of the algorithm (fraction of true hits kept) on the sample, GPU and oracle
        where = ev["truth_where"][sel, 3:]
        has = where >= 0
        eff.append((np.mean(gpu["idx"][t0:t0 + n][sel, 3:][has] == where[has]),
                    np.mean(orc["idx"][sel, 3:][has] == where[has])))
        t0 += n
    eg, eo = np.mean(eff, axis=0)
    print(f"full size {name} model {model}: {tot[1]} allowed differences {kinds} in {tot[0]} sampled steps; "
          f"true-hit efficiency GPU {eg:.4f}, oracle {eo:.4f}")
    assert abs(eg - eo) <= 2e-3 * max(1, tot[1])
    assert eg > 0.85


def _ckf_fragile(m):
    """Seeds where the oracle came close to a different decision: a ranking of
    two children of equal hit count within 1e-4 relative (the last kept against
    the first dropped, or the final first and second), a chi2 within 1e-4 of the
    cut, a window edge within 1e-4 bin of a bin boundary, or a capped window."""
    return (m["rank_gap"] < 1e-4) | (m["cut_gap"] < 1e-4) | (m["edge_gap"] < 1e-4) | (m["capped"] != 0)


@pytest.mark.parametrize("n_slots", [1, 2, 4, 8])
def test_ckf_parity(ctx, oracle_mod, n_slots):
    """Combinatorial building: per seed, the hits of the best candidate equal the
    oracle's unless the oracle's own decisions were within rounding of flipping;
    where the hits agree the fitted state agrees within the fit tolerance."""
    g = synth.geometry("barrel17")
    events = [synth.gen_event(g, 3000, synth.BASE_SEED + 21 + i) for i in range(2)]
    gpu = run.build_numpy(ctx, g, events, n_slots=n_slots)
    t0 = 0
    for ev in events:
        n = ev["n"]
        orc = oracle_mod.build_ckf(g, _binned_oracle_event(oracle_mod, g, ev), n_slots=n_slots, threads=8)
        gidx = gpu["idx"][t0:t0 + n]
        assert (gidx[:, :3] == -1).all()  # the seed layers: the caller knows those hits
        same = np.all(gidx[:, 3:] == orc["idx"][:, 3:], axis=1)
        fragile = _ckf_fragile(orc["margin"])
        unexplained = np.nonzero(~same & ~fragile)[0]
        print(f"ckf {n_slots} slots: {same.mean():.4f} identical, {fragile.mean():.4f} fragile, "
              f"{len(unexplained)} unexplained")
        assert len(unexplained) == 0, [(int(t), gidx[t, 3:].tolist(), orc["idx"][t, 3:].tolist())
                                       for t in unexplained[:3]]
        assert same.mean() >= 0.97
        ok = same & ((orc["status"] & 7) == 0)
        g_slice = {k: gpu[k][t0:t0 + n] for k in ("state", "cov", "chi2", "ndof", "status", "q")}
        res = parity.compare_fits(g_slice, _with_oracle_q(oracle_mod, g, ev, orc), np.zeros(n, int), ok)
        print("   ", parity.summary(res))
        assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
        assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
        _check_build_cov(res, orc["status"], ok)
        np.testing.assert_array_equal(gpu["ndof"][t0:t0 + n][ok], orc["ndof"][ok])
        t0 += n


def test_ckf_full_size_sampled(ctx, oracle_mod):
    """Ten events of 20,000 tracks, four slots per seed, in one launch; the oracle
    checks 300 seeds of each event; more true hits than best-hit building."""
    g = synth.geometry("barrel17")
    events = [synth.gen_event(g, 20000, synth.BASE_SEED + 3 + i) for i in range(10)]
    gpu = run.build_numpy(ctx, g, events, n_slots=4)
    best = run.build_numpy(ctx, g, events)
    t0 = 0
    eff = []
    for ev in events:
        n = ev["n"]
        ev = _binned_oracle_event(oracle_mod, g, ev)
        sel = np.sort(np.random.default_rng(t0 + 1).choice(n, 300, replace=False))
        gidx = gpu["idx"][t0:t0 + n]
        for a in np.split(sel, 6):
            for t in a:
                orc = oracle_mod.build_ckf(g, ev, n_slots=4, t0=int(t), t1=int(t) + 1)
                if not np.array_equal(gidx[t, 3:], orc["idx"][t, 3:]):
                    assert _ckf_fragile(orc["margin"][t:t + 1])[0], (int(t), gidx[t].tolist(), orc["idx"][t].tolist())
        where = ev["truth_where"][:, 3:]
        has = where >= 0
        eff.append((np.mean(gidx[:, 3:][has] == where[has]),
                    np.mean(best["idx"][t0:t0 + n][:, 3:][has] == where[has])))
        t0 += n
    ec, eb = np.mean(eff, axis=0)
    print(f"full size: true-hit efficiency, 4 slots {ec:.4f}, best-hit {eb:.4f}")
    assert ec > eb


def test_ckf_rejects_bad_arguments(ctx):
    g = synth.geometry("barrel17")
    ev = synth.gen_event(g, 50, synth.BASE_SEED + 7)
    with pytest.raises(kf.KfError):
        run.build_numpy(ctx, g, [ev], n_slots=3)
    with pytest.raises(kf.KfError):
        run.build_numpy(ctx, g, [ev], n_slots=4, precision=kf.KF_PREC_FP64)
    with pytest.raises(kf.KfError):  # measurement model 1 runs on the best-hit path only
        run.build_numpy(ctx, g, [ev], n_slots=2, meas_model=kf.KF_MEAS_HIT_2D)


def test_gather_and_final_fit(ctx, oracle_mod):
    """Gather the chosen hits (seed hits + accepted ones) and fit them again: the fit
    input equals the oracle-side assembly of the same hits, and the fit matches."""
    g = synth.geometry("barrel17")
    events = [synth.gen_event(g, 2000, synth.BASE_SEED + 9)]
    gpu = run.build_numpy(ctx, g, events)
    n = events[0]["n"]
    nl = len(events[0]["layers"])
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    lay = torch.empty(n * nl, dtype=torch.uint8, device="cuda")
    x, y, z = (torch.empty(n * nl, dtype=torch.float32, device="cuda") for _ in range(3))
    kf.kf_gather_hits(ctx, 1, nl, gpu["layers"], gpu["eoff"], gpu["sh9"], gpu["idx_dev"], off, lay, x, y, z)
    torch.cuda.synchronize()
    off_h = off.cpu().numpy()
    ev = events[0]
    # expected CSR from the chosen indices
    exp_off = [0]
    ex, ey, ez, el = [], [], [], []
    for t in range(n):
        for k in range(3):
            ex.append(ev["seed_hits"][t, k, 0]); ey.append(ev["seed_hits"][t, k, 1]); ez.append(ev["seed_hits"][t, k, 2])
            el.append(k)
        for L in range(3, nl):
            h = gpu["idx"][t, L]
            if h >= 0:
                ly = ev["layers"][L]
                ex.append(ly["x"][h]); ey.append(ly["y"][h]); ez.append(ly["z"][h]); el.append(L)
        exp_off.append(len(ex))
    np.testing.assert_array_equal(off_h, exp_off)
    m = off_h[-1]
    np.testing.assert_array_equal(x.cpu().numpy()[:m], np.array(ex, np.float32))
    np.testing.assert_array_equal(lay.cpu().numpy()[:m], np.array(el, np.uint8))
    tk = dict(offsets=off_h, layer=lay.cpu().numpy()[:m], x=x.cpu().numpy()[:m], y=y.cpu().numpy()[:m],
              z=z.cpu().numpy()[:m], n=n)
    gfit = run.fit_numpy(ctx, g, tk)
    ofit = oracle_mod.fit(g, tk)
    ok = (ofit["status"] & 7) == 0
    np.testing.assert_array_equal(gfit["ndof"], ofit["ndof"])
    res = parity.compare_fits(gfit, ofit, np.zeros(n, int), ok)
    print("final fit:", parity.summary(res))
    assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
    assert res["dcov"].max() <= parity.TOL_COV_NORM
