"""The serving loop (kf_server_*): events submitted from host memory, admitted
under a device-memory budget, merged into batches and run on overlapping
streams.  Every result must be bit-identical to the direct entry points on the
same event (bin, seed, build, gather, fit), whatever the event was batched
with; the direct path is itself checked against the oracle in
test_gpu_build.py."""
import numpy as np
import pytest
import torch

from paper_1711_06571_gb300 import kf, run, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return run.context(0)


@pytest.fixture(scope="module")
def geom():
    return synth.geometry("barrel17")


def _event_arrays(ev):
    L = len(ev["layers"])
    xs = [None if l < 3 else np.ascontiguousarray(ev["layers"][l]["x"], np.float32) for l in range(L)]
    ys = [None if l < 3 else np.ascontiguousarray(ev["layers"][l]["y"], np.float32) for l in range(L)]
    zs = [None if l < 3 else np.ascontiguousarray(ev["layers"][l]["z"], np.float32) for l in range(L)]
    surf = [int(ly["surf"]) for ly in ev["layers"]]
    return surf, xs, ys, zs, np.ascontiguousarray(ev["seed_hits"], np.float32)


def _result_arrays(n, L):
    return dict(hit_idx=np.full((L, n), -7, np.int32), state=np.zeros((6, n)), cov=np.zeros((21, n)),
                chi2=np.zeros(n), ndof=np.zeros(n, np.int32), status=np.zeros(n, np.uint32))


def submit(srv, ev, zero_copy=False, pinned_results=False):
    surf, xs, ys, zs, sh = _event_arrays(ev)
    n, L = ev["n"], len(surf)
    res = _result_arrays(n, L)
    if pinned_results:  # page-locked result arrays
        res = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in res.items()}
    rc, t = kf.kf_server_submit(srv, n, surf, xs, ys, zs, sh, zero_copy=zero_copy, **res)
    return rc, t, res


def direct(ctx, g, ev):
    """The same event through the direct entry points: bin every layer, seed,
    build, gather, final fit (grid schedule)."""
    gpu = run.build_numpy(ctx, g, [ev])
    n, nl = ev["n"], len(ev["layers"])
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    lay = torch.empty(n * nl, dtype=torch.uint8, device="cuda")
    x, y, z = (torch.empty(n * nl, dtype=torch.float32, device="cuda") for _ in range(3))
    kf.kf_gather_hits(ctx, 1, nl, gpu["layers"], gpu["eoff"], gpu["sh9"], gpu["idx_dev"], off, lay, x, y, z)
    dh = dict(offsets=off, layer=lay, x=x, y=y, z=z, n=n)
    gk = kf.make_geometry(g)
    seeds = run.make_seeds(ctx, gk, dh)
    out = run.alloc_fit_out(n)
    run.fit(ctx, gk, dh, seeds, out)
    torch.cuda.synchronize()
    return dict(hit_idx=gpu["idx_dev"].cpu().numpy(), state=out["state"].cpu().numpy(),
                cov=out["cov"].cpu().numpy(), chi2=out["chi2"].cpu().numpy(), ndof=out["ndof"].cpu().numpy(),
                status=(out["status"].cpu().numpy().astype(np.uint32) | gpu["status"]))


def assert_identical(got, exp, what):
    for k in ("hit_idx", "state", "cov", "chi2", "ndof", "status"):
        a, b = np.asarray(got[k]), np.asarray(exp[k])
        assert a.shape == b.shape, (what, k, a.shape, b.shape)
        same = (a == b) | (np.isnan(a) & np.isnan(b)) if a.dtype.kind == "f" else (a == b)
        assert same.all(), f"{what}: {k} differs at {np.argwhere(~same)[:5].tolist()}"


def _events(g, sizes, seed0):
    return [synth.gen_event(g, n, synth.BASE_SEED + seed0 + i) for i, n in enumerate(sizes)]


def test_server_alone_and_mixed_match_direct_path(ctx, geom):
    events = _events(geom, [3000, 700, 5000, 1], 40)
    ly = events[1]["layers"][7]  # an empty build layer: an empty segment of the batch's binning
    for k in ("x", "y", "z"):
        ly[k] = ly[k][:0]
    exp = [direct(ctx, geom, ev) for ev in events]
    # alone: one event per batch
    srv = kf.kf_server_create(ctx, geom, kf.server_params(max_batch_events=1))
    try:
        rc, t, res = submit(srv, events[0])
        assert rc == kf.KF_OK
        rc, lat = kf.kf_server_wait(srv, t, 60000)
        assert rc == kf.KF_OK and lat > 0
        assert_identical(res, exp[0], "alone")
    finally:
        kf.kf_server_destroy(srv)
    # mixed: all four merged into one batch by the batch window, with inputs read in
    # place or staged and results in pageable or page-locked arrays
    srv = kf.kf_server_create(ctx, geom, kf.server_params(max_batch_events=16, batch_window_ms=2000))
    try:
        subs = [submit(srv, ev, zero_copy=(i % 2 == 0), pinned_results=(i == 1)) for i, ev in enumerate(events)]
        assert all(rc == kf.KF_OK for rc, _, _ in subs)
        for (rc, t, res), e, i in zip(subs, exp, range(len(events))):
            rc, _ = kf.kf_server_wait(srv, t, 60000)
            assert rc == kf.KF_OK
            assert_identical(res, e, f"mixed event {i}")
        st = kf.kf_server_stats_get(srv)
        assert st["completed"] == len(events) and st["batches"] == 1, st
        assert st["mean_batch_events"] == len(events)
        assert st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        kf.kf_server_destroy(srv)


def _pinned_at(a, shift):
    """A copy of a in page-locked memory at `shift` bytes past a 64-byte boundary."""
    buf = torch.empty(a.nbytes + 64 + shift, dtype=torch.uint8).pin_memory().numpy()
    base = (-buf.ctypes.data) % 64 + shift
    v = buf[base:base + a.nbytes].view(a.dtype).reshape(a.shape)
    v[...] = a
    return v


def test_server_misaligned_arrays_are_staged(ctx, geom):
    """Page-locked arrays that are not aligned to their element size (doubles at
    4 bytes past an 8-byte boundary, floats at 2 bytes past a 4-byte one) are
    not handed to the kernels: the server stages them through its own aligned
    buffers, and the results are those of the direct path.  Merged in one batch
    with an event whose aligned page-locked arrays are read and written in place."""
    events = _events(geom, [1501, 999, 2000], 90)
    exp = [direct(ctx, geom, ev) for ev in events]
    srv = kf.kf_server_create(ctx, geom, kf.server_params(max_batch_events=16, batch_window_ms=2000))
    try:
        subs = []
        for i, ev in enumerate(events):
            surf, xs, ys, zs, sh = _event_arrays(ev)
            n, L = ev["n"], len(surf)
            res = _result_arrays(n, L)
            if i == 0:  # results misaligned, inputs aligned and read in place
                res = {k: _pinned_at(v, 4) for k, v in res.items()}
                xs, ys, zs = ([None if a is None else _pinned_at(a, 0) for a in c] for c in (xs, ys, zs))
                sh = _pinned_at(sh, 0)
            elif i == 1:  # inputs misaligned (zero-copy asked for), results aligned
                res = {k: _pinned_at(v, 0) for k, v in res.items()}
                xs, ys, zs = ([None if a is None else _pinned_at(a, 2) for a in c] for c in (xs, ys, zs))
                sh = _pinned_at(sh, 2)
            else:  # everything aligned and page-locked
                res = {k: _pinned_at(v, 0) for k, v in res.items()}
                xs, ys, zs = ([None if a is None else _pinned_at(a, 0) for a in c] for c in (xs, ys, zs))
                sh = _pinned_at(sh, 0)
            rc, t = kf.kf_server_submit(srv, n, surf, xs, ys, zs, sh, zero_copy=True, **res)
            assert rc == kf.KF_OK
            subs.append((t, res))
        for (t, res), e, i in zip(subs, exp, range(len(events))):
            assert kf.kf_server_wait(srv, t, 60000)[0] == kf.KF_OK
            assert_identical(res, e, f"event {i}")
        st = kf.kf_server_stats_get(srv)
        assert st["completed"] == len(events) and st["batches"] == 1 and st["rc"] == kf.KF_OK, st
    finally:
        kf.kf_server_destroy(srv)


def test_server_many_events_overlapping_batches(ctx, geom):
    """A stream of events of mixed sizes through several batches in flight."""
    events = _events(geom, [400, 2500, 60, 1200, 3100, 900, 10, 2000, 1500, 700], 60)
    exp = [direct(ctx, geom, ev) for ev in events]
    srv = kf.kf_server_create(ctx, geom, kf.server_params(max_batches=3, max_batch_events=3))
    try:
        subs = [submit(srv, ev, zero_copy=True) for ev in events]
        for (rc, t, res), e, i in zip(subs, exp, range(len(events))):
            assert rc == kf.KF_OK
            assert kf.kf_server_wait(srv, t, 60000)[0] == kf.KF_OK
            assert_identical(res, e, f"event {i}")
        st = kf.kf_server_stats_get(srv, reset=True)
        assert st["completed"] == len(events) and st["rc"] == kf.KF_OK
        assert st["queued"] == 0 and st["in_flight_events"] == 0 and st["bytes_in_use"] == 0
    finally:
        kf.kf_server_destroy(srv)


def test_server_admission_stays_within_budget(ctx, geom):
    events = _events(geom, [2000, 2000, 2000, 2000], 80)
    # footprint of one event, as the server reserves it
    srv = kf.kf_server_create(ctx, geom, kf.server_params(max_batch_events=1))
    try:
        rc, t, _ = submit(srv, events[0])
        assert rc == kf.KF_OK and kf.kf_server_wait(srv, t, 60000)[0] == kf.KF_OK
        one = kf.kf_server_stats_get(srv)["peak_bytes_in_use"]
        assert one > 0
    finally:
        kf.kf_server_destroy(srv)
    budget = int(one * 1.5)  # room for one event at a time
    srv = kf.kf_server_create(ctx, geom, kf.server_params(mem_budget_bytes=budget, max_batches=4,
                                                          max_batch_events=8))
    try:
        subs = [submit(srv, ev) for ev in events]
        assert all(rc == kf.KF_OK for rc, _, _ in subs)
        for rc, t, _ in subs:
            assert kf.kf_server_wait(srv, t, 60000)[0] == kf.KF_OK
        st = kf.kf_server_stats_get(srv)
        assert 0 < st["peak_bytes_in_use"] <= budget
        assert st["batches"] == len(events)  # never two at once
        # an event that alone needs more than the budget is refused at submission
        big = synth.gen_event(geom, 8000, synth.BASE_SEED + 99)
        rc, _, _ = submit(srv, big)
        assert rc == kf.KF_EBUSY
        assert kf.kf_server_stats_get(srv)["rejected"] == 1
    finally:
        kf.kf_server_destroy(srv)


def test_server_staging_limits_and_tickets(ctx, geom):
    ev = synth.gen_event(geom, 3000, synth.BASE_SEED + 120)
    srv = kf.kf_server_create(ctx, geom, kf.server_params(host_staging_bytes=1 << 20))
    try:
        rc, _, _ = submit(srv, ev)  # needs more pinned staging than the whole arena
        assert rc == kf.KF_EBUSY
    finally:
        kf.kf_server_destroy(srv)
    srv = kf.kf_server_create(ctx, geom, kf.server_params(batch_window_ms=3000))
    try:
        rc, t, res = submit(srv, ev)
        assert rc == kf.KF_OK
        assert kf.kf_server_poll(srv, t)[0] == kf.KF_EAGAIN  # held by the batch window
        assert kf.kf_server_wait(srv, t, 5.0)[0] == kf.KF_ETIMEOUT
        assert kf.kf_server_wait(srv, t, 60000)[0] == kf.KF_OK
        assert kf.kf_server_poll(srv, t)[0] == kf.KF_EINVAL  # reported once
        assert kf.kf_server_poll(srv, 987654321)[0] == kf.KF_EINVAL
        assert (res["hit_idx"][:3] == -1).all() and (res["hit_idx"] != -7).all()
    finally:
        kf.kf_server_destroy(srv)


def test_server_rejects_malformed_events(ctx, geom):
    ev = synth.gen_event(geom, 50, synth.BASE_SEED + 130)
    surf, xs, ys, zs, sh = _event_arrays(ev)
    srv = kf.kf_server_create(ctx, geom)
    try:
        with pytest.raises(kf.KfError):
            kf.kf_server_submit(srv, ev["n"], surf[:3], xs[:3], ys[:3], zs[:3], sh)  # no build layer
        bad = list(surf)
        bad[5] = 99
        with pytest.raises(kf.KfError):
            kf.kf_server_submit(srv, ev["n"], bad, xs, ys, zs, sh)
        with pytest.raises(kf.KfError):
            kf.kf_server_submit(srv, 0, surf, xs, ys, zs, sh)
    finally:
        kf.kf_server_destroy(srv)
