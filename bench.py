"""Benchmark of the batched Kalman-filter track fit on GB300.

Workload (one step): seed estimate + KF fit of 1,000,000 synthetic tracks over
17 barrel layers (R = 4..100 cm, Bz = 3.8 T, x/X0 = 0.02, seeds from three hits,
seed covariance 1e4), mixed precision (FP32 + FP64 S solve and seed phase).
Metric: track-layer updates per second (one update = propagation, transport,
scattering noise and KF update of one track at one layer).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KF track-layer updates/sec, FP32 vs FP64 on one GB300 at stated err; p99 event ms"
UNIT = "updates/s"
N_TRACKS = 1_000_000
WORKLOAD = ("KF fit of 1,000,000 tracks x 17 barrel layers (R 4-100 cm), Bz 3.8 T, x/X0 0.02, "
            "pT log-uniform 0.5-10 GeV, |eta|<1, seeds from 3 hits, seed cov 1e4")

# Algorithmic work per unit, counted from the formulas the two fit kernels evaluate.
# Phase 1 (fit_seed_kernel, per track with barrel seed hits): the first
# transport in FP64 on the covariance the closed-form seed-hit update leaves
# (151 FLOP) and the conversions of that covariance to FP64 and back (42 FLOP),
# chi2 (1); the rest in double-float on the FP32 pipe.  Phase 2
# (fit_loop_kernel, per later update): the FP64 S solve (LDL^T 29 + chi2 15);
# FP32 (propagation ~250, transport 310, noise ~25, update ~314).
# DRAM bytes (read + write) of one fit_loop_kernel launch on this workload, from
# an ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); None whenever the kernel changes until it is captured again
LOOP_KERNEL_DRAM_BYTES = 1.475e9
FP64_FLOP_PHASE1_BARREL = 194.0
FP64_FLOP_PER_FP32_UPDATE = 44.0
FP32_FLOP_PER_FP32_UPDATE = 900.0
# carry from phase 1 to phase 2 per track: state 11 + covariance 21 floats, chi2, k, used, status
CARRY_BYTES_PER_TRACK = 4 * 11 + 4 * 21 + 8 + 3 * 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tracks", type=int, default=N_TRACKS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop sweep")
    ap.add_argument("--part", default="all", choices=["all", "build", "serving", "uneven", "layout", "nonideal"],
                    help="build / serving: only that measurement, printed as its own JSON line")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="--impl reference: tracks of the workload the oracle fits per step "
                         "(0: sized so the run takes about two minutes)")
    ap.add_argument("--serving-memory", default="pinned", choices=["pinned", "pageable"],
                    help="client buffers of the serving sweep: page-locked (allocated once) or pageable")
    ap.add_argument("--serving-copy", action="store_true", help="serving sweep: staged copies instead of zero-copy")
    ap.add_argument("--serving-rates", default="auto",
                    help="comma-separated arrival rates (events/s) of the serving sweep, or auto")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed device-resident fit steps (the command the profiles capture)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
            os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait(timeout=10)
        text = open(self.path).read()
        os.unlink(self.path)
        return self.parse(text)

    @staticmethod
    def parse(text):
        """Median SM clock, maximum clock and the throttle reasons seen, from
        nvidia-smi's CSV rows; rows cut short (the sampler is stopped in the
        middle of a line) are skipped."""
        rows = [[f.strip() for f in l.split(",")] for l in text.splitlines() if l.strip()]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    samples=len(rows), reasons=reasons)


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def _reduce(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX)


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM)


def rank_seed(rank):
    """Each rank fits its own tracks: independent units, no exchange step."""
    from paper_1711_06571_gb300 import synth
    return synth.BASE_SEED + 2 + 1000 * rank


def aggregate(ms_local, units_local, world):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    ms = max_over_ranks(ms_local, world)
    total = sum_over_ranks(units_local, world)
    return ms, total, total / (ms * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_baseline(geom, tk, n_sample, threads, passes=1):
    """FP64 oracle fit of the first n_sample tracks on `threads` host threads,
    `passes` times over."""
    import oracle
    oracle.build_lib()
    off = tk["offsets"]
    sub = dict(offsets=off[:n_sample + 1], layer=tk["layer"], x=tk["x"], y=tk["y"], z=tk["z"])
    upd = 0
    t0 = time.perf_counter()
    for _ in range(passes):
        r = oracle.fit(geom, sub, t1=n_sample, threads=threads)
        upd += int(np.sum((r["ndof"][:n_sample] + 5) // 2))
    dt = time.perf_counter() - t0
    return upd / dt, upd, dt


BUILD_WORKLOAD = ("best-hit build of 10 events x 20,000 tracks, 17 barrel layers + 20% uniform noise hits per "
                  "layer, 1024 phi x 64 z bins, window 3 sigma, <= 32 candidates, chi2 cut 30, all events in one "
                  "launch")


def build_bench(ctx, geom, steps, warmup, n_events=10, n_tracks=20000, meas_model=0, ckf_slots=(2, 4, 8)):
    """One step: bin every layer of every event (kf_bin_hits_batched), seed
    estimate from the seed hits (kf_make_seeds), best-hit build of all events
    (kf_build_besthit).  Inputs resident on the device."""
    import torch
    from paper_1711_06571_gb300 import kf, run, synth
    events = [synth.gen_event(geom, n_tracks, synth.BASE_SEED + 300 + e) for e in range(n_events)]
    L = len(events[0]["layers"])
    segs = [ev["layers"][l] for ev in events for l in range(L)]
    so = np.concatenate([[0], np.cumsum([len(ly["x"]) for ly in segs])]).astype(np.int64)
    half = [geom["surfaces"][ly["surf"]]["half_or_rin"] for ly in segs]
    H, ns = int(so[-1]), len(segs)
    dev = torch.device("cuda")
    x, y, z = (torch.from_numpy(np.concatenate([ly[k] for ly in segs]).astype(np.float32)).to(dev)
               for k in ("x", "y", "z"))
    perm = torch.empty(H, dtype=torch.int32, device=dev)
    offs = torch.empty((ns, kf.KF_NBINS + 1), dtype=torch.int32, device=dev)
    packed = torch.empty((H, 4), dtype=torch.float32, device=dev)
    layers = kf.binned_layers([dict(n_hits=int(so[i + 1] - so[i]), surface=int(segs[i]["surf"]),
                                    packed=packed[so[i]:so[i + 1]] if so[i + 1] > so[i] else packed,
                                    offsets=offs[i]) for i in range(ns)])
    counts = [ev["n"] for ev in events]
    eoff = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(eoff[-1])
    sh = np.concatenate([ev["seed_hits"].reshape(-1, 9) for ev in events]).astype(np.float32).reshape(n, 3, 3)
    sk = dict(offsets=(np.arange(n + 1) * 3).astype(np.int32), layer=np.zeros(3 * n, np.uint8),
              x=sh[:, :, 0].reshape(-1), y=sh[:, :, 1].reshape(-1), z=sh[:, :, 2].reshape(-1))
    dsk = run.hits_to_device(sk)
    sh9 = torch.from_numpy(np.ascontiguousarray(sh.reshape(n, 9).T)).to(dev)
    g = kf.make_geometry(geom)
    seed_st = torch.empty((6, n), dtype=torch.float32, device=dev)
    seed_q = torch.empty(n, dtype=torch.int8, device=dev)
    idx = torch.empty((L, n), dtype=torch.int32, device=dev)
    out = run.alloc_fit_out(n)
    fp, bp = kf.fit_params(meas_model=meas_model), kf.build_params()
    stream = torch.cuda.current_stream()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        kf.kf_bin_hits_batched(ctx, so, half, x, y, z, perm, offs, packed)
        kf.kf_make_seeds(ctx, g, n, dsk["offsets"], dsk["x"], dsk["y"], dsk["z"], seed_st, seed_q)
        if evs:
            evs[1].record(stream)
        kf.kf_build_besthit(ctx, g, fp, bp, n_events, L, layers, eoff, seed_st, seed_q, sh9, idx, out["state"],
                            out["cov"], out["chi2"], out["ndof"], out["status"])
        if evs:
            evs[2].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for k in range(steps):
        step(evs[k])
    torch.cuda.synchronize()
    t_bin = float(np.mean([a.elapsed_time(b) for a, b, _ in evs]))
    t_build = float(np.mean([b.elapsed_time(c) for _, b, c in evs]))
    t_step = float(np.mean([a.elapsed_time(c) for a, _, c in evs]))
    units = n * (L - 3)  # track-layer build steps per launch
    found = float((idx[3:] >= 0).float().mean().item())
    where = np.concatenate([ev["truth_where"][:, 3:] for ev in events])
    has = where >= 0
    eff_best = float(np.mean(idx[3:].t().cpu().numpy()[has] == where[has]))

    # combinatorial building of the same seeds: n_slots candidates per seed
    ckf = {}
    for ns in ckf_slots:
        def ckf_launch():
            kf.kf_build_ckf(ctx, g, fp, bp, ns, n_events, L, layers, eoff, seed_st, seed_q, sh9, idx,
                            out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
        for _ in range(warmup):
            ckf_launch()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(steps):
            ckf_launch()
        a1.record(stream)
        torch.cuda.synchronize()
        ms = a0.elapsed_time(a1) / steps
        eff = float(np.mean(idx[3:].t().cpu().numpy()[has] == where[has]))
        ckf[f"{ns}_slots"] = dict(build_launch_ms=ms, candidate_steps_per_s=units * ns / (ms * 1e-3),
                                  seed_steps_per_s=units / (ms * 1e-3), true_hit_efficiency=eff)
    return dict(workload=BUILD_WORKLOAD, value=units / (t_step * 1e-3), unit="track-layer build steps/s",
                ms_per_step=t_step, bin_and_seed_ms=t_bin, build_launch_ms=t_build,
                build_kernel_steps_per_s=units / (t_build * 1e-3), hits_binned=H, tracks=n,
                steps_measured=steps, fraction_of_steps_with_a_hit=found, true_hit_efficiency=eff_best,
                # binning (key, FP64 keys, scan, scatter, rank), seed estimate, order pass (3),
                # seed pre-pass, layer kernel
                gpu_launches_per_step=5 + 1 + 3 + 2, combinatorial=ckf)


NONIDEAL_WORKLOAD = ("non-ideal barrel (Sec. 4.1): 17 layers whose modules sit at alternating radii "
                     "R - 0.25 / R + 0.25 cm (R = 4 + 6 i cm), measurement model 1 (each barrel hit reached on "
                     "the cylinder through it, 2-D update on its tangent plane); fit of 1,000,000 tracks and "
                     "best-hit building (two propagation steps per layer) of 10 events x 20,000 tracks")


def nonideal_bench(ctx, steps, warmup, n_tracks=1_000_000):
    """Measurement model 1 on the staggered barrel: the fit (kf_fit, grid schedule)
    and best-hit building, with model 0 on the same inputs for comparison (its
    parity against the oracle is the tests' business)."""
    import torch
    from paper_1711_06571_gb300 import kf, run, synth
    geom = synth.geometry("barrel17s")
    g = kf.make_geometry(geom)
    tk = synth.gen_tracks(geom, n_tracks, synth.BASE_SEED + 400)
    n = tk["n"]
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, g, dh)
    stream = torch.cuda.current_stream()
    fits = {}
    for model in (1, 0):
        out = run.alloc_fit_out(n)
        p = kf.fit_params(meas_model=model)

        def launch():
            kf.kf_fit(ctx, g, p, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                      out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
        for _ in range(warmup):
            launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            launch()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        upd = int(((out["ndof"] + 5) // 2).clamp(min=0).sum().item())
        chi2 = out["chi2"].cpu().numpy()
        ndof = out["ndof"].cpu().numpy()
        good = ndof > 0
        fits[f"model_{model}"] = dict(fit_ms_per_launch=ms, updates_per_s=upd / (ms * 1e-3),
                                      median_chi2_per_ndof=float(np.median(chi2[good] / ndof[good])))
    b1 = build_bench(ctx, geom, steps, warmup, meas_model=1, ckf_slots=())
    b0 = build_bench(ctx, geom, 2, 1, meas_model=0, ckf_slots=())
    build = dict(model_1=dict((k, b1[k]) for k in ("value", "unit", "ms_per_step", "bin_and_seed_ms",
                                                      "build_launch_ms", "true_hit_efficiency")),
                 model_0_true_hit_efficiency=b0["true_hit_efficiency"])
    return dict(workload=NONIDEAL_WORKLOAD, tracks=n, fit=fits, build=build)


UNEVEN_WORKLOAD = ("KF fit of 2,000,000 tracks, |eta| < 2.5, 17 barrel cylinders + 2 x 12 end-cap disks at "
                   "|z| = 30-270 cm (4-26 hits per track), mixed precision, tracks bucketed by hit count, "
                   "persistent kernel with an atomic work queue replayed as a CUDA graph, launch shape from "
                   "kf_autotune_fit")


def uneven_bench(ctx, steps, warmup, n_tracks=2_000_000):
    """The uneven batch in one persistent launch: autotune, then time the
    graph-replayed persistent fit and, for comparison, the grid schedule."""
    import torch
    from paper_1711_06571_gb300 import kf, run, synth
    geom = synth.geometry("lids")
    g = kf.make_geometry(geom)
    # the generator runs on the GPU here (2e6 tracks take minutes on the host)
    tk = synth.gen_tracks(geom, n_tracks, synth.BASE_SEED + 4, eta_max=2.5, min_hits=4, device="cuda")
    n = tk["n"]
    nh = np.diff(tk["offsets"])
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, g, dh)
    out = run.alloc_fit_out(n)
    stream = torch.cuda.current_stream()
    p_grid = kf.fit_params(schedule=kf.KF_SCHED_GRID)
    p_pers = kf.fit_params(schedule=kf.KF_SCHED_PERSISTENT)
    report = kf.kf_autotune_fit(ctx, g, p_pers, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"],
                                dh["y"], dh["z"], out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])

    def timed(params):
        def launch():
            kf.kf_fit(ctx, g, params, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                      out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
        for _ in range(warmup):
            launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            launch()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    ms_pers = timed(p_pers)
    upd = int(((out["ndof"] + 5) // 2).clamp(min=0).sum().item())
    ms_grid = timed(p_grid)
    return dict(workload=UNEVEN_WORKLOAD, value=upd / (ms_pers * 1e-3), unit="updates/s", ms_per_launch=ms_pers,
                tracks=int(n), updates_per_launch=upd, hits_per_track=dict(min=int(nh.min()), max=int(nh.max()),
                                                                          mean=float(nh.mean())),
                autotune="block,tracks_per_thread,grid,ms = " + report, grid_schedule_ms=ms_grid,
                persistent_speedup=ms_grid / ms_pers, steps_measured=steps)


def layout_study(ctx, sizes=(32 * 1024, 256 * 1024, 2 * 1024 * 1024, 8 * 1024 * 1024), reps=20):
    """Sec. 4.3's layout study on GB300: the covariance transport P' = J P J^T of n
    matrices per launch (one per thread, FP32, operands in registers), in the AOS,
    SOA and Matriplex-like BLOCK layouts; time per launch and the bytes it moves."""
    import torch
    from paper_1711_06571_gb300 import kf
    stream = torch.cuda.current_stream()
    out = []
    for n in sizes:
        J = torch.randn(n * 36, device="cuda")
        P = torch.randn(n * 21, device="cuda")
        Po = torch.empty(n * 21, device="cuda")
        row = dict(n=n, bytes_per_launch=n * (36 + 21 + 21) * 4)
        for name, layout in (("aos", kf.KF_LAYOUT_AOS), ("soa", kf.KF_LAYOUT_SOA), ("block", kf.KF_LAYOUT_BLOCK)):
            for _ in range(3):
                kf.kf_layout_transport(ctx, layout, n, J, P, Po)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                kf.kf_layout_transport(ctx, layout, n, J, P, Po)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            row[name] = dict(ms=ms, ns_per_matrix=ms * 1e6 / n, gb_s=row["bytes_per_launch"] / (ms * 1e-3) / 1e9)
        out.append(row)
        del J, P, Po
    return dict(workload="P' = J P J^T, FP32, one matrix per thread; J 36 + P 21 floats in, 21 out", rows=out)


SERVING_WORKLOAD = ("serving loop: Poisson arrivals, event sizes log-uniform 500-50,000 tracks (a pool of 64 "
                    "distinct events drawn at random per request), 17 barrel layers, 20% noise hits per layer, "
                    "best-hit build + final fit per event, 40 GB device-memory budget")


def result_arrays_layout(n, L):
    """(name, shape, dtype) of an event's result arrays, as kf_server_submit takes them."""
    return (("hit_idx", (L, n), np.int32), ("state", (6, n), np.float64), ("cov", (21, n), np.float64),
            ("chi2", (n,), np.float64), ("ndof", (n,), np.int32), ("status", (n,), np.uint32))


def result_slot_bytes(max_n, L):
    """Bytes of one slot of the serving client's ring of result buffers: the
    arrays of an event of up to max_n tracks, each at a 64-byte boundary within
    the slot, and the slot itself a multiple of 64 bytes, so that every array of
    every slot is aligned to its element size when the ring's base is (the
    server writes page-locked results in place only at that alignment)."""
    return sum((int(np.prod(sh)) * np.dtype(dt).itemsize + 63) // 64 * 64
               for _, sh, dt in result_arrays_layout(max_n, L))


def result_views(ring_buf, slot_bytes, slot, n, L):
    """The result arrays of an event of n tracks in slot `slot` of ring_buf (a
    flat uint8 array of whole slots)."""
    out, off = {}, slot * slot_bytes
    for k, sh, dt in result_arrays_layout(n, L):
        nb = int(np.prod(sh)) * np.dtype(dt).itemsize
        out[k] = ring_buf[off:off + nb].view(dt).reshape(sh)
        off += (nb + 63) // 64 * 64
    return out


def serving_sweep(ctx, geom, rates=None, pool_size=64, seconds_per_rate=4.0, memory="pinned", zero_copy=True):
    """Events through kf_server: first as fast as they can be submitted (the
    saturation throughput), then Poisson streams at fractions of it.  Latency is
    the library's own submit -> results-in-caller-arrays time per event.

    memory = "pinned": the client keeps its events and result buffers in
    page-locked memory allocated once (what a serving client does), so the
    server's kernels read the hits in place (zero_copy) and write the results
    straight into the caller's arrays.  memory = "pageable": ordinary numpy
    arrays, result arrays freshly allocated per request."""
    import torch
    from paper_1711_06571_gb300 import kf, synth

    def host(a):
        a = np.ascontiguousarray(a)
        return torch.from_numpy(a).pin_memory().numpy() if memory == "pinned" else a

    rng = np.random.default_rng(synth.BASE_SEED + 499)
    sizes = np.exp(rng.uniform(np.log(500), np.log(50000), pool_size)).astype(np.int64)
    pool = []
    for i, sz in enumerate(sizes):
        # particles simulated on the GPU (the host generator takes seconds per large event)
        ev = synth.gen_event(geom, int(sz), synth.BASE_SEED + 500 + i, device="cuda")
        L = len(ev["layers"])
        lay = [ev["layers"][l] if l >= 3 else None for l in range(L)]
        xs = [None if ly is None else host(np.asarray(ly["x"], np.float32)) for ly in lay]
        ys = [None if ly is None else host(np.asarray(ly["y"], np.float32)) for ly in lay]
        zs = [None if ly is None else host(np.asarray(ly["z"], np.float32)) for ly in lay]
        surf = [int(ly["surf"]) for ly in ev["layers"]]
        pool.append((ev["n"], surf, xs, ys, zs, host(np.asarray(ev["seed_hits"], np.float32)), L))
    max_events = 600
    ring = 96  # result buffers of the client: at most this many requests outstanding
    arena = None
    per = result_slot_bytes(max(p[0] for p in pool), pool[0][6])
    if memory == "pinned":
        # page-locked result buffers allocated once, reused round robin
        arena = torch.empty(per * ring, dtype=torch.uint8).pin_memory().numpy()
    srv = kf.kf_server_create(ctx, geom, kf.server_params(mem_budget_bytes=40 << 30, max_batches=4,
                                                          max_batch_events=16))

    def results(n, L, slot):
        if arena is None:
            return {k: np.empty(sh, dt) for k, sh, dt in result_arrays_layout(n, L)}
        return result_views(arena, per, slot % ring, n, L)

    def stream(rate, n_ev, seed):
        t_arr, _ = synth.serving_stream(seed, n_ev, rate if rate else 1.0)
        pick = np.random.default_rng(seed + 1).integers(0, pool_size, n_ev)
        kf.kf_server_stats_get(srv, reset=True)
        tickets, tracks, lag = [], 0, 0.0
        done_early = set()
        t0 = time.perf_counter()
        for i in range(n_ev):
            if rate:
                dt = t0 + t_arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                else:
                    lag = max(lag, -dt)
            n, surf, xs, ys, zs, sh, L = pool[pick[i]]
            if arena is not None and i >= ring:  # the buffer's previous request must be done
                if kf.kf_server_wait(srv, tickets[i - ring], 120000)[0] != kf.KF_OK:
                    raise RuntimeError("serving: an event failed")
                done_early.add(i - ring)
            res = results(n, L, i)
            while True:
                rc, t = kf.kf_server_submit(srv, n, surf, xs, ys, zs, sh, zero_copy=zero_copy, **res)
                if rc != kf.KF_EAGAIN:
                    break
                time.sleep(2e-4)
            if rc != kf.KF_OK:
                raise RuntimeError(f"kf_server_submit: {rc}")
            tickets.append(t)
            tracks += n
        t_sub = time.perf_counter() - t0
        bad = [t for i, t in enumerate(tickets)
               if i not in done_early and kf.kf_server_wait(srv, t, 120000)[0] != kf.KF_OK]
        wall = time.perf_counter() - t0
        st = kf.kf_server_stats_get(srv, reset=True)
        if bad or st["rc"] != kf.KF_OK:
            raise RuntimeError(f"serving: {len(bad)} events failed")
        return dict(rate_hz=rate if rate else "saturation", events=n_ev, tracks=int(tracks),
                    p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], max_ms=st["max_ms"], events_per_s=n_ev / wall,
                    tracks_per_s=tracks / wall, mean_batch_events=st["mean_batch_events"],
                    peak_device_bytes=int(st["peak_bytes_in_use"]), max_submit_lag_ms=lag * 1e3,
                    submit_loop_s=t_sub, wall_s=wall, batch_device_ms=st["batch_device_ms"],
                    copy_out_ms_per_batch=st["copy_out_ms"], submit_ms_per_event=st["stage_ms"])

    try:
        stream(None, 32, synth.BASE_SEED + 600)  # warm-up: pool, streams, pinned arena
        sat = stream(None, 400, synth.BASE_SEED + 601)
        if rates is None:
            rates = [f * sat["events_per_s"] for f in (0.25, 0.5, 0.8)]
        runs = [stream(r, int(min(max_events, max(60, r * seconds_per_rate))), synth.BASE_SEED + 610 + k)
                for k, r in enumerate(rates)]
    finally:
        kf.kf_server_destroy(srv)
    return dict(workload=SERVING_WORKLOAD, client_memory=memory, zero_copy=zero_copy, saturation=sat, rates=runs)


def run_reference(args, world, rank):
    """--impl reference: the FP64 oracle, as it stands, on the host cores."""
    from paper_1711_06571_gb300 import synth
    if rank != 0:
        return
    geom = synth.geometry("barrel17")
    threads = os.cpu_count() or 1
    n_sample = args.ref_sample
    if n_sample <= 0:
        # size each step so that the whole run takes about two minutes of oracle time
        tk = synth.gen_tracks(geom, 4000, rank_seed(0))
        _, _, dt = oracle_baseline(geom, tk, 4000, threads)
        per_step = 120.0 / max(1, args.steps + args.warmup)
        n_sample = int(min(200_000, max(500, 4000 * per_step / max(dt, 1e-4))))
    tk = synth.gen_tracks(geom, n_sample, rank_seed(0))
    vals = []
    for i in range(args.warmup + args.steps):
        v, upd, dt = oracle_baseline(geom, tk, n_sample, threads)
        if i >= args.warmup:
            vals.append((upd, dt))
    tot_upd = sum(u for u, _ in vals)
    tot_t = sum(d for _, d in vals)
    value = tot_upd / tot_t
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * tot_t / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD + f" (per step a sample of {n_sample} tracks)", tracks=n_sample),
                cpu_baseline=dict(value=value, unit=UNIT, cores=threads, kind="oracle",
                                  sample=f"{n_sample} tracks x up to 17 layers per step"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                runs_on=f"host cores only ({threads} threads); n_gpus is the launch's world size")
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_1711_06571_gb300 import build as kbuild, kf, run, synth
    kbuild.build()
    torch.cuda.set_device(local)
    ctx = run.context(local)
    geom = synth.geometry("barrel17")
    g = kf.make_geometry(geom)
    if args.part != "all":
        if rank == 0:
            if args.part == "build":
                r = build_bench(ctx, geom, args.steps, args.warmup)
            elif args.part == "uneven":
                r = uneven_bench(ctx, args.steps, args.warmup)
            elif args.part == "layout":
                r = layout_study(ctx)
            elif args.part == "nonideal":
                r = nonideal_bench(ctx, args.steps, args.warmup)
            else:
                rates = None if args.serving_rates == "auto" else [float(v) for v in args.serving_rates.split(",")]
                r = serving_sweep(ctx, geom, rates, memory=args.serving_memory, zero_copy=not args.serving_copy)
            print(json.dumps(dict(part=args.part, **r)), flush=True)
        return
    n = args.tracks
    tk = synth.gen_tracks(geom, n, rank_seed(rank))
    n = tk["n"]
    dh = run.hits_to_device(tk)
    seeds = run.make_seeds(ctx, g, dh)
    out = run.alloc_fit_out(n)
    stream = torch.cuda.current_stream()
    params = kf.fit_params(precision=kf.KF_PREC_MIXED)

    def step():
        kf.kf_make_seeds(ctx, g, n, dh["offsets"], dh["x"], dh["y"], dh["z"], seeds[0], seeds[1])
        kf.kf_fit(ctx, g, params, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                  out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    updates_per_step = int(((out["ndof"] + 5) // 2).clamp(min=0).sum().item())
    # per-launch timing of the fit kernel (events on the launching stream)
    fit_ms = []
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kf.kf_fit_timing(ctx, True)  # events around the two fit kernels of every timed step (no sync)
    e0.record(stream)
    for k in range(args.steps):
        kf.kf_make_seeds(ctx, g, n, dh["offsets"], dh["x"], dh["y"], dh["z"], seeds[0], seeds[1])
        ev[k][0].record(stream)
        kf.kf_fit(ctx, g, params, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                  out["state"], out["cov"], out["chi2"], out["ndof"], out["status"])
        ev[k][1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    n_timed, ms_phase1, ms_phase2 = kf.kf_fit_phase_times(ctx)
    kf.kf_fit_timing(ctx, False)
    ms_local = e0.elapsed_time(e1) / args.steps
    fit_ms = [a.elapsed_time(b) for a, b in ev]
    ms, total_updates, value = aggregate(ms_local, updates_per_step, world)

    # roofline of the dominant kernel, phase 2 (fit_loop_kernel): FP64 pipe (its
    # S solves), with the FP32 pipe and HBM beside it; phase 1 (fit_seed_kernel) apart
    nh = len(tk["x"])
    fp32_updates = updates_per_step - 3 * n
    fp64_flop2 = FP64_FLOP_PER_FP32_UPDATE * fp32_updates
    fp32_flop2 = FP32_FLOP_PER_FP32_UPDATE * fp32_updates
    fp64_flop1 = FP64_FLOP_PHASE1_BARREL * n
    bytes_alg = 4 * (n + 1) + 13 * nh + 25 * n + (48 + 168 + 8 + 4 + 4) * n  # the whole fit
    bytes2 = 4 * (n + 1) + 13 * (nh - 3 * n) + 4 * n + CARRY_BYTES_PER_TRACK * n + (48 + 168 + 8 + 4 + 4) * n
    fit_avg = float(np.mean(fit_ms))
    peak64 = kf.kf_measure_peak(ctx, 0)
    peak32 = kf.kf_measure_peak(ctx, 1)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach64 = fp64_flop2 / (ms_phase2 * 1e-3) / 1e12
    roofline = dict(bound="alu", pipe="fp64", kernel="fit_loop_kernel (phase 2: the FP32 layer loop)",
                    achieved=ach64, peak=peak64 / 1e12, unit="TFLOP/s", frac=ach64 / (peak64 / 1e12),
                    traffic=LOOP_KERNEL_DRAM_BYTES if n == N_TRACKS and LOOP_KERNEL_DRAM_BYTES else None,
                    peak_source="kf_measure_peak FP64 FMA chains (measured in this run); nominal 152 SMs x 2 "
                                "DFMA/clock x 2 FLOP x 2.07 GHz = 1.26 TFLOP/s",
                    kernel_ms_per_launch=ms_phase2, launches_timed=n_timed, fp64_flop_per_launch=fp64_flop2,
                    fp32=dict(achieved=fp32_flop2 / (ms_phase2 * 1e-3) / 1e12, peak=peak32 / 1e12,
                              unit="TFLOP/s", frac=fp32_flop2 / (ms_phase2 * 1e-3) / peak32,
                              flop_per_launch=fp32_flop2),
                    hbm=dict(achieved=bytes2 / (ms_phase2 * 1e-3) / 1e9, peak=hbm, unit="GB/s",
                             frac=bytes2 / (ms_phase2 * 1e-3) / 1e9 / hbm, bytes_per_launch=bytes2,
                             peak_source="MEASURED_PEAKS.json"),
                    phase1=dict(kernel="fit_seed_kernel (seed phase: double-float U-D, FP64 first transport)",
                                ms_per_launch=ms_phase1, fp64_flop_per_launch=fp64_flop1,
                                fp64_achieved=fp64_flop1 / (ms_phase1 * 1e-3) / 1e12),
                    fit_ms_per_launch=fit_avg, fit_bytes_per_launch=bytes_alg)

    if args.quick:
        if rank == 0:
            print(json.dumps(dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                                  warmup=args.warmup, ms_per_step=ms, fit_ms_per_launch=fit_avg,
                                  higher_is_better=True, roofline=roofline, clocks=clk)), flush=True)
        return

    # all-FP64 GPU path on the same inputs, for comparison
    p64 = kf.fit_params(precision=kf.KF_PREC_FP64)
    out64 = run.alloc_fit_out(n)
    for _ in range(2):
        kf.kf_fit(ctx, g, p64, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                  out64["state"], out64["cov"], out64["chi2"], out64["ndof"], out64["status"])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    reps = max(3, args.steps // 4)
    for _ in range(reps):
        kf.kf_fit(ctx, g, p64, n, seeds[0], seeds[1], dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"],
                  out64["state"], out64["cov"], out64["chi2"], out64["ndof"], out64["status"])
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b) / reps

    # outward-inward refit of the same tracks from the forward fit (kf_refit_inward)
    outr = run.alloc_fit_out(n)

    def refit():
        kf.kf_refit_inward(ctx, g, params, n, dh["offsets"], dh["layer"], dh["x"], dh["y"], dh["z"], out["state"],
                           out["cov"], seeds[1], out["ndof"], 100.0, outr["state"], outr["cov"], outr["chi2"],
                           outr["ndof"], outr["status"])
    for _ in range(2):
        refit()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        refit()
    b.record(stream)
    torch.cuda.synchronize()
    ms_refit = a.elapsed_time(b) / reps
    refit_updates = int(((outr["ndof"] + 5) // 2).clamp(min=0).sum().item())
    refit_line = dict(value=refit_updates / (ms_refit * 1e-3), unit=UNIT, ms_per_launch=ms_refit,
                      updates=refit_updates, what="reverse the used hits and the forward state (covariance x 100), "
                                                  "fit inwards, turn the result back")

    # end to end through the C ABI with host buffers (page-locked), copies inside
    hh = dict(offsets=torch.from_numpy(tk["offsets"]).pin_memory(), layer=torch.from_numpy(tk["layer"]).pin_memory(),
              x=torch.from_numpy(tk["x"]).pin_memory(), y=torch.from_numpy(tk["y"]).pin_memory(),
              z=torch.from_numpy(tk["z"]).pin_memory())
    ho = dict(state=torch.empty((6, n), dtype=torch.float64).pin_memory(),
              cov=torch.empty((21, n), dtype=torch.float64).pin_memory(),
              chi2=torch.empty(n, dtype=torch.float64).pin_memory(),
              ndof=torch.empty(n, dtype=torch.int32).pin_memory(),
              status=torch.empty(n, dtype=torch.int32).pin_memory())

    def e2e_step():
        kf.kf_fit_host(ctx, g, params, n, hh["offsets"], hh["layer"], hh["x"], hh["y"], hh["z"], ho["state"],
                       ho["cov"], ho["chi2"], ho["ndof"], ho["status"])

    for _ in range(max(2, args.warmup // 2)):
        e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    e2e_reps = max(3, args.steps // 2)
    for _ in range(e2e_reps):
        e2e_step()
    t_e2e = (time.perf_counter() - t0) / e2e_reps
    t_e2e = max_over_ranks(t_e2e, world)
    h2d = 4 * (n + 1) + 13 * nh
    d2h = (48 + 168 + 8 + 4 + 4) * n
    # the host results equal the device-resident run
    same = np.array_equal(ho["chi2"].numpy(), out["chi2"].cpu().numpy())
    # the same call with the covariance returned in FP32 (kf_tracks_out.cov_f32: the
    # mixed path's own covariance precision, 84 instead of 168 bytes per track)
    ho32 = torch.empty((21, n), dtype=torch.float32).pin_memory()

    def e2e_step32():
        kf.kf_fit_host(ctx, g, params, n, hh["offsets"], hh["layer"], hh["x"], hh["y"], hh["z"], ho["state"],
                       None, ho["chi2"], ho["ndof"], ho["status"], out_cov_f32=ho32)

    for _ in range(2):
        e2e_step32()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        e2e_step32()
    t_e2e32 = max_over_ranks((time.perf_counter() - t0) / e2e_reps, world)
    d2h32 = (48 + 84 + 8 + 4 + 4) * n

    # best-hit build of 10 events x 20,000 tracks
    build = build_bench(ctx, geom, max(10, args.steps // 4), max(3, args.warmup // 2))
    # uneven batch: barrel + disks, persistent kernel in a CUDA graph, autotuned
    uneven = uneven_bench(ctx, max(10, args.steps // 4), max(3, args.warmup // 2))
    # non-ideal barrel under measurement model 1
    nonideal = nonideal_bench(ctx, max(10, args.steps // 4), max(3, args.warmup // 2))

    # serving loop: events of mixed sizes through kf_server (one rank's GPU each)
    serving = None
    if not args.no_serving:
        rates = None if args.serving_rates == "auto" else [float(v) for v in args.serving_rates.split(",")]
        serving = serving_sweep(ctx, geom, rates, memory=args.serving_memory, zero_copy=not args.serving_copy)

    # the CPU leg (rank 0): the FP64 oracle checks a sample of this run's fits, then is timed
    parity = None
    cpu_baseline = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import parity as par
        m = 2000
        sub = dict(offsets=tk["offsets"][:m + 1], layer=tk["layer"], x=tk["x"], y=tk["y"], z=tk["z"], n=m)
        orc = oracle.fit(geom, sub, t1=m, threads=os.cpu_count() or 1)
        gsub = dict(state=out["state"][:, :m].t().cpu().numpy(), cov=run.unpack_cov(out["cov"][:, :m].cpu().numpy()),
                    chi2=out["chi2"][:m].cpu().numpy(), q=seeds[1][:m].cpu().numpy())
        orc = {k: (v[:m] if hasattr(v, "__len__") and len(v) >= m else v) for k, v in orc.items()}
        ok = (orc["status"] & 7) == 0
        res = par.compare_fits(gsub, orc, np.zeros(m, int), ok)
        parity = dict(tracks=int(ok.sum()), max_param_over_sigma=float(res["max_pull"].max()),
                      max_chi2_rel=float(res["chi2rel"].max()), max_cov_norm=float(res["dcov"].max()),
                      tolerance=dict(param_over_sigma=1e-3, chi2_rel=1e-3))
        # about 15 s of oracle work on all host cores: size the sample from a short probe
        threads = os.cpu_count() or 1
        _, _, dt0 = oracle_baseline(geom, tk, min(n, 50_000), threads)
        want = 50_000 * 15.0 / max(dt0, 1e-3)  # tracks in about 15 s
        n_sample = int(min(n, max(50_000, want)))
        passes = max(1, int(round(want / n_sample)))
        v, upd, dt = oracle_baseline(geom, tk, n_sample, threads, passes)
        # and on one host thread, about 5 s
        n1 = int(min(n, max(5_000, 50_000 * 5.0 / (max(dt0, 1e-3) * threads))))
        v1, upd1, dt1 = oracle_baseline(geom, tk, n1, 1)
        cpu_baseline = dict(value=v, unit=UNIT, cores=threads, kind="oracle",
                            sample=f"first {n_sample} tracks of the workload, {passes} pass(es) "
                                   f"({upd} updates, {dt:.1f} s)",
                            single_thread=dict(value=v1, unit=UNIT, cores=1,
                                               sample=f"first {n1} tracks ({upd1} updates, {dt1:.1f} s)"))

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32+f64",
                data="synthetic",
                config=dict(workload=WORKLOAD, tracks_per_gpu=n, layers=17, updates_per_step=updates_per_step,
                            precision="mixed: FP32 layer loop with FP64 S solves; seed phase in double-float "
                                      "U-D form (FP64 first transport)",
                            l2="inputs larger than L2 (hits 221 MB + outputs 232 MB per step)",
                            parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
                roofline=roofline, cpu_baseline=cpu_baseline,
                e2e=dict(value=total_updates / t_e2e, unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                         ms_per_step=t_e2e * 1e3, api="kf_fit_host", host_matches_device=bool(same),
                         cov_f32=dict(value=total_updates / t_e2e32, unit=UNIT, ms_per_step=t_e2e32 * 1e3,
                                      d2h_bytes_per_step=d2h32)),
                fp64_path=dict(value=updates_per_step * world / (ms64 * 1e-3), unit=UNIT, fit_ms=ms64,
                               speedup_of_mixed=ms64 / fit_avg),
                gpu_launches=6 * args.steps, clocks=clk, parity_vs_oracle=parity, build=build, uneven_batch=uneven,
                refit_inward=refit_line, nonideal=nonideal, serving=serving)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
