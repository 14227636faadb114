"""The N > 1 path of bench.py on CPU with the gloo backend, world size 2.

The fit shards into independent tracks, so ranks exchange nothing on the data
path: each fits its own tracks (its own seed), and the only collectives are
the timing and unit reductions of the whole-job figure.  These tests run two
ranks as processes on the host."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms_local = [3.0, 5.0][rank]        # the slower rank sets the job time
        units_local = [1000, 3000][rank]   # units each rank processed
        ms, total, value = bench.aggregate(ms_local, units_local, world)
        bench.barrier(world)
        out[rank] = (ms, total, value, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, total, value, _ = out[r]
        assert ms == 5.0 and total == 4000
        assert value == pytest.approx(4000 / 5e-3)
    assert out[0][3] != out[1][3]  # every rank draws its own tracks


def test_rank_shards_are_distinct_workloads():
    from paper_1711_06571_gb300 import synth
    sys.path.insert(0, ROOT)
    import bench
    g = synth.geometry("barrel17")
    a = synth.gen_tracks(g, 50, bench.rank_seed(0))
    b = synth.gen_tracks(g, 50, bench.rank_seed(1))
    assert not (a["x"][:10] == b["x"][:10]).all()


def test_reference_arm_under_torchrun_two_ranks(tmp_path):
    """--impl reference under torchrun: rank 0 alone times the oracle and
    prints one JSON line; the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-sample", "300"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=str(tmp_path), env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "updates/s"
    assert d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
