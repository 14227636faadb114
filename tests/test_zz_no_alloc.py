"""The allocation-free binning entry point, for callers that cannot call
cudaMalloc (a host framework that owns all device memory, a real-time process
with a fixed footprint).  Called through the C ABI; its output must equal
kf_bin_hits' on the same inputs, on two calls in a row (the shared scratch
array keeps the previous call's contents).  Collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_1711_06571_gb300 import kf, run, synth

pytestmark = pytest.mark.gpu


def _layer(ev, g, L):
    ly = ev["layers"][L]
    dev = torch.device("cuda")
    x, y, z = (torch.from_numpy(np.ascontiguousarray(ly[k], np.float32)).to(dev) for k in ("x", "y", "z"))
    return x, y, z, float(g["surfaces"][L]["half_or_rin"])


def _bin_ctx(ctx, x, y, z, half):
    n = x.numel()
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(kf.KF_NBINS + 1, dtype=torch.int32, device="cuda")
    packed = torch.empty((max(n, 1), 4), dtype=torch.float32, device="cuda")
    kf.kf_bin_hits(ctx, n, x, y, z, half, perm, off, packed)
    return perm[:n], off, packed[:n]


def _bin_static(x, y, z, half):
    n = x.numel()
    perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    off = torch.full((kf.KF_NBINS + 1,), -7, dtype=torch.int32, device="cuda")
    packed = torch.zeros((max(n, 1), 4), dtype=torch.float32, device="cuda")
    rc = kf.kf_bin_hits_static(n, x, y, z, half, perm, off, packed)
    assert rc == kf.KF_OK
    return perm[:n], off, packed[:n]


def test_static_binning_equals_workspace_binning_twice():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1711_06571_gb300 import build
    build.build()
    ctx = run.context(0)
    g = synth.geometry("barrel17")
    ev = synth.gen_event(g, 20000, synth.BASE_SEED + 3)
    # two calls in a row on different layers (the second one sees the first one's
    # leftovers in the shared array), then the first layer again
    for L in (16, 4, 16):
        x, y, z, half = _layer(ev, g, L)
        pa, oa, ka = _bin_ctx(ctx, x, y, z, half)
        pb, ob, kb = _bin_static(x, y, z, half)
        torch.cuda.synchronize()
        assert torch.equal(oa, ob)
        assert torch.equal(pa, pb)
        assert torch.equal(ka.view(torch.int32), kb.view(torch.int32))


def test_static_binning_limits():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_1711_06571_gb300 import build
    build.build()
    dev = torch.device("cuda")
    # largest allowed size works, one more is refused before any GPU work
    n = kf.KF_STATIC_MAX_HITS
    phi = torch.linspace(-3.1, 3.1, n, device=dev)
    x, y = (30 * torch.cos(phi)).float(), (30 * torch.sin(phi)).float()
    z = torch.zeros(n, device=dev)
    pb, ob, _ = _bin_static(x, y, z, 40.0)
    torch.cuda.synchronize()
    assert int(ob[-1].item()) == n
    assert torch.all(pb[1:] >= 0)
    big = torch.zeros(n + 1, device=dev)
    perm = torch.empty(n + 1, dtype=torch.int32, device=dev)
    off = torch.empty(kf.KF_NBINS + 1, dtype=torch.int32, device=dev)
    assert kf.kf_bin_hits_static(n + 1, big, big, big, 40.0, perm, off) == kf.KF_ESIZE
    # host memory is refused
    hx = torch.zeros(10)
    assert kf.kf_bin_hits_static(10, hx, hx, hx, 40.0, perm, off) == kf.KF_EINVAL
    # empty layer: offsets all zero
    e = torch.zeros(0, device=dev)
    assert kf.kf_bin_hits_static(0, e, e, e, 40.0, perm, off) == kf.KF_OK
    torch.cuda.synchronize()
    assert int(off.abs().sum().item()) == 0
