"""Seeded synthetic workloads shaped like the paper's toy studies (Sec. 3, Sec. 4.1).

This module makes inputs only.  It simulates "truth": charged particles from the
origin in a uniform longitudinal field, crossing an ideal barrel of cylinders
(optionally closed by end-cap disks, the barrel-plus-disks detector of Sec. 4.1),
with a multiple-scattering kick at every crossing and Gaussian hit smearing.
It holds no step of the Kalman filter: it does not fit, seed, bin or select.
The crossing points are computed here by intersecting the helix circle with
the cylinder (angles about the helix centre), independently of both the
oracle and the CUDA library, so the truth it records can pin them.

All randomness comes from one ``torch.Generator`` seeded by the caller; the
same (seed, device) always gives the same arrays.
"""
from __future__ import annotations

import math

import numpy as np
import torch

KAPPA = 0.299792458e-2      # GeV / (T cm)
PION_MASS = 0.13957039      # GeV
BZ = 3.8                    # T
SIG_RPHI = 0.01             # cm
SIG_Z = 0.1                 # cm
SIG_R_DISK = 0.1            # cm, radial resolution on disks
X_X0 = 0.02                 # radiation lengths per layer at normal incidence
BASE_SEED = 1711065710


def barrel_half_length(R: float) -> float:
    """Half length of a barrel cylinder of radius R (cm): 30 + 1.6 R."""
    return 30.0 + 1.6 * R


def _barrel(R, x_x0=X_X0):
    return dict(kind=0, pos=float(R), half_or_rin=barrel_half_length(R), r_out=0.0, x_x0=x_x0,
                sig_n=SIG_RPHI, sig_rphi=SIG_RPHI, sig_3=SIG_Z)


def _disk(Z, x_x0=X_X0):
    return dict(kind=1, pos=float(Z), half_or_rin=abs(Z) / 7.0 + 5.0, r_out=100.0, x_x0=x_x0,
                sig_n=SIG_RPHI, sig_rphi=SIG_RPHI, sig_3=SIG_R_DISK)


def geometry(name: str, x_x0: float = X_X0, bz: float = BZ) -> dict:
    """Detector geometries of the workloads.

    barrel10: 10 cylinders at R = 4, 8, ..., 40 cm (1,000-track fit).
    barrel17: 17 cylinders at R = 4 + 6 i, i = 0..16 (fit at scale, best-hit building, serving).
    lids:     barrel17 plus 2 x 12 disks at |z| = 30 + 240 j / 11, j = 0..11, r in [|z|/7 + 5, 100].
    barrel17s: barrel17 whose layers are rings of modules at alternating radii R - 0.25 and
              R + 0.25 cm (sectors about 10 cm wide in r-phi): a non-ideal geometry where hits
              do not lie on the layer's average cylinder (Sec. 4.1).  The surfaces carry the
              average radius; "stagger" and "n_mod" describe the modules for the generator.
    """
    if name == "barrel10":
        surfs = [_barrel(4.0 * (i + 1), x_x0) for i in range(10)]
    elif name == "barrel17":
        surfs = [_barrel(4.0 + 6.0 * i, x_x0) for i in range(17)]
    elif name == "barrel17s":
        surfs = [_barrel(4.0 + 6.0 * i, x_x0) for i in range(17)]
        for sf in surfs:
            sf["stagger"] = 0.25
            sf["dr"] = 0.25  # the layer's radial half-extent, as a reconstruction sees it
            sf["n_mod"] = max(4, 2 * int(round(math.pi * sf["pos"] / 10.0)))  # even: radii alternate
    elif name == "lids":
        surfs = [_barrel(4.0 + 6.0 * i, x_x0) for i in range(17)]
        for sgn in (1.0, -1.0):
            for j in range(12):
                surfs.append(_disk(sgn * (30.0 + 240.0 * j / 11.0), x_x0))
    else:
        raise ValueError(f"unknown geometry {name!r}")
    return dict(name=name, bz=bz, mass=PION_MASS, surfaces=surfs)


def _highland(p, t, mass):
    # PDG Highland formula, unit charge, p in GeV
    beta = p / torch.sqrt(p * p + mass * mass)
    return 0.0136 / (beta * p) * torch.sqrt(t) * (1.0 + 0.038 * torch.log(t / (beta * beta)))


def _wrap(a):
    return torch.remainder(a + math.pi, 2.0 * math.pi) - math.pi


class _Tracks:
    """Vectorised truth state of a batch of particles."""

    def __init__(self, q, pt, phi, theta, dev):
        n = q.shape[0]
        self.q = q
        self.pt = pt
        self.phi = phi
        self.theta = theta
        self.x = torch.zeros(n, dtype=torch.float64, device=dev)
        self.y = torch.zeros_like(self.x)
        self.z = torch.zeros_like(self.x)
        self.turn = torch.zeros_like(self.x)  # accumulated |c| s

    def curv(self, bz):
        return -self.q * KAPPA * bz / self.pt


def _barrel_s(tr, idx, c, R):
    """Transverse path to the cylinder R for tracks idx: first crossing, via the helix
    centre and the angle swept about it.  Returns s (inf where none)."""
    x, y, phi = tr.x[idx], tr.y[idx], tr.phi[idx]
    xc = x - torch.sin(phi) / c
    yc = y + torch.cos(phi) / c
    rho = 1.0 / c.abs()
    d = torch.sqrt(xc * xc + yc * yc)
    a = (R * R - rho * rho + d * d) / (2.0 * d)
    h2 = R * R - a * a
    ok = (h2 >= 0) & ((x * x + y * y) < R * R)
    h = torch.sqrt(torch.clamp(h2, min=0.0))
    psi0 = torch.atan2(y - yc, x - xc)
    best = torch.full_like(x, math.inf)
    for sg in (1.0, -1.0):
        X = a * xc / d - sg * h * yc / d
        Y = a * yc / d + sg * h * xc / d
        psi = torch.atan2(Y - yc, X - xc)
        dpsi = torch.where(c > 0, psi - psi0, psi0 - psi)
        dpsi = torch.remainder(dpsi, 2.0 * math.pi)
        s = dpsi * rho
        s = torch.where(ok & (s > 1e-9), s, torch.full_like(s, math.inf))
        best = torch.minimum(best, s)
    return best


def _move(tr, idx, c, s):
    """Move tracks idx along their helix by transverse path s (centre form)."""
    x, y, phi = tr.x[idx], tr.y[idx], tr.phi[idx]
    xc = x - torch.sin(phi) / c
    yc = y + torch.cos(phi) / c
    phi1 = phi + c * s
    tr.x[idx] = xc + torch.sin(phi1) / c
    tr.y[idx] = yc - torch.cos(phi1) / c
    tr.z[idx] = tr.z[idx] + s / torch.tan(tr.theta[idx])
    tr.phi[idx] = _wrap(phi1)


def _disk_s(tr, idx, Z):
    cot = 1.0 / torch.tan(tr.theta[idx])
    s = (Z - tr.z[idx]) / cot
    return torch.where(s > 1e-9, s, torch.full_like(s, math.inf))


def _xy_after(tr, idx, c, s):
    """Transverse position of tracks idx after a transverse path s."""
    x, y, phi = tr.x[idx], tr.y[idx], tr.phi[idx]
    xc = x - torch.sin(phi) / c
    yc = y + torch.cos(phi) / c
    phi1 = phi + c * s
    return xc + torch.sin(phi1) / c, yc - torch.cos(phi1) / c


def _radius_after(tr, idx, c, s):
    x, y, phi = tr.x[idx], tr.y[idx], tr.phi[idx]
    xc = x - torch.sin(phi) / c
    yc = y + torch.cos(phi) / c
    phi1 = phi + c.unsqueeze(-1) * s if s.dim() > 1 else phi + c * s
    if s.dim() > 1:
        X = xc.unsqueeze(-1) + torch.sin(phi1) / c.unsqueeze(-1)
        Y = yc.unsqueeze(-1) - torch.cos(phi1) / c.unsqueeze(-1)
        Zp = tr.z[idx].unsqueeze(-1) + s / torch.tan(tr.theta[idx]).unsqueeze(-1)
    else:
        X = xc + torch.sin(phi1) / c
        Y = yc - torch.cos(phi1) / c
        Zp = tr.z[idx] + s / torch.tan(tr.theta[idx])
    return torch.sqrt(X * X + Y * Y), Zp


def gen_tracks(geom: dict, n: int, seed: int, eta_max: float = 1.0, pt_min: float = 0.5, pt_max: float = 10.0,
               ms_on: bool = True, smear: bool = True, device: str = "cpu", min_hits: int = 3,
               keep_truth: bool = False, max_hits: int = 64):
    """Simulate n particles from the origin and return their hits as CSR in path order.

    Particles: charge +-1 equiprobable, pT log-uniform in [pt_min, pt_max], phi uniform,
    eta uniform in (-eta_max, eta_max), theta = 2 atan(exp(-eta)).  At each crossing the hit is
    recorded (smeared along the surface: r-phi by sig_rphi, z by sig_z on barrels, r by sig_r on
    disks) and then the direction is kicked by the Highland angle (theta += N(0, th0),
    phi += N(0, th0 / sin theta)); pT is held fixed.  Only outward crossings count and a track ends at
    its apex (once it heads inwards, or after half a turn of transverse path).  Tracks with fewer than min_hits hits are dropped.  Returns numpy arrays: offsets (n+1), layer (uint8), x, y, z (float32) and, with
    keep_truth, truth (per hit: state (x, y, z, 1/pT, phi, theta) after the kick) and truth_q.
    """
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=dev)
    bz, mass = geom["bz"], geom["mass"]
    surfs = geom["surfaces"]
    q = torch.where(torch.rand(n, generator=g, **f64) < 0.5, -1.0, 1.0).to(torch.float64)
    lpt = math.log(pt_min) + (math.log(pt_max) - math.log(pt_min)) * torch.rand(n, generator=g, **f64)
    pt = torch.exp(lpt)
    phi = (2.0 * torch.rand(n, generator=g, **f64) - 1.0) * math.pi
    eta = (2.0 * torch.rand(n, generator=g, **f64) - 1.0) * eta_max
    theta = 2.0 * torch.atan(torch.exp(-eta))
    tr = _Tracks(q, pt, phi, theta, dev)

    barrels = [i for i, s in enumerate(surfs) if s["kind"] == 0]
    disks = [i for i, s in enumerate(surfs) if s["kind"] == 1]
    barrel_only = len(disks) == 0
    H = len(barrels) if barrel_only else max_hits
    HX = torch.zeros((n, H), **f64)
    HY = torch.zeros_like(HX)
    HZ = torch.zeros_like(HX)
    HL = torch.full((n, H), -1, dtype=torch.int64, device=dev)
    TR = torch.zeros((n, H, 6), **f64) if keep_truth else None
    alive = torch.ones(n, dtype=torch.bool, device=dev)
    nh = torch.zeros(n, dtype=torch.int64, device=dev)
    R_b = torch.tensor([surfs[i]["pos"] for i in barrels], **f64)
    L_b = torch.tensor([surfs[i]["half_or_rin"] for i in barrels], **f64)

    for step in range(H):
        idx = torch.nonzero(alive).squeeze(1)
        if idx.numel() == 0:
            break
        c = tr.curv(bz)[idx]
        if barrel_only:
            sf = surfs[barrels[step]]
            R = sf["pos"]
            s = _barrel_s(tr, idx, c, torch.full_like(c, R))
            if sf.get("stagger", 0.0) > 0.0:
                # the module the track meets: its sector from the azimuth at the average
                # radius, its radius R -+ stagger alternating with the sector
                fin = torch.isfinite(s)
                xa, ya = _xy_after(tr, idx, c, torch.where(fin, s, torch.zeros_like(s)))
                sec = torch.floor((torch.atan2(ya, xa) + math.pi) * (sf["n_mod"] / (2.0 * math.pi)))
                sec = torch.remainder(sec, sf["n_mod"])
                Rm = R + sf["stagger"] * torch.where(torch.remainder(sec, 2) == 1, 1.0, -1.0).to(torch.float64)
                s = torch.where(fin, _barrel_s(tr, idx, c, Rm), s)
            surf_id = torch.full_like(idx, barrels[step])
        else:
            # smallest positive path over every surface whose crossing lies on the surface
            best_s = torch.full_like(c, math.inf)
            surf_id = torch.full_like(idx, -1)
            for bi, si in enumerate(barrels):
                sb = _barrel_s(tr, idx, c, R_b[bi].expand_as(c))
                fin = torch.isfinite(sb)
                if fin.any():
                    _, zz = _radius_after(tr, idx, c, torch.where(fin, sb, torch.zeros_like(sb)))
                    sb = torch.where(fin & (zz.abs() <= L_b[bi]), sb, torch.full_like(sb, math.inf))
                better = sb < best_s
                best_s = torch.where(better, sb, best_s)
                surf_id = torch.where(better, torch.full_like(surf_id, si), surf_id)
            for si in disks:
                Z = surfs[si]["pos"]
                sd = _disk_s(tr, idx, Z)
                fin = torch.isfinite(sd)
                if fin.any():
                    rr, _ = _radius_after(tr, idx, c, torch.where(fin, sd, torch.zeros_like(sd)))
                    ok = fin & (rr >= surfs[si]["half_or_rin"]) & (rr <= surfs[si]["r_out"])
                    sd = torch.where(ok, sd, torch.full_like(sd, math.inf))
                better = sd < best_s
                best_s = torch.where(better, sd, best_s)
                surf_id = torch.where(better, torch.full_like(surf_id, si), surf_id)
            s = best_s
        hit = torch.isfinite(s)
        if barrel_only:
            zlim = torch.tensor(surfs[barrels[step]]["half_or_rin"], **f64)
        alive_next = alive.clone()
        alive_next[idx[~hit]] = False
        ih = idx[hit]
        if ih.numel() == 0:
            alive = alive_next
            break
        # a track ends at its first apex: no crossing beyond half a turn of
        # transverse path (loopers spiralling along z are not in these workloads)
        turn = tr.turn[ih] + (c[hit] * s[hit]).abs()
        past = turn > math.pi
        if past.any():
            alive_next[ih[past]] = False
            keep = ~past
            ih, s_h, c_h, sid_h = ih[keep], s[hit][keep], c[hit][keep], surf_id[hit][keep]
            turn = turn[keep]
        else:
            s_h, c_h, sid_h = s[hit], c[hit], surf_id[hit]
        if ih.numel() == 0:
            alive = alive_next
            continue
        tr.turn[ih] = turn
        _move(tr, ih, c_h, s_h)
        sid = sid_h
        if not barrel_only:
            is_disk = torch.tensor([surfs[int(k)]["kind"] == 1 for k in range(len(surfs))],
                                   device=dev)[sid]
            zd = torch.tensor([surfs[int(k)]["pos"] for k in range(len(surfs))], **f64)[sid]
            tr.z[ih] = torch.where(is_disk, zd, tr.z[ih])
        else:
            is_disk = torch.zeros(ih.numel(), dtype=torch.bool, device=dev)
            out_z = tr.z[ih].abs() > zlim
            if out_z.any():
                alive_next[ih[out_z]] = False
                keep = ~out_z
                ih, sid, is_disk = ih[keep], sid[keep], is_disk[keep]
        # record the (smeared) hit
        X, Y, Zz = tr.x[ih], tr.y[ih], tr.z[ih]
        rr = torch.sqrt(X * X + Y * Y)
        if smear:
            g1 = torch.randn(ih.numel(), generator=g, **f64)
            g2 = torch.randn(ih.numel(), generator=g, **f64)
            dpos = g1 * SIG_RPHI / rr
            cd, sd_ = torch.cos(dpos), torch.sin(dpos)
            Xs, Ys = X * cd - Y * sd_, X * sd_ + Y * cd
            # disks: radial smear, barrels: z smear
            scale = torch.where(is_disk, (rr + g2 * SIG_R_DISK) / rr, torch.ones_like(rr))
            Xs, Ys = Xs * scale, Ys * scale
            Zs = torch.where(is_disk, Zz, Zz + g2 * SIG_Z)
        else:
            Xs, Ys, Zs = X, Y, Zz
        col = nh[ih]
        HX[ih, col] = Xs
        HY[ih, col] = Ys
        HZ[ih, col] = Zs
        HL[ih, col] = sid
        # scattering kick after the hit
        if ms_on:
            th = tr.theta[ih]
            sn = torch.sin(th)
            p = tr.pt[ih] / sn
            if True:
                cos_b = sn * (X * torch.cos(tr.phi[ih]) + Y * torch.sin(tr.phi[ih])) / rr
                cos_a = torch.where(is_disk, torch.cos(th), cos_b).abs().clamp(min=0.05)
            xx0 = torch.tensor([surfs[int(k)]["x_x0"] for k in range(len(surfs))], **f64)[sid]
            t = xx0 / cos_a
            th0 = _highland(p, t, mass)
            th0 = torch.where(xx0 > 0, th0, torch.zeros_like(th0))
            k1 = torch.randn(ih.numel(), generator=g, **f64)
            k2 = torch.randn(ih.numel(), generator=g, **f64)
            tr.theta[ih] = th + k1 * th0
            tr.phi[ih] = _wrap(tr.phi[ih] + k2 * th0 / sn)
        if keep_truth:
            TR[ih, col] = torch.stack([tr.x[ih], tr.y[ih], tr.z[ih], 1.0 / tr.pt[ih], tr.phi[ih], tr.theta[ih]],
                                      dim=1)
        nh[ih] += 1
        # a track ends at its apex: once it heads inwards it would only loop back
        inward = (tr.x[ih] * torch.cos(tr.phi[ih]) + tr.y[ih] * torch.sin(tr.phi[ih])) <= 0
        alive_next[ih[inward]] = False
        alive = alive_next
        if not barrel_only:
            # stop tracks that left the tracker volume
            out = (torch.sqrt(tr.x ** 2 + tr.y ** 2) >= 100.0 - 1e-9) | (tr.z.abs() >= 270.0 - 1e-9)
            alive = alive & ~out & (nh < H)

    keep = nh >= min_hits
    nh_k = nh[keep]
    mask = torch.arange(H, device=dev).unsqueeze(0) < nh_k.unsqueeze(1)
    offsets = torch.zeros(int(keep.sum()) + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(nh_k, 0)
    out = dict(
        offsets=offsets.to(torch.int32).cpu().numpy(),
        layer=HL[keep][mask].to(torch.uint8).cpu().numpy(),
        x=HX[keep][mask].to(torch.float32).cpu().numpy(),
        y=HY[keep][mask].to(torch.float32).cpu().numpy(),
        z=HZ[keep][mask].to(torch.float32).cpu().numpy(),
        n=int(keep.sum()),
    )
    if keep_truth:
        out["truth"] = TR[keep][mask].cpu().numpy()
        out["truth_q"] = q[keep].to(torch.int8).cpu().numpy()
        out["truth_pt"] = pt[keep].cpu().numpy()
    return out


def gen_event(geom: dict, n_signal: int, seed: int, noise_frac: float = 0.2, eta_max: float = 1.0,
              pt_min: float = 0.5, pt_max: float = 10.0, device: str = "cpu", ms_on: bool = True):
    """One best-hit-building event on a barrel geometry: n_signal particles plus, on every
    layer, round(noise_frac * signal hits on that layer) noise hits uniform in phi and z over
    the layer.  Each layer's hits are shuffled; ``truth`` gives the particle index of each hit
    (-1 for noise).  Seeds are the particles' hits on layers 0, 1, 2 (original indices in
    ``seed_idx``, coordinates in ``seed_hits``)."""
    surfs = geom["surfaces"]
    nl = len(surfs)
    trk = gen_tracks(geom, n_signal, seed, eta_max=eta_max, pt_min=pt_min, pt_max=pt_max, ms_on=ms_on,
                     device=device, min_hits=3)
    n = trk["n"]
    rng = np.random.default_rng(int(seed) + 7919)
    off = trk["offsets"].astype(np.int64)
    nh = np.diff(off)
    tid = np.repeat(np.arange(n), nh)
    lay = trk["layer"].astype(np.int64)
    layers = []
    where = np.full((n, nl), -1, np.int64)   # original index of particle t's hit on layer l
    for l in range(nl):
        sel = np.nonzero(lay == l)[0]
        ns = len(sel)
        nn = int(round(noise_frac * ns))
        R = surfs[l]["pos"]
        Lz = surfs[l]["half_or_rin"]
        ph = rng.uniform(-math.pi, math.pi, nn)
        x = np.concatenate([trk["x"][sel], (R * np.cos(ph)).astype(np.float32)])
        y = np.concatenate([trk["y"][sel], (R * np.sin(ph)).astype(np.float32)])
        z = np.concatenate([trk["z"][sel], rng.uniform(-Lz, Lz, nn).astype(np.float32)])
        truth = np.concatenate([tid[sel], np.full(nn, -1, np.int64)])
        perm = rng.permutation(ns + nn)
        x, y, z, truth = x[perm], y[perm], z[perm], truth[perm]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(ns + nn)
        where[tid[sel], l] = inv[:ns]
        layers.append(dict(x=x, y=y, z=z, truth=truth.astype(np.int32), surf=l))
    seed_idx = where[:, :3].astype(np.int32)
    seed_hits = np.zeros((n, 3, 3), np.float32)
    for k in range(3):
        ly = layers[k]
        seed_hits[:, k, 0] = ly["x"][seed_idx[:, k]]
        seed_hits[:, k, 1] = ly["y"][seed_idx[:, k]]
        seed_hits[:, k, 2] = ly["z"][seed_idx[:, k]]
    return dict(layers=layers, seed_idx=seed_idx, seed_hits=seed_hits, truth_where=where.astype(np.int32), n=n)


def serving_stream(seed: int, n_events: int, rate_hz: float, size_min: int = 500, size_max: int = 50000):
    """Poisson arrival times (s) and log-uniform event sizes (tracks) of a serving run."""
    rng = np.random.default_rng(int(seed))
    gaps = rng.exponential(1.0 / rate_hz, n_events)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(math.log(size_min), math.log(size_max), n_events)).astype(np.int64)
    return t, sizes
