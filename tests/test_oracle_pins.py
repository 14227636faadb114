"""Pins for the FP64 oracle: each test checks an oracle routine against something
other than the oracle itself (closed forms, finite differences, the information
form of the update, a global least-squares fit, brute force, statistics on
simulated truth).  CPU only."""
import math
import os

import numpy as np
import pytest

import parity

from paper_1711_06571_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
KAPPA = 0.299792458e-2
BZ = 3.8


def _barrel(R, x_x0=0.02):
    return dict(kind=0, pos=R, half_or_rin=30 + 1.6 * R, r_out=0.0, x_x0=x_x0, sig_n=0.01, sig_rphi=0.01,
                sig_3=0.1)


def _disk(Z, x_x0=0.02):
    return dict(kind=1, pos=Z, half_or_rin=abs(Z) / 7 + 5, r_out=100.0, x_x0=x_x0, sig_n=0.01, sig_rphi=0.01,
                sig_3=0.1)


# ---------------------------------------------------------------------- Highland (Sec. 2)

def test_highland_pdg_values(oracle_mod):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "highland_pdg.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for p, t, th0 in rows:
        got = oracle_mod.highland(float(p), synth.PION_MASS, float(t))
        assert got == pytest.approx(float(th0), rel=2e-7)


def test_highland_scaling_invariants(oracle_mod):
    # massless: beta = 1, so theta0 is exactly proportional to 1/p
    a = oracle_mod.highland(1.0, 0.0, 0.02)
    b = oracle_mod.highland(4.0, 0.0, 0.02)
    assert a / b == pytest.approx(4.0, rel=1e-14)
    # at beta = 1 and t = 1 the log term vanishes: theta0 = 13.6 MeV / p
    assert oracle_mod.highland(2.0, 0.0, 1.0) == pytest.approx(0.0136 / 2.0, rel=1e-14)
    # infinite momentum: no scattering
    assert oracle_mod.highland(math.inf, 0.14, 0.02) == 0.0


def test_ms_noise_placement(oracle_mod):
    # barrel crossed at normal incidence, theta = 60 deg: t = x/X0 / sin(theta)
    th = math.pi / 3
    st = np.array([10.0, 0.0, 0.0, 1.0, 0.0, th])
    rc, P = oracle_mod.ms_noise(st, 0.13957039, _barrel(10.0), np.zeros((6, 6)))
    p = 1.0 / math.sin(th)
    th0 = oracle_mod.highland(p, 0.13957039, 0.02 / math.sin(th))
    expect = np.zeros((6, 6))
    expect[5, 5] = th0 ** 2
    expect[4, 4] = th0 ** 2 / math.sin(th) ** 2
    assert rc == 0
    np.testing.assert_allclose(P, expect, rtol=1e-13, atol=0)
    # disk: incidence from cos(theta)
    st = np.array([10.0, 0.0, 50.0, 1.0, 0.0, 0.3])
    rc, P = oracle_mod.ms_noise(st, 0.13957039, _disk(50.0), np.zeros((6, 6)))
    th0 = oracle_mod.highland(1.0 / math.sin(0.3), 0.13957039, 0.02 / math.cos(0.3))
    assert P[5, 5] == pytest.approx(th0 ** 2, rel=1e-13)
    # grazing guard
    st = np.array([10.0, 0.0, 0.0, 1.0, math.pi / 2, math.pi / 2])
    rc, P = oracle_mod.ms_noise(st, 0.13957039, _barrel(10.0), np.zeros((6, 6)))
    assert rc == oracle_mod.ST_GRAZING
    th0 = oracle_mod.highland(1.0, 0.13957039, 0.02 / 0.05)
    assert P[5, 5] == pytest.approx(th0 ** 2, rel=1e-13)


# ---------------------------------------------------------------------- helix (Sec. 3, Sec. 4.1)

@pytest.mark.parametrize("q", [-1, 1])
@pytest.mark.parametrize("pt", [0.5, 1.3, 10.0])
def test_barrel_crossing_from_origin_closed_form(oracle_mod, q, pt):
    # a helix from the origin crosses r = R after s = 2 rho asin(R / (2 rho)), at azimuth
    # phi0 + c s / 2 (the chord direction), with direction phi0 + c s
    phi0, th = 0.7, 1.1
    st = np.array([0.0, 0.0, 0.0, 1.0 / pt, phi0, th])
    c = -q * KAPPA * BZ / pt
    rho = 1.0 / abs(c)
    for R in (4.0, 22.0, 58.0):
        if R > 2 * rho:
            continue
        rc, out, _ = oracle_mod.propagate(st, q, BZ, _barrel(R), want_jac=False)
        s = 2 * rho * math.asin(R / (2 * rho))
        assert rc == 0
        assert out[0] == pytest.approx(R * math.cos(phi0 + c * s / 2), abs=1e-11)
        assert out[1] == pytest.approx(R * math.sin(phi0 + c * s / 2), abs=1e-11)
        assert out[2] == pytest.approx(s / math.tan(th), abs=1e-11)
        assert out[4] == pytest.approx(phi0 + c * s, abs=1e-13)


def test_barrel_unreachable(oracle_mod):
    # pT = 0.5 GeV: rho = 43.9 cm, the circle from the origin never gets beyond 2 rho = 87.8 cm
    st = np.array([0.0, 0.0, 0.0, 2.0, 0.3, 1.2])
    rc, _, _ = oracle_mod.propagate(st, 1, BZ, _barrel(94.0), want_jac=False)
    assert rc == oracle_mod.ST_NO_INTERSECT
    rc, _, _ = oracle_mod.propagate(st, 1, BZ, _barrel(82.0), want_jac=False)
    assert rc == 0


def test_disk_crossing_closed_form(oracle_mod):
    q, pt, phi0, th = 1, 0.8, -2.0, 0.4
    st = np.array([0.0, 0.0, 0.0, 1.0 / pt, phi0, th])
    c = -q * KAPPA * BZ / pt
    Z = 60.0
    rc, out, _ = oracle_mod.propagate(st, q, BZ, _disk(Z), want_jac=False)
    s = Z * math.tan(th)
    assert rc == 0
    assert out[2] == Z
    assert math.hypot(out[0], out[1]) == pytest.approx(2 / abs(c) * abs(math.sin(c * s / 2)), rel=1e-12)
    assert out[4] == pytest.approx(phi0 + c * s, abs=1e-13)
    # a disk behind the state is reached backwards, s = -Z tan(theta) < 0
    rc, out, _ = oracle_mod.propagate(st, q, BZ, _disk(-Z), want_jac=False)
    assert rc == 0 and out[2] == -Z
    assert out[4] == pytest.approx(phi0 - c * s, abs=1e-13)
    # theta = pi/2 (up to rounding) never meets a disk
    rc, _, _ = oracle_mod.propagate(np.array([0, 0, 0, 1.0, 0.1, math.pi / 2]), q, BZ, _disk(Z), want_jac=False)
    assert rc == oracle_mod.ST_NO_INTERSECT


def test_barrel_backward_when_outside(oracle_mod):
    # a state just outside r = R (pulled there by a measurement) goes back to the
    # crossing behind it, not around the whole circle
    q, pt, phi0, th = -1, 2.0, 0.3, 1.2
    c = -q * KAPPA * BZ / pt
    rho = 1 / abs(c)
    st0 = np.array([0.0, 0.0, 0.0, 1 / pt, phi0, th])
    rc, a, _ = oracle_mod.propagate(st0, q, BZ, _barrel(30.0), want_jac=False)
    rc2, b, _ = oracle_mod.propagate(a, q, BZ, _barrel(29.9), want_jac=False)
    s_ab = 2 * rho * math.asin(29.9 / (2 * rho)) - 2 * rho * math.asin(30.0 / (2 * rho))
    assert rc == 0 and rc2 == 0
    assert math.hypot(b[0], b[1]) == pytest.approx(29.9, abs=1e-11)
    assert b[2] - a[2] == pytest.approx(s_ab / math.tan(th), abs=1e-11)
    # straight line, same rule
    st = np.array([10.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    rc, o, _ = oracle_mod.propagate(st, 1, 0.0, _barrel(9.0), want_jac=False)
    assert rc == 0 and o[0] == pytest.approx(9.0, abs=1e-13)


def test_seed_hit_choice(oracle_mod):
    # barrel layers 4 cm apart: hits 0, 1, 2
    x = np.array([4, 8, 12, 16], np.float32)
    assert oracle_mod.seed_hits(x, np.zeros(4, np.float32))[1:] == (1, 2)
    # a disk/barrel pair 0.03 cm apart is skipped
    x = np.array([4, 9.97, 10.0, 16, 22], np.float32)
    assert oracle_mod.seed_hits(x, np.zeros(5, np.float32))[1:] == (1, 3)
    x = np.array([4, 5.0, 7.0, 7.5, 9.5], np.float32)
    assert oracle_mod.seed_hits(x, np.zeros(5, np.float32))[1:] == (2, 4)
    # nothing far enough: fall back to 1, 2
    x = np.array([4, 4.5, 5.0], np.float32)
    assert oracle_mod.seed_hits(x, np.zeros(3, np.float32))[1:] == (1, 2)


def test_helix_straight_line_limit(oracle_mod):
    st = np.array([1.0, -2.0, 3.0, 0.0, 0.4, 1.0])
    out = oracle_mod.helix_at(st, 0.0, 7.5)
    np.testing.assert_allclose(out[:3], [1 + 7.5 * math.cos(0.4), -2 + 7.5 * math.sin(0.4), 3 + 7.5 / math.tan(1.0)],
                               atol=1e-13)
    # small curvature: x = x0 + s cos(phi) - c s^2/2 sin(phi) + O(c^2 s^3), same for y
    for c in (1e-6, -1e-6, 3e-5):
        a = oracle_mod.helix_at(st, c, 7.5)
        ex = 1 + 7.5 * math.cos(0.4) - c * 7.5 ** 2 / 2 * math.sin(0.4)
        ey = -2 + 7.5 * math.sin(0.4) + c * 7.5 ** 2 / 2 * math.cos(0.4)
        np.testing.assert_allclose(a[:2], [ex, ey], atol=5 * c * c * 7.5 ** 3)
    # the chord form equals the textbook form (sin phi(s) - sin phi) / c away from c = 0
    c = 0.02
    a = oracle_mod.helix_at(st, c, 7.5)
    np.testing.assert_allclose(a[:2], [1 + (math.sin(0.4 + c * 7.5) - math.sin(0.4)) / c,
                                       -2 - (math.cos(0.4 + c * 7.5) - math.cos(0.4)) / c], atol=1e-12)


def test_noise_free_propagation_matches_simulated_truth(oracle_mod):
    # the generator computes crossings from angles about the helix centre, independently
    for gname in ("barrel17", "lids"):
        g = synth.geometry(gname)
        tk = synth.gen_tracks(g, 300, 11, eta_max=2.5 if gname == "lids" else 1.0, ms_on=False, smear=False,
                              keep_truth=True)
        off = tk["offsets"]
        q = tk["truth_q"]
        worst = 0.0
        for t in range(tk["n"]):
            o0, o1 = off[t], off[t + 1]
            st = tk["truth"][o0].copy()
            for k in range(o0 + 1, o1):
                rc, st, _ = oracle_mod.propagate(st, int(q[t]), g["bz"], g["surfaces"][tk["layer"][k]],
                                                 want_jac=False)
                assert rc == 0
                d = np.abs(st[:3] - tk["truth"][k][:3]).max()
                worst = max(worst, d)
                np.testing.assert_allclose(st[3:], tk["truth"][k][3:], atol=1e-11)
        assert worst < 1e-9, (gname, worst)


# ---------------------------------------------------------------------- Jacobian (Sec. 2.1)

@pytest.mark.parametrize("case", range(8))
def test_jacobian_vs_central_differences(oracle_mod, case):
    rng = np.random.default_rng(100 + case)
    q = int(rng.choice([-1, 1]))
    pt = float(np.exp(rng.uniform(math.log(0.6), math.log(10))))
    r0 = rng.uniform(5, 30)
    a0 = rng.uniform(-math.pi, math.pi)
    st = np.array([r0 * math.cos(a0), r0 * math.sin(a0), rng.uniform(-10, 10), 1.0 / pt,
                   a0 + rng.uniform(-0.3, 0.3), rng.uniform(0.6, 2.5)])
    surf = _barrel(r0 + rng.uniform(3, 12)) if case < 5 else _disk(
        float(np.sign(math.cos(st[5])) * (abs(st[2]) + rng.uniform(5, 20))))
    rc, out, J = oracle_mod.propagate(st, q, BZ, surf)
    assert rc == 0
    Jn = np.zeros((6, 6))
    for j in range(6):
        h = 1e-6 * max(1.0, abs(st[j]))
        a = st.copy()
        b = st.copy()
        a[j] += h
        b[j] -= h
        _, oa, _ = oracle_mod.propagate(a, q, BZ, surf, want_jac=False)
        _, ob, _ = oracle_mod.propagate(b, q, BZ, surf, want_jac=False)
        d = oa - ob
        d[4] = (d[4] + math.pi) % (2 * math.pi) - math.pi
        Jn[:, j] = d / (2 * h)
    scale = np.maximum(np.abs(Jn), 1.0)
    assert np.max(np.abs(J - Jn) / scale) < 1e-6


# ---------------------------------------------------------------------- update (Sec. 4.1)

def test_update_equals_information_form(oracle_mod):
    # textbook information form: P+ = (P^-1 + H^T R^-1 H)^-1, x+ = P+ (P^-1 x + H^T R^-1 m),
    # chi2 = r^T (H P H^T + R)^-1 r
    rng = np.random.default_rng(5)
    H = np.hstack([np.eye(3), np.zeros((3, 3))])
    for _ in range(20):
        A = rng.normal(size=(6, 6))
        P = A @ A.T * 0.01 + np.eye(6) * 1e-3
        B = rng.normal(size=(3, 3))
        R = B @ B.T * 1e-4 + np.eye(3) * 1e-5
        x = rng.normal(size=6)
        x[4] = 0.3
        m = x[:3] + rng.normal(size=3) * 0.05
        rc, xo, Po, chi2 = oracle_mod.update(x, P, m, R)
        Pi = np.linalg.inv(np.linalg.inv(P) + H.T @ np.linalg.inv(R) @ H)
        xi = Pi @ (np.linalg.solve(P, x) + H.T @ np.linalg.solve(R, m))
        r = m - x[:3]
        assert rc == 0
        np.testing.assert_allclose(Po, Pi, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(xo, xi, rtol=1e-9, atol=1e-12)
        assert chi2 == pytest.approx(r @ np.linalg.solve(P[:3, :3] + R, r), rel=1e-10)


def test_meas_cov_frames(oracle_mod):
    # barrel: radial / phi / z resolutions along the hit's own axes
    s = dict(kind=0, pos=10.0, half_or_rin=50, r_out=0, x_x0=0.02, sig_n=0.03, sig_rphi=0.01, sig_3=0.1)
    a = 0.9
    R = oracle_mod.meas_cov(s, np.array([10 * math.cos(a), 10 * math.sin(a), 1.0]))
    er = np.array([math.cos(a), math.sin(a), 0])
    ep = np.array([-math.sin(a), math.cos(a), 0])
    assert er @ R @ er == pytest.approx(0.03 ** 2, rel=1e-12)
    assert ep @ R @ ep == pytest.approx(0.01 ** 2, rel=1e-12)
    assert R[2, 2] == pytest.approx(0.01, rel=1e-12)
    assert abs(er @ R @ ep) < 1e-18
    # disk: z is the normal, r the third axis
    s = dict(kind=1, pos=50.0, half_or_rin=10, r_out=100, x_x0=0.02, sig_n=0.01, sig_rphi=0.02, sig_3=0.1)
    R = oracle_mod.meas_cov(s, np.array([20 * math.cos(a), 20 * math.sin(a), 50.0]))
    assert R[2, 2] == pytest.approx(1e-4, rel=1e-12)
    assert er @ R @ er == pytest.approx(0.01, rel=1e-12)
    assert ep @ R @ ep == pytest.approx(4e-4, rel=1e-12)


def test_kf_equals_global_least_squares_linear_model(oracle_mod):
    """Scattering off, propagation linearised about the true trajectory: the filter's
    final state, covariance and summed chi2 equal the batch generalised least-squares
    solution with the Gaussian seed prior (the Kalman/GLS identity)."""
    g = synth.geometry("barrel17")
    ref = synth.gen_tracks(g, 6, 21, ms_on=False, smear=False, keep_truth=True)
    noisy = synth.gen_tracks(g, 6, 21, ms_on=False, smear=True, keep_truth=True)
    assert np.array_equal(ref["offsets"], noisy["offsets"])
    H = np.hstack([np.eye(3), np.zeros((3, 3))])
    for t in range(ref["n"]):
        o0, o1 = ref["offsets"][t], ref["offsets"][t + 1]
        if o1 - o0 < 6:
            continue
        o1 = o0 + 6
        q = int(ref["truth_q"][t])
        trj = ref["truth"][o0:o1]
        lay = ref["layer"][o0:o1]
        hx, hy, hz = noisy["x"][o0:o1], noisy["y"][o0:o1], noisy["z"][o0:o1]
        seed = trj[0] + np.array([0.02, -0.01, 0.05, 0.01, 0.002, -0.003])
        P0 = 0.5
        res = oracle_mod.fit_one(g, lay, hx, hy, hz, seed, q, seed_cov=P0, ms_on=False, lin_ref=trj)
        assert res["status"] == 0
        # batch model: x_k = ref_k + Phi_k (x_0 - ref_0)
        Phi = [np.eye(6)]
        for k in range(1, 6):
            _, _, J = oracle_mod.propagate(trj[k - 1], q, g["bz"], g["surfaces"][lay[k]])
            Phi.append(J @ Phi[-1])
        Ainf = np.eye(6) / P0
        b = (seed - trj[0]) / P0
        for k in range(6):
            m = np.array([hx[k], hy[k], hz[k]], float)
            R = oracle_mod.meas_cov(g["surfaces"][lay[k]], m)
            Ri = np.linalg.inv(R)
            Hk = H @ Phi[k]
            Ainf += Hk.T @ Ri @ Hk
            b += Hk.T @ Ri @ (m - trj[k][:3])
        cov0 = np.linalg.inv(Ainf)
        d0 = cov0 @ b
        xN = trj[5] + Phi[5] @ d0
        PN = Phi[5] @ cov0 @ Phi[5].T
        chi2 = (d0 - (seed - trj[0])) @ (d0 - (seed - trj[0])) / P0
        for k in range(6):
            m = np.array([hx[k], hy[k], hz[k]], float)
            R = oracle_mod.meas_cov(g["surfaces"][lay[k]], m)
            rk = m - trj[k][:3] - H @ Phi[k] @ d0
            chi2 += rk @ np.linalg.solve(R, rk)
        sig = np.sqrt(np.diag(PN))
        assert np.max(np.abs(res["state"] - xN) / sig) < 1e-6
        np.testing.assert_allclose(res["cov"], PN, rtol=1e-6, atol=1e-12 * np.abs(PN).max())
        assert res["chi2"] == pytest.approx(chi2, rel=1e-7)


# ---------------------------------------------------------------------- seed (Sec. 2)

@pytest.mark.parametrize("q", [-1, 1])
def test_seed_on_exact_helix(oracle_mod, q):
    pt, phi0, th = 1.7, -2.9, 2.0
    c = -q * KAPPA * BZ / pt
    rho = 1 / abs(c)
    hits = []
    for R in (4.0, 8.0, 12.0):
        s = 2 * rho * math.asin(R / (2 * rho))
        hits.append(np.array([R * math.cos(phi0 + c * s / 2), R * math.sin(phi0 + c * s / 2), s / math.tan(th)]))
    st, qs = oracle_mod.seed(hits[0], hits[1], hits[2], BZ)
    s1 = 2 * rho * math.asin(4.0 / (2 * rho))
    assert qs == q
    np.testing.assert_allclose(st[:3], hits[0], atol=1e-14)
    assert st[3] == pytest.approx(1 / pt, rel=1e-10)
    d = (st[4] - (phi0 + c * s1) + math.pi) % (2 * math.pi) - math.pi
    assert abs(d) < 1e-11
    assert st[5] == pytest.approx(th, abs=1e-11)


def test_seed_collinear(oracle_mod):
    st, q = oracle_mod.seed(np.array([1.0, 1, 0]), np.array([2.0, 2, 1]), np.array([3.0, 3, 2]), BZ)
    assert q == 1 and st[3] == 0.0
    assert st[4] == pytest.approx(math.pi / 4, abs=1e-15)
    assert st[5] == pytest.approx(math.atan2(2 * math.sqrt(2), 2), abs=1e-15)


# ---------------------------------------------------------------------- full fit (Sec. 2)

def test_noise_free_fit_recovers_truth(oracle_mod):
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 200, 31, ms_on=False, smear=False, keep_truth=True)
    r = oracle_mod.fit(g, tk, ms_on=False)
    last = tk["offsets"][1:] - 1
    tru = tk["truth"][last]
    assert np.all(r["status"] == 0)
    sig = np.sqrt(np.diagonal(r["cov"], axis1=1, axis2=2))
    d = r["state"] - tru
    d[:, 3] = r["q"] * r["state"][:, 3] - tk["truth_q"] * tru[:, 3]
    # the only noise left is the float32 rounding of the hit coordinates (~4e-6 cm)
    assert np.max(np.abs(d) / sig) < 0.01
    assert np.max(r["chi2"]) < 1e-3


def test_fit_straight_line_without_field(oracle_mod):
    g = synth.geometry("barrel10", bz=0.0)
    rng = np.random.default_rng(3)
    for _ in range(5):
        phi0, th = rng.uniform(-3, 3), rng.uniform(0.8, 2.3)
        d = np.array([math.sin(th) * math.cos(phi0), math.sin(th) * math.sin(phi0), math.cos(th)])
        R = np.array([s["pos"] for s in g["surfaces"]])
        pts = d[None, :] * (R / math.sin(th))[:, None]
        lay = np.arange(10, dtype=np.uint8)
        st, q = oracle_mod.seed(pts[0], pts[1], pts[2], 0.0)
        res = oracle_mod.fit_one(g, lay, pts[:, 0], pts[:, 1], pts[:, 2], st, q, ms_on=False)
        assert res["status"] == 0
        np.testing.assert_allclose(res["state"][:3], pts[-1], atol=2e-5)
        assert res["state"][4] == pytest.approx(phi0, abs=1e-6)
        assert res["state"][5] == pytest.approx(th, abs=1e-6)


def test_fit_statistics_on_simulated_tracks(oracle_mod):
    """Pulls of the five surface parameters ~ N(0,1) and chi2 ~ chi2(2N-5) on 1e5 tracks."""
    from scipy import stats
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 100_000, synth.BASE_SEED + 1, keep_truth=True)
    r = oracle_mod.fit(g, tk, threads=4)
    assert np.all(r["status"] & ~np.uint32(oracle_mod.ST_GRAZING) == 0)
    last = tk["offsets"][1:] - 1
    tru = tk["truth"][last]
    st = r["state"]
    C = r["cov"]
    # local barrel frame at the truth point: r-phi displacement, z
    a = np.arctan2(tru[:, 1], tru[:, 0])
    ep = np.stack([-np.sin(a), np.cos(a)], 1)
    drphi = np.sum((st[:, :2] - tru[:, :2]) * ep, 1)
    srphi = np.sqrt(np.einsum("ni,nij,nj->n", ep, C[:, :2, :2], ep))
    pulls = {
        "rphi": drphi / srphi,
        "z": (st[:, 2] - tru[:, 2]) / np.sqrt(C[:, 2, 2]),
        "q/pT": (r["q"] * st[:, 3] - tk["truth_q"] * tru[:, 3]) / np.sqrt(C[:, 3, 3]),
        "phi": ((st[:, 4] - tru[:, 4] + np.pi) % (2 * np.pi) - np.pi) / np.sqrt(C[:, 4, 4]),
        "theta": (st[:, 5] - tru[:, 5]) / np.sqrt(C[:, 5, 5]),
    }
    for k, p in pulls.items():
        assert abs(p.mean()) < 0.02, (k, p.mean())
        assert abs(p.std() - 1.0) < 0.03, (k, p.std())
    assert np.all(r["ndof"] == 2 * 10 - 5)
    assert abs(np.mean(r["chi2"] / r["ndof"]) - 1.0) < 0.02
    pv = stats.chi2.sf(r["chi2"], r["ndof"])
    assert stats.kstest(pv[:20000], "uniform").pvalue > 1e-3


def test_output_covariances_psd_rank5_and_symmetric(oracle_mod):
    """The fitted covariance is symmetric positive semi-definite with exactly one null
    direction: the fitted point lies on the last surface, so the position variance along
    the surface normal is zero (six parameters, five degrees of freedom)."""
    g = synth.geometry("lids")
    tk = synth.gen_tracks(g, 3000, 41, eta_max=2.5, keep_truth=False, min_hits=4)
    r = oracle_mod.fit(g, tk)
    ok = r["status"] & np.uint32(oracle_mod.ST_NO_INTERSECT | oracle_mod.ST_CHOL_FAIL) == 0
    assert ok.mean() > 0.99
    for t in np.nonzero(ok)[0]:
        C = r["cov"][t]
        assert np.max(np.abs(C - C.T)) <= 1e-12 * np.abs(C).max()
        ev = np.linalg.eigvalsh(C)
        assert ev[0] >= -1e-12 * ev[-1]
        assert ev[1] > 1e-9 * ev[-1]
        # the null vector is the normal of the last surface (position block only)
        w, V = np.linalg.eigh(C)
        v = V[:, 0]
        assert np.linalg.norm(v[:3]) > 0.99, (t, v)


def test_fp64_oracle_vs_high_precision_reference(oracle_mod):
    """Bound the oracle's own rounding error: the same filter steps in 40-digit arithmetic
    (mpmath) give the same final state to < 1e-4 sigma."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 3, 7, keep_truth=True)
    r = oracle_mod.fit(g, tk)
    for t in range(tk["n"]):
        o0, o1 = tk["offsets"][t], tk["offsets"][t + 1]
        q = int(r["q"][t])
        st = mp.matrix(r["seed"][t].tolist())
        P = mp.eye(6) * mp.mpf(10000)
        chi = mp.mpf(0)
        for k in range(o1 - o0):
            sf = g["surfaces"][tk["layer"][o0 + k]]
            stf = np.array([float(v) for v in st])
            if k > 0:
                _, nx, J = oracle_mod.propagate(stf, q, g["bz"], sf)
                Jm = mp.matrix(J.tolist())
                P = Jm * P * Jm.T
                st = mp.matrix(nx.tolist())
                stf = nx
            _, Q = oracle_mod.ms_noise(stf, g["mass"], sf, np.zeros((6, 6)))
            P = P + mp.matrix(Q.tolist())
            hit = np.array([tk["x"][o0 + k], tk["y"][o0 + k], tk["z"][o0 + k]], float)
            R = mp.matrix(oracle_mod.meas_cov(sf, hit).tolist())
            rr = mp.matrix([mp.mpf(float(hit[i])) - st[i] for i in range(3)])
            S = P[0:3, 0:3] + R
            Si = S ** -1
            K = P[:, 0:3] * Si
            st = st + K * rr
            P = P - K * P[0:3, :]
            chi += (rr.T * Si * rr)[0]
        ref = np.array([float(v) for v in st])
        sig = np.sqrt(np.array([float(P[i, i]) for i in range(6)]))
        d = (r["state"][t] - ref) / sig
        assert np.max(np.abs(d)) < 1e-4
        assert r["chi2"][t] == pytest.approx(float(chi), rel=1e-5)


# ---------------------------------------------------------------------- binning (Sec. 3.1)

def test_bin_key_at_bin_centres(oracle_mod):
    Lz = 40.0
    for j in (0, 1, 511, 512, 1000, 1023):
        for zb in (0, 17, 63):
            phi = -math.pi + (j + 0.5) * 2 * math.pi / 1024
            z = -Lz + (zb + 0.5) * 2 * Lz / 64
            key = oracle_mod.bin_key(20 * math.cos(phi), 20 * math.sin(phi), z, Lz)
            assert key == zb * 1024 + j
    # clamping: z beyond the layer, phi exactly pi
    assert oracle_mod.bin_key(-20.0, 0.0, 1e3, Lz) == 63 * 1024 + 1023
    assert oracle_mod.bin_key(-20.0, -0.0, -1e3, Lz) == 0


def test_bin_layer_is_stable_counting_sort(oracle_mod):
    rng = np.random.default_rng(8)
    n = 5000
    Lz = 30 + 1.6 * 40
    phi = rng.uniform(-math.pi, math.pi, n)
    # crowd some hits into a few bins to exercise stability
    phi[:600] = 0.1
    x = (40 * np.cos(phi)).astype(np.float32)
    y = (40 * np.sin(phi)).astype(np.float32)
    z = rng.uniform(-Lz - 5, Lz + 5, n).astype(np.float32)
    z[:300] = 1.0
    perm, offsets = oracle_mod.bin_layer(x, y, z, Lz)
    keys = [oracle_mod.bin_key(x[i], y[i], z[i], Lz) for i in range(n)]
    expect = sorted(range(n), key=lambda i: (keys[i], i))
    assert list(perm) == expect
    counts = np.bincount(keys, minlength=65536)
    assert offsets[0] == 0 and offsets[-1] == n
    np.testing.assert_array_equal(np.diff(offsets), counts)
    # empty layer
    perm, offsets = oracle_mod.bin_layer(np.zeros(0, np.float32), np.zeros(0, np.float32),
                                         np.zeros(0, np.float32), Lz)
    assert len(perm) == 0 and np.all(offsets == 0)


# ---------------------------------------------------------------------- best-hit building (Sec. 2)

def _binned_event(oracle_mod, g, n, seed, noise=0.2):
    ev = synth.gen_event(g, n, seed, noise_frac=noise)
    for ly in ev["layers"]:
        Lz = g["surfaces"][ly["surf"]]["half_or_rin"]
        ly["perm"], ly["offsets"] = oracle_mod.bin_layer(ly["x"], ly["y"], ly["z"], Lz)
    return ev


def test_besthit_window_enumeration_brute_force(oracle_mod):
    g = synth.geometry("barrel17")
    ev = _binned_event(oracle_mod, g, 400, 5)
    out = oracle_mod.build_besthit(g, ev, record=True)
    rec = out["rec"]
    checked = 0
    for t in range(0, ev["n"], 7):
        for L in range(3, 17):
            r = rec[t, L]
            if r["status"] != 0 or r["phi_n"] == 0:
                continue
            ly = ev["layers"][L]
            Lz = g["surfaces"][L]["half_or_rin"]
            zset = set(range(r["z_lo"], r["z_hi"] + 1))
            pset = set((r["phi_lo"] + k) % 1024 for k in range(r["phi_n"]))
            inwin = [i for i in range(len(ly["x"]))
                     if (lambda kk: kk // 1024 in zset and kk % 1024 in pset)(
                         oracle_mod.bin_key(ly["x"][i], ly["y"][i], ly["z"][i], Lz))]
            assert r["n_cand"] == min(len(inwin), 32)
            assert bool(r["capped"]) == (len(inwin) > 32)
            if r["best"] >= 0:
                assert r["best"] in inwin
                assert r["chi2_best"] < 30.0
            checked += 1
    assert checked > 100


def test_besthit_finds_true_hits(oracle_mod):
    g = synth.geometry("barrel17")
    ev = _binned_event(oracle_mod, g, 2000, 6)
    out = oracle_mod.build_besthit(g, ev)
    where = ev["truth_where"]
    has = where[:, 3:] >= 0
    found = out["idx"][:, 3:]
    eff = np.mean(found[has] == where[:, 3:][has])
    fake = np.mean((found >= 0) & (found != where[:, 3:]))
    assert eff > 0.97, eff
    assert fake < 0.03, fake
    # seed layers carry the given seed hits
    np.testing.assert_array_equal(out["idx"][:, :3], ev["seed_idx"])


# ---------------------------------------------------------------------- combinatorial building (Sec. 2, 4.3)

def test_ckf_with_one_slot_is_besthit(oracle_mod):
    """One candidate per seed: the ranking keeps the smallest-chi2 hit below the
    cut, else the candidate without a hit -- best-hit building, to the bit."""
    g = synth.geometry("barrel17")
    ev = _binned_event(oracle_mod, g, 600, 31)
    bh = oracle_mod.build_besthit(g, ev)
    ck = oracle_mod.build_ckf(g, ev, n_slots=1)
    for k in ("idx", "state", "cov", "chi2", "ndof", "status"):
        np.testing.assert_array_equal(ck[k], bh[k])


def _small_event(oracle_mod, n_signal, seed):
    """Three seed layers and three build layers of the 10-cylinder barrel, a few
    hits a layer (signal + noise)."""
    g = synth.geometry("barrel10")
    ev = synth.gen_event(g, n_signal, synth.BASE_SEED + seed, noise_frac=0.5)
    ev["layers"] = ev["layers"][:6]
    g = dict(g, surfaces=g["surfaces"][:6])
    for ly in ev["layers"]:
        ly["perm"], ly["offsets"] = oracle_mod.bin_layer(ly["x"], ly["y"], ly["z"], g["surfaces"][ly["surf"]]["half_or_rin"])
    return g, ev


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_ckf_equals_exhaustive_search_without_pruning(oracle_mod, seed):
    """With more slots than paths, a window wider than the layer and scattering off,
    nothing is pruned: the first candidate must be the best of all hit choices
    (one hit or none per build layer), found by fitting every path and keeping
    those whose every hit passes the chi2 cut -- more hits first, then smaller
    total chi2."""
    import itertools
    g, ev = _small_event(oracle_mod, 3, seed)
    nl = len(ev["layers"])
    cut = 30.0
    ck = oracle_mod.build_ckf(g, ev, n_slots=1024, nsigma=1e4, chi2_cut=cut, max_cand=1024, ms_on=False)
    checked = 0
    for t in range(ev["n"]):
        sh = ev["seed_hits"][t]
        seed_state, q = oracle_mod.seed(sh[0], sh[1], sh[2], g["bz"])
        choices = [[-1] + list(range(len(ev["layers"][L]["x"]))) for L in range(3, nl)]
        best = None
        for path in itertools.product(*choices):
            lay = [0, 1, 2] + [3 + k for k, h in enumerate(path) if h >= 0]
            hx = [sh[0, 0], sh[1, 0], sh[2, 0]] + [ev["layers"][3 + k]["x"][h] for k, h in enumerate(path) if h >= 0]
            hy = [sh[0, 1], sh[1, 1], sh[2, 1]] + [ev["layers"][3 + k]["y"][h] for k, h in enumerate(path) if h >= 0]
            hz = [sh[0, 2], sh[1, 2], sh[2, 2]] + [ev["layers"][3 + k]["z"][h] for k, h in enumerate(path) if h >= 0]
            surf = [ev["layers"][L]["surf"] for L in lay]
            r = oracle_mod.fit_one(g, surf, hx, hy, hz, seed_state, q, ms_on=False)
            if r["status"] & 7 or r["n_used"] != len(lay):
                continue
            if np.any(r["chi2_each"][3:] >= cut):
                continue
            key = (-len(lay), r["chi2"])
            if best is None or key < best[0]:
                best = (key, path, r)
        assert best is not None
        (negnh, chi2), path, r = best
        np.testing.assert_array_equal(ck["idx"][t, 3:], np.array(path))
        assert ck["chi2"][t] == pytest.approx(chi2, rel=1e-9)
        np.testing.assert_allclose(ck["state"][t], r["state"], rtol=1e-9, atol=1e-9)
        checked += 1
    assert checked == ev["n"]


def test_ckf_more_slots_recover_inefficiency(oracle_mod):
    """Keeping several candidates per seed recovers true hits that best-hit loses
    to a noise hit with a smaller chi2 (the branching of Sec. 2)."""
    g = synth.geometry("barrel17")
    ev = _binned_event(oracle_mod, g, 2000, 32)
    where = ev["truth_where"][:, 3:]
    has = where >= 0
    effs = []
    for ns in (1, 4):
        ck = oracle_mod.build_ckf(g, ev, n_slots=ns)
        effs.append(np.mean(ck["idx"][:, 3:][has] == where[has]))
        np.testing.assert_array_equal(ck["idx"][:, :3], ev["seed_idx"])
    assert effs[1] > effs[0], effs


# ---------------------------------------------------------------------- outward-inward refit

def test_refit_inward_noise_free_recovers_truth_at_first_hit(oracle_mod):
    """Noise-free tracks (no smearing, no scattering): the backward fit ends on the
    first hit with the true state there."""
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 200, 33, ms_on=False, smear=False, keep_truth=True)
    fw = oracle_mod.fit(g, tk, ms_on=False)
    bw = oracle_mod.refit_inward(g, tk, fw["state"], fw["cov"], fw["q"], fw["ndof"], ms_on=False)
    first = tk["offsets"][:-1]
    tru = tk["truth"][first]
    assert np.all(bw["status"] == 0)
    sig = np.sqrt(np.diagonal(bw["cov"], axis1=1, axis2=2))
    d = bw["state"] - tru
    d[:, 3] = fw["q"] * bw["state"][:, 3] - tk["truth_q"] * tru[:, 3]
    d[:, 4] = (d[:, 4] + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(d) / sig) < 0.01
    assert np.max(bw["chi2"]) < 1e-3
    np.testing.assert_array_equal(bw["ndof"], fw["ndof"])


def test_refit_inward_statistics_at_first_hit(oracle_mod):
    """Smeared hits, no scattering: the backward estimate at the first hit against
    the true state there.  Pulls of the five surface parameters have unit width and
    the full five-parameter chi2 (which uses the correlations, so a wrong sign in
    the reversed covariance shows) has mean 5."""
    import sys
    sys.path.insert(0, HERE)
    import parity
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 4000, 34, ms_on=False, keep_truth=True)
    fw = oracle_mod.fit(g, tk, ms_on=False)
    bw = oracle_mod.refit_inward(g, tk, fw["state"], fw["cov"], fw["q"], fw["ndof"], ms_on=False)
    ok = (fw["status"] == 0) & (bw["status"] == 0) & (fw["q"] == tk["truth_q"])
    first = tk["offsets"][:-1]
    tru = tk["truth"][first][ok]
    st, C6 = bw["state"][ok], bw["cov"][ok]
    T = parity.local_frame(tru, np.zeros(len(tru), int))
    d = st - tru
    d[:, 4] = (d[:, 4] + np.pi) % (2 * np.pi) - np.pi
    dl = np.einsum("nij,nj->ni", T, d)
    C5 = np.einsum("nai,nij,nbj->nab", T, C6, T)
    pulls = dl / np.sqrt(np.diagonal(C5, axis1=1, axis2=2))
    chi2 = np.einsum("ni,ni->n", dl, np.linalg.solve(C5, dl[:, :, None])[:, :, 0])
    m = len(tru)
    assert m > 0.9 * tk["n"]
    np.testing.assert_allclose(pulls.std(axis=0), 1.0, atol=0.06)
    np.testing.assert_allclose(pulls.mean(axis=0), 0.0, atol=0.06)
    assert abs(chi2.mean() - 5.0) < 5 * np.sqrt(10.0 / m)


def test_refit_inward_counts_the_forward_fit_at_weight_one_over_scale(oracle_mod):
    """The backward pass starts from the forward estimate with its covariance times
    cov_scale, so (no scattering: every hit's information adds) the forward fit's
    information enters once more at weight 1 / cov_scale.  The forward covariance
    holds the information of the same hits, so the covariance at the first hit with
    cov_scale = 100 is the one with a diffuse start (cov_scale = 1e8) divided by
    1 + 1/100: each variance by 1.01.  A start that counted the forward
    information at full weight (halving the variances), or not at all, fails.  Per
    track the ratio scatters by up to a few percent (the two passes and the forward
    fit linearise the helix at slightly different states); its mean over the tracks
    is held to 3e-4."""
    g = synth.geometry("barrel10")
    tk = synth.gen_tracks(g, 300, 35, ms_on=False)
    fw = oracle_mod.fit(g, tk, ms_on=False)
    b100 = oracle_mod.refit_inward(g, tk, fw["state"], fw["cov"], fw["q"], fw["ndof"], cov_scale=100.0,
                                   ms_on=False)
    bdif = oracle_mod.refit_inward(g, tk, fw["state"], fw["cov"], fw["q"], fw["ndof"], cov_scale=1e8,
                                   ms_on=False)
    ok = (fw["status"] == 0) & (b100["status"] == 0) & (bdif["status"] == 0)
    assert ok.mean() > 0.95
    # the five free directions: 1/pT, phi, theta and the two position coordinates on the first layer
    first = tk["offsets"][:-1]
    x, y = tk["x"][first][ok].astype(float), tk["y"][first][ok].astype(float)
    r = np.hypot(x, y)
    v100, vdif = b100["cov"][ok], bdif["cov"][ok]
    ratios = [v100[:, i, i] / vdif[:, i, i] for i in (3, 4, 5)]
    # r-phi position variance: t = (-y, x) / r
    def tt(c):
        return (y * y * c[:, 0, 0] - 2 * x * y * c[:, 1, 0] + x * x * c[:, 1, 1]) / (r * r)
    ratios += [tt(v100) / tt(vdif), v100[:, 2, 2] / vdif[:, 2, 2]]
    for rt in ratios:
        np.testing.assert_allclose(rt, 1.0 / 1.01, rtol=5e-2)
        assert abs(rt.mean() * 1.01 - 1.0) < 3e-4, rt.mean() * 1.01


# ---------------------------------------------------------------------- measurement model 1 (Sec. 4.1)

def test_update2d_equals_information_form(oracle_mod):
    """The 2-D update on the tangent plane at the hit azimuth equals the
    information form with H = [(-sin a, cos a, 0, ...), (0, 0, 1, ...)]."""
    rng = np.random.default_rng(15)
    surf = _barrel(30.0)
    for _ in range(20):
        A = rng.normal(size=(6, 6))
        P = A @ A.T * 0.01 + np.eye(6) * 1e-3
        x = rng.normal(size=6)
        x[4] = 0.3
        a = rng.uniform(-math.pi, math.pi)
        m = np.array([30.0 * math.cos(a), 30.0 * math.sin(a), rng.normal()])
        H = np.zeros((2, 6))
        H[0, 0], H[0, 1], H[1, 2] = -math.sin(a), math.cos(a), 1.0
        R = np.diag([surf["sig_rphi"] ** 2, surf["sig_3"] ** 2])
        rc, xo, Po, chi2 = oracle_mod.update2d(x, P, m, surf)
        r = H[:, :3] @ (m - x[:3])
        Pi = np.linalg.inv(np.linalg.inv(P) + H.T @ np.linalg.inv(R) @ H)
        xi = x + Pi @ H.T @ np.linalg.solve(R, r)
        assert rc == 0
        np.testing.assert_allclose(Po, Pi, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(xo, xi, rtol=1e-8, atol=1e-11)
        assert chi2 == pytest.approx(r @ np.linalg.solve(H @ P @ H.T + R, r), rel=1e-10)


def _local_pulls(st, C, tru, q, tq):
    a = np.arctan2(tru[:, 1], tru[:, 0])
    ep = np.stack([-np.sin(a), np.cos(a)], 1)
    drphi = np.sum((st[:, :2] - tru[:, :2]) * ep, 1)
    srphi = np.sqrt(np.einsum("ni,nij,nj->n", ep, C[:, :2, :2], ep))
    return {
        "rphi": drphi / srphi,
        "z": (st[:, 2] - tru[:, 2]) / np.sqrt(C[:, 2, 2]),
        "q/pT": (q * st[:, 3] - tq * tru[:, 3]) / np.sqrt(C[:, 3, 3]),
        "phi": ((st[:, 4] - tru[:, 4] + np.pi) % (2 * np.pi) - np.pi) / np.sqrt(C[:, 4, 4]),
        "theta": (st[:, 5] - tru[:, 5]) / np.sqrt(C[:, 5, 5]),
    }


def test_model1_noise_free_staggered_modules(oracle_mod):
    """Modules at R -+ 0.25 cm: hits off the layer's average cylinder.  Model 1
    (each hit on its own cylinder, 2-D update) recovers the true state of
    noise-free tracks; model 0 (hits on the average cylinder) cannot."""
    g = synth.geometry("barrel17s")
    tk = synth.gen_tracks(g, 300, 35, ms_on=False, smear=False, keep_truth=True)
    last = tk["offsets"][1:] - 1
    tru = tk["truth"][last]
    r1 = oracle_mod.fit(g, tk, ms_on=False, meas_model=1)
    assert np.all(r1["status"] == 0)
    for k, p in _local_pulls(r1["state"], r1["cov"], tru, r1["q"], tk["truth_q"]).items():
        assert np.max(np.abs(p)) < 0.01, k
    assert np.max(r1["chi2"]) < 1e-3
    r0 = oracle_mod.fit(g, tk, ms_on=False, meas_model=0)
    assert np.median(r0["chi2"] / r0["ndof"]) > 10.0


def test_model1_statistics_staggered_modules(oracle_mod):
    """Model 1 on the staggered geometry with scattering and smearing: pulls of
    the five surface parameters ~ N(0, 1), and chi2 / ndof as under model 1 on
    the ideal geometry (compared as the mean over tracks without the top 1%: on
    17 layers a few low-pT tracks carry most of the chi2 tail)."""
    g = synth.geometry("barrel17s")
    tk = synth.gen_tracks(g, 20000, synth.BASE_SEED + 36, keep_truth=True)
    r = oracle_mod.fit(g, tk, meas_model=1, threads=4)
    ok = ((r["status"] & 7) == 0) & (r["q"] == tk["truth_q"])
    last = tk["offsets"][1:] - 1
    tru = tk["truth"][last][ok]
    for k, p in _local_pulls(r["state"][ok], r["cov"][ok], tru, r["q"][ok], tk["truth_q"][ok]).items():
        assert abs(p.mean()) < 0.04, (k, p.mean())
        assert abs(p.std() - 1.0) < 0.05, (k, p.std())
    g0 = synth.geometry("barrel17")
    tk0 = synth.gen_tracks(g0, 20000, synth.BASE_SEED + 36)
    r0 = oracle_mod.fit(g0, tk0, threads=4, meas_model=1)
    ok0 = (r0["status"] & 7) == 0

    def trimmed(rr, m):
        x = np.sort(rr["chi2"][m] / rr["ndof"][m])
        return x[: int(0.99 * len(x))].mean()

    t1, t0 = trimmed(r, ok), trimmed(r0, ok0)
    assert abs(t1 - t0) < 0.01, (t1, t0)
    assert 0.9 < t1 < 1.05


def test_besthit_two_step_on_staggered_modules(oracle_mod):
    """Best-hit building on the staggered geometry: with two-step propagation
    (average cylinder for the window, then each candidate's own cylinder) it keeps
    the true hits as well as on the ideal geometry; taking the hits as lying on
    the average cylinder (model 0) loses most of them."""
    effs = {}
    for name, model in (("barrel17", 0), ("barrel17", 1), ("barrel17s", 1), ("barrel17s", 0)):
        g = synth.geometry(name)
        ev = _binned_event(oracle_mod, g, 2000, 37)
        out = oracle_mod.build_besthit(g, ev, meas_model=model)
        where = ev["truth_where"][:, 3:]
        has = where >= 0
        effs[(name, model)] = np.mean(out["idx"][:, 3:][has] == where[has])
    # on the ideal geometry the two models choose alike
    assert abs(effs[("barrel17", 1)] - effs[("barrel17", 0)]) < 0.002, effs
    assert effs[("barrel17s", 1)] > effs[("barrel17", 0)] - 0.01, effs
    assert effs[("barrel17s", 0)] < 0.5, effs


def test_model1_reduces_to_model0_on_the_ideal_barrel(oracle_mod):
    """On the ideal barrel every hit lies on its layer (to the float rounding of
    its coordinates, ~5e-6 cm at 100 cm), so model 1's 2-D update on the hit's
    cylinder and model 0's 3-D update on the layer measure the same thing: the
    surface-constrained transport leaves no prior variance along the radius,
    the radial row of model 0's gain vanishes and its residual there is ~0.
    A wrong sign, row or tangent direction in the 2-D update shows on every
    track; rounding of the hit radius moves the few tracks that cross a layer
    near their apex, hence the median and 99th-percentile bounds."""
    g = synth.geometry("barrel17")
    tk = synth.gen_tracks(g, 3000, 77)
    r0 = oracle_mod.fit(g, tk, meas_model=0, threads=4)
    r1 = oracle_mod.fit(g, tk, meas_model=1, threads=4)
    assert np.array_equal(r0["status"], r1["status"]) and np.array_equal(r0["ndof"], r1["ndof"])
    ok = (r0["status"] & 7) == 0
    res = parity.compare_fits(r1, r0, np.zeros(tk["n"], int), ok)
    assert np.median(res["max_pull"]) < 1e-4, parity.summary(res)
    assert np.percentile(res["max_pull"], 99) < 1e-2, parity.summary(res)
    assert np.median(res["chi2rel"]) < 1e-4, parity.summary(res)


# ---------------------------------------------------------------------- theta range (reading of the parametrisation's pole)

def test_propagation_refused_outside_theta_range(oracle_mod):
    """A state whose theta has left (0, pi) is not propagated: the (.., phi, theta)
    parametrisation has its pole there (dz/ds = cot(theta) diverges and changes sign)."""
    surf = _barrel(10.0)
    start = np.array([4.0, 0.0, 0.0, 0.2, 0.0, 0.0])
    for th, want in ((0.05, 0), (math.pi - 0.05, 0), (-0.05, 1 | 32), (math.pi + 0.05, 1 | 32), (0.0, 1 | 32)):
        st = start.copy()
        st[5] = th
        rc, out, _ = oracle_mod.propagate(st, 1, BZ, surf)
        assert rc == want, (th, rc)
        if want == 0:
            assert math.hypot(out[0], out[1]) == pytest.approx(10.0, abs=1e-9)


def test_fit_ends_when_an_update_crosses_the_theta_pole(oracle_mod):
    """Hits far above a steep prediction pull theta through zero in the second
    update; the fit keeps that update (its state is reported) and ends before the
    next propagation, with NO_INTERSECT | THETA_RANGE.  Hits that keep theta in
    range are all used."""
    g = synth.geometry("barrel10")
    hx = np.array([4.0, 8.0, 12.0, 16.0], np.float32)
    hy = np.zeros(4, np.float32)
    seed = np.array([4.0, 0.0, 0.0, 0.2, 0.0, 0.05])
    far = oracle_mod.fit_one(g, [0, 1, 2, 3], hx, hy, np.array([0, 200, 400, 600], np.float32), seed, 1)
    assert far["status"] & 32 and far["status"] & 1
    assert far["n_used"] == 2 and far["ndof"] == -1
    assert not (0.0 < far["state"][5] < math.pi)
    near = oracle_mod.fit_one(g, [0, 1, 2, 3], hx, hy, np.array([0, 50, 100, 150], np.float32), seed, 1)
    assert not (near["status"] & 33)
    assert near["n_used"] == 4 and 0.0 < near["state"][5] < math.pi


# ---------------------------------------------------------------------- build window (Sec. 3.1, 4.1)

def _tangent_cov(phi0, sig_t, sig_z, rho_tz, sig_n=0.0, rho_nt=0.0):
    """6x6 covariance whose position block has variance sig_t^2 along phi-hat at azimuth
    phi0, sig_n^2 along r-hat, sig_z^2 along z, with correlations rho_tz (phi-hat, z) and
    rho_nt (r-hat, phi-hat); the angle block is an arbitrary positive diagonal."""
    rh = np.array([math.cos(phi0), math.sin(phi0), 0.0])
    ph = np.array([-math.sin(phi0), math.cos(phi0), 0.0])
    zh = np.array([0.0, 0.0, 1.0])
    E = np.stack([rh, ph, zh], 1)
    L = np.array([[sig_n ** 2, rho_nt * sig_n * sig_t, 0.0],
                  [rho_nt * sig_n * sig_t, sig_t ** 2, rho_tz * sig_t * sig_z],
                  [0.0, rho_tz * sig_t * sig_z, sig_z ** 2]])
    P = np.diag([0.0, 0.0, 0.0, 1e-4, 1e-6, 1e-6])
    P[:3, :3] = E @ L @ E.T
    return P


@pytest.mark.parametrize("case", ["x_axis", "y_axis", "diag45_correlated", "diag135_radial", "generic"])
def test_window_widths_match_sampled_prediction_and_hit_scatter(oracle_mod, case):
    """The window is nsigma times the spread of (hit - prediction): sample predicted
    positions from N(pred, P_pos) and hits scattered by the resolution on the cylinder
    (r-phi by sig_rphi, z by sig_z), and compare the sample std of the azimuth and z
    differences with the oracle's half widths / nsigma.  Position blocks with an x-y
    correlation (off the axes), a radial component and r-phi/z correlation make a sign
    error on the x-y term, r^2 for r^4, or a dropped resolution term each fail."""
    R = 30.0
    surf = _barrel(R)
    phi0, sig_t, sig_n, rho_nt = dict(x_axis=(0.0, 0.02, 0.0, 0.0), y_axis=(math.pi / 2, 0.02, 0.0, 0.0),
                                      diag45_correlated=(math.pi / 4, 0.015, 0.01, 0.6),
                                      diag135_radial=(3 * math.pi / 4, 0.012, 0.02, -0.5),
                                      generic=(-2.2, 0.008, 0.004, 0.3))[case]
    P = _tangent_cov(phi0, sig_t, 0.05, 0.4, sig_n, rho_nt)
    st = np.array([R * math.cos(phi0), R * math.sin(phi0), 3.0, 0.3, phi0 + 0.2, 1.2])
    dphi, dz = oracle_mod.window(st, P, surf, nsigma=3.0)
    rng = np.random.default_rng(11)
    N = 1_000_000
    pos = rng.multivariate_normal(st[:3], P[:3, :3], size=N, method="eigh")
    # hits: truth at the prediction's centre, scattered on the cylinder
    a_hit = phi0 + rng.normal(0.0, surf["sig_rphi"], N) / R
    z_hit = st[2] + rng.normal(0.0, surf["sig_3"], N)
    dphi_s = (a_hit - np.arctan2(pos[:, 1], pos[:, 0]) + np.pi) % (2 * np.pi) - np.pi
    dz_s = z_hit - pos[:, 2]
    s_phi, s_z = np.std(dphi_s), np.std(dz_s)
    # sampling error of a std over 1e6 draws ~ 0.07 %; curvature of atan2 ~ (sigma / R)^2
    assert dphi / 3.0 == pytest.approx(s_phi, rel=4e-3), (dphi / 3.0, s_phi)
    assert dz / 3.0 == pytest.approx(s_z, rel=4e-3), (dz / 3.0, s_z)


def test_window_with_a_point_prediction_is_the_hit_resolution(oracle_mod):
    """No prediction uncertainty: the window is nsigma times the hit's own scatter,
    sig_rphi / R in azimuth and sig_z in z."""
    for R in (4.0, 40.0, 100.0):
        surf = _barrel(R)
        st = np.array([0.0, R, -7.0, 0.5, 1.6, 1.0])
        dphi, dz = oracle_mod.window(st, np.zeros((6, 6)), surf, nsigma=2.5)
        assert dphi == pytest.approx(2.5 * 0.01 / R, rel=1e-12)
        assert dz == pytest.approx(2.5 * 0.1, rel=1e-12)


@pytest.mark.parametrize("a,theta", [(0.1, 1.2), (0.6, 0.8), (1.1, 2.0), (-0.8, 1.45)])
def test_window_model1_widening_is_the_sweep_over_dr(oracle_mod, a, theta):
    """Measurement model 1 widens the window by the azimuth and z that the track sweeps
    while it crosses +-dr around the average radius.  Propagate the predicted state
    (10 GeV, nearly straight) with the oracle's own helix to R - dr and R + dr and take
    the mean of the two excursions of the position's azimuth and z (their first-order
    part: the second-order terms, ~ (dr / R) tan^2(a), have opposite signs on the two
    sides); it equals the widening."""
    R, dr = 30.0, 0.25
    surf = dict(_barrel(R), dr=dr)
    phi_pos = 0.4
    st = np.array([R * math.cos(phi_pos), R * math.sin(phi_pos), 2.0, 0.1, phi_pos + a, theta])
    P = _tangent_cov(phi_pos, 0.02, 0.05, 0.0)
    d0 = oracle_mod.window(st, P, surf, nsigma=3.0, meas_model=0)
    d1 = oracle_mod.window(st, P, surf, nsigma=3.0, meas_model=1)
    sweep_phi, sweep_z = [], []
    for Rt in (R - dr, R + dr):
        rc, out, _ = oracle_mod.propagate(st, 1, BZ, _barrel(Rt), want_jac=False)
        assert rc == 0
        sweep_phi.append(abs((math.atan2(out[1], out[0]) - phi_pos + math.pi) % (2 * math.pi) - math.pi))
        sweep_z.append(abs(out[2] - st[2]))
    # what is left: (dr / R)^2 terms and the helix's bend over the crossing, O(c dr)
    assert d1[0] - d0[0] == pytest.approx(np.mean(sweep_phi), rel=3e-3)
    assert d1[1] - d0[1] == pytest.approx(np.mean(sweep_z), rel=3e-3)
