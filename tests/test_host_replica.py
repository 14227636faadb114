"""The kernels' per-track fit compiled for the host (tests/host_replica.py) against
the FP64 oracle, on the CPU: the same tolerances as the GPU parity tests.  This
keeps the host copy that the precision readings were measured with honest (it
fails if it drifts from what the oracle and the GPU agree on), and tests the mixed
arithmetic of the fit without a GPU."""
import numpy as np
import pytest

import host_replica
import parity
from paper_1711_06571_gb300 import kf, synth

ST_BAD = 7


@pytest.fixture(scope="module")
def replica():
    return host_replica.build()


def _oracle_and_replica(oracle_mod, replica, g, tk, meas_model=0):
    o0 = oracle_mod.fit(g, tk, threads=4, meas_model=meas_model)
    seed = o0["seed"].astype(np.float32)
    orc = oracle_mod.fit(g, tk, seeds=seed.astype(np.float64), q=o0["q"], threads=4, meas_model=meas_model)
    host = host_replica.host_fit(replica, g, tk, seed, orc["q"], meas_model=meas_model)
    np.testing.assert_array_equal(host["status"] & ST_BAD, orc["status"] & ST_BAD)
    np.testing.assert_array_equal(host["ndof"], orc["ndof"])
    ok = (orc["status"] & ST_BAD) == 0
    kinds = np.array([g["surfaces"][s]["kind"] for s in parity.last_surface(tk, orc["ndof"])])
    return orc, host, ok, kinds


@pytest.mark.parametrize("name,model", [("barrel17", 0), ("barrel17s", 1)])
def test_host_replica_barrel(oracle_mod, replica, name, model):
    g = synth.geometry(name)
    tk = synth.gen_tracks(g, 3000, synth.BASE_SEED + 41)
    orc, host, ok, kinds = _oracle_and_replica(oracle_mod, replica, g, tk, model)
    res = parity.compare_fits(host, orc, kinds, ok)
    print(name, parity.summary(res))
    assert ok.mean() > 0.99
    assert res["max_pull"].max() <= parity.TOL_PARAM_SIGMA
    assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
    assert res["dcov"].max() <= parity.TOL_COV_NORM


def test_host_replica_barrel_with_disks(oracle_mod, replica):
    """Barrel + end-cap disks, |eta| < 2.5: each track within max(1e-3 sigma, 3 x the
    oracle's own resolution), as on the GPU; tracks that met a crossing within a few
    degrees of tangent (KF_ST_GRAZING) within 5e-3 sigma, since there the host's
    sines and reciprocal approximations, which differ from the GPU's in their last
    bits, are amplified most (one such track of 3,982 at 1.7e-3)."""
    g = synth.geometry("lids")
    tk = synth.gen_tracks(g, 4000, synth.BASE_SEED + 42, eta_max=2.5, min_hits=4)
    orc, host, ok, kinds = _oracle_and_replica(oracle_mod, replica, g, tk)
    noise = parity.oracle_self_noise(oracle_mod, g, tk, orc, kinds)
    res = parity.compare_fits(host, orc, kinds, ok)
    print("lids", parity.summary(res))
    graz = (orc["status"][ok] & kf.KF_ST_GRAZING) != 0
    lim = np.maximum(np.where(graz, 5 * parity.TOL_PARAM_SIGMA, parity.TOL_PARAM_SIGMA), 3.0 * noise[ok])
    assert np.all(res["max_pull"] <= lim)
    assert res["chi2rel"].max() <= parity.TOL_CHI2_REL
    assert res["dcov"].max() <= parity.TOL_COV_NORM
