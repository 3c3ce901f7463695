"""The scenario-count study and the DVH report on the GPU (paper Sec. 3.1,
Fig. times-scenario_scaling; Sec. 3.2 DVH bands), checked against the oracle.

Each problem restricted to its first k scenarios (nominal first) is a problem of
its own; the GPU's ADMM-BB and PGD must reach that problem's exact optimum
(lsq_box on the k-scenario stacked system).  The DVH report computed from the
GPU's doses matches the one computed from the oracle's doses of the same spot
vector."""
import numpy as np
import pytest

from oracle import Weighted, lsq_box
from synthetic import config_tiny_plain

from tests.gpu_util import gpu_lib, plan_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


@pytest.fixture(scope="module")
def tiny():
    return config_tiny_plain(0)


@pytest.mark.parametrize("k", [1, 3, 7, 13])
def test_first_k_scenarios_reach_their_own_optimum(rpt, tiny, k):
    sub = tiny.subset_scenarios(range(k))
    W = Weighted(sub)
    xs = lsq_box(W)
    fs = W.f(xs)
    with plan_of(rpt, sub) as P:
        z, ia = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000)
        xp, ip = P.pgd_solve(f_target=fs * (1 + 1e-5), tol_rel_df=0.0, max_iter=50000)
    assert ia["status"] == 0 and ip["status"] == 0
    assert np.all(z >= sub.lb) and np.all(z <= sub.ub)
    assert (W.f(z) - fs) / fs <= 1e-6, (k, (W.f(z) - fs) / fs)
    # PGD stops on the GPU's own objective, a sum of float32 row residuals squared
    # (relative error up to about 2 (L + 8) eps32 of the sum of squared magnitudes,
    # ~1e-5 here), so its target is met to that accuracy
    assert (W.f(xp) - fs) / fs <= 3e-5, (k, (W.f(xp) - fs) / fs)


def test_dvh_report_from_gpu_doses_matches_the_oracle(rpt, tiny):
    import bench
    W = Weighted(tiny)
    with plan_of(rpt, tiny) as P:
        z, _ = P.admm_bb_solve(eps_abs=1e-5, eps_rel=1e-5)
        f, D = P.objective(z, dose=True)
    Dref = np.stack([W.dose(s, z) for s in range(tiny.N)])
    # float32 doses: each a dot of at most L terms
    L = max(int(np.diff(rp).max()) for rp in tiny.row_ptr)
    mag = np.stack([abs(W.A[s]) @ np.abs(z) for s in range(tiny.N)])
    assert np.all(np.abs(D - Dref) <= (L + 4) * np.finfo(np.float32).eps * mag + 1e-30)
    got = bench.dvh_report(D, tiny.labels)
    ref = bench.dvh_report(Dref, tiny.labels)
    assert got.keys() == ref.keys()
    for name in ref:
        for key, (lo, med, hi) in ref[name]["metrics_gy"].items():
            np.testing.assert_allclose(got[name]["metrics_gy"][key], [lo, med, hi], rtol=1e-4, atol=1e-4)
        # DVH fractions can only move where a dose sits within rounding of a level
        dv = np.abs(np.asarray(got[name]["dvh_nominal"]) - np.asarray(ref[name]["dvh_nominal"]))
        assert dv.max() <= 2.0 / ref[name]["voxels"]
