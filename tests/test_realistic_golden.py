"""The stored full-size optimum (tests/golden/realistic_seed0_oracle.json,
written by tests/golden/make_realistic_golden.py from the oracle) checked
against the optimality conditions of the box-constrained least squares of
Eq. 2, recomputed here on the regenerated realistic workload (13 scenarios,
299,088 voxels, 5,000 spots): z* feasible, the projected gradient and every
KKT sign condition zero to rounding, f(z*) and |D(z*)| as stored.  CPU only;
about a minute (generating the workload is most of it)."""
import json
import os

import numpy as np
import pytest

from oracle import Weighted, certificates
from oracle.problem import lipschitz
from synthetic import config_realistic

pytestmark = pytest.mark.slow
GOLD = os.path.join(os.path.dirname(__file__), "golden", "realistic_seed0_oracle.json")


def test_stored_optimum_meets_the_kkt_conditions():
    g = json.load(open(GOLD))
    if "z_star" not in g:
        pytest.skip("no stored optimum")
    prob = config_realistic(0, workers=min(16, os.cpu_count() or 1))
    assert g["value_sum"] == pytest.approx(float(sum(float(np.sum(v.astype(np.float64))) for v in prob.val)),
                                           rel=1e-12)
    W = Weighted(prob)
    zs = np.asarray(g["z_star"], dtype=np.float64)
    assert zs.shape == (prob.n,)
    c = certificates(W, zs, L=lipschitz(W, iters=5))
    assert c["infeas"] == 0.0
    assert c["pg"] <= 1e-12 and c["kkt"] <= 1e-12, c
    assert c["f"] == pytest.approx(g["f_star"], rel=1e-12)
    assert int((zs <= W.lb).sum()) == g["exact"]["at_lb"] and int((zs >= W.ub).sum()) == g["exact"]["at_ub"]
    assert float(np.linalg.norm(W.stacked_weighted_dose(zs))) == pytest.approx(g["dose_norm_star"], rel=1e-12)
