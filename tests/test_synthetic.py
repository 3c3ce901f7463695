"""The seeded input generator against its stated recipe (no method arithmetic
here: shapes, value ranges, scenario sets, truncation and scaling rules, and
the separability of block-diagonal stacking, checked with the oracle)."""
import itertools

import numpy as np
import pytest

from synthetic import (config_tiny_plain, config_realistic, random_problem, block_diagonal,
                       scenario_set_13, scenario_set_49, reweighted, sample_weights, N_WEIGHT_SLOTS)
from synthetic.phantom import _bragg
from oracle import Weighted, lsq_box


def _csr_ok(prob):
    for s in range(prob.N):
        rp, ci, va = prob.row_ptr[s], prob.col_idx[s], prob.val[s]
        assert rp.dtype == np.int32 and ci.dtype == np.int32 and va.dtype == np.float32
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == ci.size == va.size
        assert ci.size == 0 or (ci.min() >= 0 and ci.max() < prob.n)
        for i in range(prob.m):
            assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
        assert np.all(np.isfinite(va)) and np.all(va >= 0)


def test_scenario_sets_are_the_stated_combinations():
    s13 = scenario_set_13()
    assert len(set(s13)) == 13 and s13[0] == (0.0, 0.0, 0.0, 0.0)
    shifts = [sc for sc in s13 if sc[3] == 0.0 and sc[:3] != (0.0, 0.0, 0.0)]
    assert sorted(shifts) == sorted([tuple(v) + (0.0,) for v in
                                     (3.0 * e * g for e in np.eye(3) for g in (1.0, -1.0))])
    ranged = [sc for sc in s13 if sc[3] != 0.0]
    assert sorted(ranged) == sorted((0.0, 0.0, dz, k) for dz in (0.0, 3.0, -3.0) for k in (0.035, -0.035))
    s49 = scenario_set_49()
    assert len(set(s49)) == 49
    lattice = {sc[:3] for sc in s49 if sc[3] == 0.0}
    assert lattice == set(itertools.product((-3.0, 0.0, 3.0), repeat=3))
    assert sum(1 for sc in s49 if sc[3] != 0.0) == 22


def test_bragg_curve_shape():
    for R in (20.0, 80.0, 150.0):
        sR = 0.012 * R + 1.0
        assert _bragg(np.array([R]), R)[0] == pytest.approx(1.0)
        assert _bragg(np.array([R - 1e-9]), R)[0] == pytest.approx(1.0, abs=1e-9)   # continuous at R
        assert _bragg(np.array([R - 10 * sR]), R)[0] == pytest.approx(0.25, abs=1e-9)
        assert _bragg(np.array([R + 4 * sR]), R)[0] < 4e-4
        d = np.linspace(0.0, R, 200)
        assert np.all(np.diff(_bragg(d, R)) >= 0)                                  # rises to the peak
        d = np.linspace(R, R + 5 * sR, 200)
        assert np.all(np.diff(_bragg(d, R)) <= 0)                                  # falls beyond it


def test_tiny_config_recipe():
    prob = config_tiny_plain(0)
    assert (prob.n, prob.N) == (200, 13) and prob.m == 8000
    _csr_ok(prob)
    lab = prob.labels
    assert set(np.unique(lab)) == {0, 1, 2}
    np.testing.assert_array_equal(prob.voxel_w, np.where(lab == 1, 100.0, np.where(lab == 2, 10.0, 1.0)))
    np.testing.assert_array_equal(prob.presc, np.where(lab == 1, 70.0, 0.0))
    # voxel centres inside the r = 6 mm and r = 4 mm spheres (volumes of 113 and 34 voxels of 8 mm^3)
    assert 100 <= int((lab == 1).sum()) <= 150 and 25 <= int((lab == 2).sum()) <= 45
    # scaling: x = 1 gives a mean nominal target dose of 70/3
    d1 = prob.csr(0) @ np.ones(prob.n)
    assert d1[lab == 1].mean() == pytest.approx(70.0 / 3.0, rel=1e-5)
    # truncation: entries below 1e-3 of each scenario's maximum are dropped
    for s in range(prob.N):
        v = prob.val[s]
        assert v.min() >= 1e-3 * v.max() * (1 - 1e-6)
    np.testing.assert_array_equal(prob.lb, 0.0)
    np.testing.assert_array_equal(prob.ub, 10.0)


def test_realistic_recipe_small_scale():
    """The realistic generator at reduced scale: the truncation is tuned so the
    nominal scenario has the requested entries per spot column, and the target
    scaling rule holds."""
    prob = config_realistic(3, n_spots=600, nnz_per_col=300.0, workers=0, scale=0.35)
    assert prob.n == 600 and prob.N == 13
    _csr_ok(prob)
    assert prob.nnz()[0] / prob.n == pytest.approx(300.0, rel=0.01)
    lab = prob.labels
    assert set(np.unique(lab)) <= {0, 1, 2, 3, 4} and {0, 1} <= set(np.unique(lab))
    d1 = prob.csr(0) @ np.ones(prob.n)
    assert d1[lab == 1].mean() == pytest.approx(70.0 / 3.0, rel=1e-5)
    # every spot reaches the body in the nominal scenario
    assert np.all(np.diff(prob.csr(0).tocsc().indptr) > 0)


def test_random_problem_has_the_promised_edge_structure():
    prob = random_problem(7, m=400, n=50, N=3, mean_row=6.0, empty_frac=0.3, long_rows=2, zero_w_frac=0.1)
    _csr_ok(prob)
    for s in range(prob.N):
        lens = np.diff(prob.row_ptr[s])
        assert 0.2 < np.mean(lens == 0) < 0.4
        assert np.any(lens == 1)
        assert np.sum(lens == prob.n) >= 1
    assert np.any(prob.voxel_w == 0.0)


def test_block_diagonal_optimum_is_the_parts_side_by_side():
    parts = [random_problem(k, m=60 + 20 * k, n=6 + 2 * k, N=2, mean_row=4.0, ub=3.0, scen_weight=False)
             for k in range(3)]
    big = block_diagonal(parts)
    assert big.m == sum(p.m for p in parts) and big.n == sum(p.n for p in parts) and big.N == 2
    _csr_ok(big)
    Wb = Weighted(big)
    xb = lsq_box(Wb)
    fsum = 0.0
    for (r0, m, c0, n), p in zip(big.meta["blocks"], parts):
        Wp = Weighted(p)
        xp = lsq_box(Wp)
        fsum += Wp.f(xp)
        np.testing.assert_allclose(xb[c0:c0 + n], xp, rtol=1e-6, atol=1e-8)
        np.testing.assert_array_equal(big.voxel_w[r0:r0 + m], p.voxel_w)
    assert Wb.f(xb) == pytest.approx(fsum, rel=1e-10)


def test_weight_sweep_inputs():
    prob = config_tiny_plain(0)
    rng = np.random.default_rng(11)
    for _ in range(20):
        sw, d = sample_weights(rng, prob.labels)
        assert sw.shape == (N_WEIGHT_SLOTS,)
        present = set(np.unique(prob.labels))
        for k in range(N_WEIGHT_SLOTS):
            if k in present:
                assert 0.1 <= sw[k] <= 100.0
            else:
                assert sw[k] == 0.0
        assert 60.0 <= d <= 75.0
        q = reweighted(prob, sw, d)
        np.testing.assert_array_equal(q.voxel_w, sw[prob.labels])
        np.testing.assert_array_equal(q.presc, np.where(prob.labels == 1, d, 0.0))
        assert q.val is prob.val                      # matrices shared, not copied


def test_realistic_workload_matches_the_golden_file():
    """The full-size workload regenerates exactly what the stored golden values
    were computed on (entry counts per scenario and the sum of all values)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "realistic_seed0_oracle.json")))
    prob = config_realistic(0, workers=8)
    assert (prob.m, prob.n, prob.N) == (g["m"], g["n"], g["N"])
    assert prob.nnz() == g["nnz"]
    value_sum = float(sum(float(np.sum(v.astype(np.float64))) for v in prob.val))
    assert value_sum == pytest.approx(g["value_sum"], rel=1e-12)
