"""Cached-factor x-update (App. A, the paper's subproblem solver) on the GPU:
B_s = A~_s^T A~_s + (rho/2) I formed, factored and inverted in FP32 once per
(plan, rho), then x_s = B_s^{-1} c_s every iteration.  Checked against the
oracle's ADMM-BB with exact (float64 Cholesky) subproblems, iterate by
iterate, and against the exact optimum."""
import math

import numpy as np
import pytest

from oracle import Weighted, admm_bb, default_rho, lsq_box, certificates
from synthetic import random_problem, config_tiny_plain

from tests.gpu_util import gpu_lib, plan_of, max_col_count

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


@pytest.mark.parametrize("path", [1, 2, 3, 4])
def test_iterates_match_oracle_cholesky_admm(rpt, path):
    """Error budget of one x-update: the FP32 inverse of B_s (Cholesky, then
    L^{-T} L^{-1}) is accurate to about 4 n cond(B_s) eps32 relative, and B_s
    itself carries (K + 2) eps32 |A~_s|'|A~_s| from its FP32 sums (K = longest
    column); both act through ||B_s^{-1}|| <= 2/rho.  k iterations add up."""
    prob = random_problem(23, m=400, n=60, N=3, mean_row=9.0, scen_weight=True, ub=6.0)
    W = Weighted(prob)
    rho = default_rho(W)
    K = max_col_count(prob)
    kappa = []
    for s in range(prob.N):
        ev = np.linalg.eigvalsh(W.B_dense(s, rho))
        kappa.append(ev[-1] / ev[0])
    with plan_of(rpt, prob, row_path=path) as P:
        for k in (1, 2, 4, 10):
            ref = admm_bb(W, rho=rho, max_iter=k, eps_abs=0.0, eps_rel=0.0, subproblem="chol")
            _, info = P.admm_bb_solve(rho=rho, max_iter=k, eps_abs=0.0, eps_rel=0.0, subproblem=rpt.SUB_CHOL)
            z, X, Y = P.state_get()
            e2 = 0.0
            for s in range(prob.N):
                xs = np.abs(ref["x"][s])
                Aa = abs(W.At[s])
                cs = np.linalg.norm(W.b(s)) + 0.5 * rho * np.linalg.norm(ref["x"][s]) + np.linalg.norm(ref["y"][s])
                e = (2.0 / rho) * EPS32 * (4.0 * prob.n * kappa[s] * cs + (K + 2) * np.linalg.norm(Aa.T @ (Aa @ xs)))
                e2 += e * e
            bound = 10.0 * k * math.sqrt(e2)
            assert np.linalg.norm(X - ref["x"]) <= bound, (k, np.linalg.norm(X - ref["x"]), bound)
            assert np.linalg.norm(z - ref["z"]) <= bound
            sz = np.abs(ref["z"]).max()
            np.testing.assert_allclose(z, ref["z"], rtol=1e-4, atol=1e-5 * sz)
            assert info["row_passes"] <= 2                      # only the final objective pass
            assert info["step"] == pytest.approx(ref["step"], rel=1e-3)


def test_reaches_the_exact_optimum_and_caches_the_factor(rpt):
    prob = config_tiny_plain(0)
    W = Weighted(prob)
    xs = lsq_box(W)
    fs = W.f(xs)
    with plan_of(rpt, prob) as P:
        # 1e-6: the FP32 inverse leaves a residual floor near 1e-8 relative
        z, info = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, subproblem=rpt.SUB_CHOL)
        z2, info2 = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, subproblem=rpt.SUB_CHOL)
        zc, infoc = P.admm_bb_solve(subproblem=rpt.SUB_CHOL, rho_scale=2.0)   # another rho: new factor
    assert info["status"] == 0 and (W.f(z) - fs) / fs <= 1e-6, ((W.f(z) - fs) / fs, info)
    assert certificates(W, z)["pg"] < 1e-3
    assert info["setup_seconds"] > 0 and info2["setup_seconds"] == 0
    np.testing.assert_allclose(z2, z, rtol=1e-6, atol=1e-9)
    assert infoc["setup_seconds"] > 0 and infoc["status"] == 0


@pytest.mark.parametrize("fmt", [1, 2])
def test_quantised_plan_uses_the_dequantised_matrix(rpt, fmt):
    from oracle.quantize import quantised_problem
    prob = random_problem(24, m=500, n=50, N=2, mean_row=10.0, ub=5.0)
    Wq = Weighted(quantised_problem(prob, {1: "bf16", 2: "fp8"}[fmt]))
    xq = lsq_box(Wq)
    with plan_of(rpt, prob, value_format=fmt, index_width=16) as P:
        z, info = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, subproblem=rpt.SUB_CHOL)
    assert info["status"] == 0 and (Wq.f(z) - Wq.f(xq)) / Wq.f(xq) <= 1e-6
