"""The paper's parallel form of the oracle (oracle.parallel: cached-Cholesky
subproblems on worker processes, Sec. 2.3 / App. A) computes the same iterates
as the serial cached-Cholesky ADMM-BB: same iteration count and status, and z,
x_s, y_s equal to rounding (the same LAPACK factor and solve on both sides)."""
import numpy as np
import pytest

from oracle import Weighted, admm_bb, lsq_box
from oracle.parallel import admm_bb_chol_parallel
from synthetic import random_problem


@pytest.mark.parametrize("workers", [1, 2, 3])
def test_parallel_cholesky_admm_equals_serial(workers):
    prob = random_problem(61, m=300, n=30, N=3, mean_row=7.0, ub=5.0, scen_weight=True)
    W = Weighted(prob)
    kw = dict(eps_abs=1e-9, eps_rel=1e-9, max_iter=3000)
    ser = admm_bb(W, subproblem="chol", **kw)
    par = admm_bb_chol_parallel(W, workers=workers, blas_threads=1, **kw)
    assert par["status"] == ser["status"] == "converged"
    assert par["iterations"] == ser["iterations"]
    for key in ("z", "x", "y"):
        np.testing.assert_allclose(par[key], ser[key], rtol=1e-10, atol=1e-12 * np.abs(ser[key]).max())
    assert par["workers"] == min(workers, prob.N) and par["setup_s"] > 0
    xs = lsq_box(W)
    assert (W.f(par["z"]) - W.f(xs)) / W.f(xs) < 1e-9
