"""The batched entry points (rpt_plans_create_batched, rpt_plan_batch_query,
rpt_admm_bb_solve_batched) on the GPU: the library's own stacking gives the
same plan as the generator's block-diagonal stacking, and the per-problem
results of one batched solve are the problems' own optima (checked block by
block against the oracle)."""
import numpy as np
import pytest

from oracle import Weighted, lsq_box
from synthetic import random_problem, block_diagonal

from tests.gpu_util import gpu_lib, plan_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def test_batched_entry_points(rpt):
    probs = [random_problem(31, m=300, n=40, N=3, mean_row=8.0, ub=6.0),
             random_problem(32, m=500, n=70, N=3, mean_row=12.0, ub=6.0, long_rows=3),
             random_problem(33, m=200, n=25, N=3, mean_row=5.0, ub=6.0)]
    big = block_diagonal(probs)
    with rpt.Plan.batched(probs) as P, plan_of(rpt, big) as Q:
        sp, sq = P.stats(), Q.stats()
        for key in ("m", "n", "N", "m_active", "nnz", "matrix_bytes", "default_rho", "const_term"):
            assert sp[key] == sq[key], key
        np.testing.assert_array_equal(P.batch_offsets(), [0, 40, 110, 135])
        np.testing.assert_array_equal(Q.batch_offsets(), [0, 135])
        xs, info = P.admm_bb_solve_batched(eps_abs=1e-8, eps_rel=1e-8, max_iter=20000)
    assert info["status"] == 0
    assert [x.size for x in xs] == [40, 70, 25]
    for x, p in zip(xs, probs):
        W = Weighted(p)
        xo = lsq_box(W)
        fo = W.f(xo)
        assert np.all(x >= p.lb) and np.all(x <= p.ub)
        assert (W.f(x) - fo) / fo <= 1e-6
