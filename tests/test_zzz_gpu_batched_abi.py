"""The batched entry points (rpt_plans_create_batched, rpt_plan_batch_query,
rpt_admm_bb_solve_batched) on the GPU: the library's own stacking gives the
same plan as the generator's block-diagonal stacking, and the per-problem
results of one batched solve are the problems' own optima (checked block by
block against the oracle), on several ring configurations.

Tolerance.  eps_abs = eps_rel = 1e-7 is the tightest decade the float32 row
passes reach on these problems: at 1e-8 the GPU's primal residual stalls at
about 3.4 eps_prim (measured on the bundled row path; the x-updates cannot be
computed more accurately than the float32 operator, whose elements carry
relative errors of order sqrt(L) eps32 for rows of L entries), while the
float64 oracle converges there.  The solves use the bundled row path with
exact sums (accumulate = 1): its operator is exact up to its float32 products
and order-independent, so every ring configuration gives the same iterates bit
for bit; with float atomics the rounding noise of the sums varies from pass to
pass, and at 1e-7 the residual of these problems can stall just above eps."""
import numpy as np
import pytest

from oracle import Weighted, lsq_box
from synthetic import random_problem, block_diagonal

from tests.gpu_util import gpu_lib, plan_of

pytestmark = pytest.mark.gpu

RINGS = [dict(accumulate=1), dict(accumulate=1, autotune=1),
         dict(accumulate=1, chunk_entries=512, chunk_rows=8, stages=2),
         dict(accumulate=1, chunk_entries=1024, chunk_rows=32, stages=3)]


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def _probs():
    return [random_problem(31, m=300, n=40, N=3, mean_row=8.0, ub=6.0),
            random_problem(32, m=500, n=70, N=3, mean_row=12.0, ub=6.0, long_rows=3),
            random_problem(33, m=200, n=25, N=3, mean_row=5.0, ub=6.0)]


def test_batched_entry_points(rpt):
    probs = _probs()
    big = block_diagonal(probs)
    with rpt.Plan.batched(probs) as P, plan_of(rpt, big) as Q:
        sp, sq = P.stats(), Q.stats()
        for key in ("m", "n", "N", "m_active", "nnz", "matrix_bytes", "default_rho", "const_term"):
            assert sp[key] == sq[key], key
        np.testing.assert_array_equal(P.batch_offsets(), [0, 40, 110, 135])
        np.testing.assert_array_equal(Q.batch_offsets(), [0, 135])


@pytest.mark.parametrize("ring", range(len(RINGS)))
def test_batched_solve_reaches_every_optimum_on_every_ring(rpt, ring):
    probs = _probs()
    with rpt.Plan.batched(probs, **RINGS[ring]) as P:
        st = P.stats()
        xs, info = P.admm_bb_solve_batched(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert st["row_path"] == 4
    assert info["status"] == 0, info
    assert [x.size for x in xs] == [40, 70, 25]
    for x, p in zip(xs, probs):
        W = Weighted(p)
        xo = lsq_box(W)
        fo = W.f(xo)
        assert np.all(x >= p.lb) and np.all(x <= p.ub)
        assert (W.f(x) - fo) / fo <= 1e-6
    # the same bits on every ring configuration (order-independent fixed-point sums)
    with rpt.Plan.batched(probs, accumulate=1) as P0:
        xs0, info0 = P0.admm_bb_solve_batched(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert info0["iterations"] == info["iterations"]
    for a, b in zip(xs, xs0):
        np.testing.assert_array_equal(a, b)
