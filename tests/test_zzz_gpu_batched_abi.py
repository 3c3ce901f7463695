"""The batched entry points (rpt_plans_create_batched, rpt_plan_batch_query,
rpt_admm_bb_solve_batched) on the GPU.  A batched plan solves its problems side
by side, each with its own penalty, BB step and stopping test: every problem's
result is its own optimum (checked against the oracle), and with the exact
fixed-point row sums (accumulate = 1) every problem follows, bit for bit and
iteration for iteration, the solve of a plan that holds it alone.

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
        for key in ("m", "n", "N", "m_active", "nnz"):
            assert sp[key] == sq[key], key
        # the same sums in another order
        for key in ("default_rho", "const_term"):
            assert sp[key] == pytest.approx(sq[key], rel=1e-12), key
        np.testing.assert_array_equal(P.batch_offsets(), [0, 40, 110, 135])
        np.testing.assert_array_equal(Q.batch_offsets(), [0, 135])
        # calls that take one problem's vectors refuse a batched plan
        with pytest.raises(rpt.RptError) as e:
            P.admm_bb_solve()
        assert e.value.status == rpt.EUNSUPPORTED
        with pytest.raises(rpt.RptError) as e:
            P.objective(np.zeros(sp["n"]))
        assert e.value.status == rpt.EUNSUPPORTED


@pytest.mark.parametrize("ring", range(len(RINGS)))
def test_batched_solve_reaches_every_optimum_on_every_ring(rpt, ring):
    probs = _probs()
    with rpt.Plan.batched(probs, **RINGS[ring]) as P:
        st = P.stats()
        xs, info, per = P.admm_bb_solve_batched(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert st["row_path"] == 4
    assert info["status"] == 0, info
    assert [x.size for x in xs] == [40, 70, 25]
    assert [q["status"] for q in per] == [0, 0, 0]
    assert info["iterations"] == max(q["iterations"] for q in per)
    assert info["inner"] == sum(q["inner"] for q in per)
    for x, p in zip(xs, probs):
        W = Weighted(p)
        xo = lsq_box(W)
        fo = W.f(xo)
        assert np.all(x >= p.lb) and np.all(x <= p.ub)
        assert (W.f(x) - fo) / fo <= 1e-6
    # the same bits on every ring configuration (order-independent fixed-point sums)
    with rpt.Plan.batched(probs, accumulate=1) as P0:
        xs0, info0, per0 = P0.admm_bb_solve_batched(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert info0["iterations"] == info["iterations"]
    assert [q["iterations"] for q in per0] == [q["iterations"] for q in per]
    for a, b in zip(xs, xs0):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("subproblem", ["cg", "chol"])
def test_every_problem_follows_its_own_solve(rpt, subproblem):
    """Per problem: the iterations, penalty, objective and result of the plan
    of that problem alone (own penalty, BB step and stop), and an earlier stop
    for the problems that converge first.  CG subproblems: the same bits (the
    units' layouts and every reduction are those of the problem's own plan,
    with the widest problem's extra spots adding exact zeros).  Cached factor:
    the float32 inverse of the padded B_s is applied with another summation
    order when the spot counts differ, so there the results agree to rounding."""
    probs = _probs()
    kw = dict(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000,
              subproblem=rpt.SUB_CHOL if subproblem == "chol" else rpt.SUB_CG)
    with rpt.Plan.batched(probs, accumulate=1) as P:
        xs, info, per = P.admm_bb_solve_batched(**kw)
    alone = []
    for p in probs:
        with plan_of(rpt, p, accumulate=1) as Q:
            x, i = Q.admm_bb_solve(**kw)
            alone.append((x, i))
    for k, (x, i) in enumerate(alone):
        assert per[k]["status"] == i["status"] == 0
        assert per[k]["rho"] == i["rho"], k
        if subproblem == "cg":
            assert per[k]["iterations"] == i["iterations"], k
            assert per[k]["f"] == pytest.approx(i["f"], rel=1e-12)
            np.testing.assert_array_equal(xs[k], x)
        else:
            assert abs(per[k]["iterations"] - i["iterations"]) <= 3 + 0.05 * i["iterations"], k
            assert per[k]["f"] == pytest.approx(i["f"], rel=1e-6)
            np.testing.assert_allclose(xs[k], x, rtol=1e-4, atol=1e-4 * max(1.0, np.abs(x).max()))
    iters = [q["iterations"] for q in per]
    assert len(set(iters)) > 1, iters          # the problems stop at different iterations
    assert info["iterations"] == max(iters)
