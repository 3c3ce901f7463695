"""Batched form: several plans of uneven size in one plan (block-diagonal
stacking, so one persistent row pass covers every plan's scenarios), and the
autotuner that times the bulk-copy ring configurations at plan creation.
Checked against the oracle block by block: the stacked problem's optimum is the
plans' optima side by side."""
import numpy as np
import pytest

from oracle import Weighted, lsq_box
from synthetic import random_problem, block_diagonal

from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def _plans():
    return [random_problem(31, m=300, n=40, N=3, mean_row=8.0, ub=6.0),
            random_problem(32, m=500, n=70, N=3, mean_row=12.0, ub=6.0, long_rows=3),
            random_problem(33, m=200, n=25, N=3, mean_row=5.0, ub=6.0)]


def test_batched_operator_and_optimum_block_by_block(rpt):
    probs = _plans()
    big = block_diagonal(probs)
    rng = np.random.default_rng(8)
    V = rng.normal(size=(big.N, big.n))
    with plan_of(rpt, big, autotune=1) as P:
        st = P.stats()
        U = P.apply_normal(V, 1.1)
        z, info = P.admm_bb_solve(eps_abs=1e-8, eps_rel=1e-8, max_iter=20000)
    assert st["row_path"] == 4 and st["autotuned"] >= 2 and st["autotune_ms"] > 0
    for k, (r0, m, c0, n) in enumerate(big.meta["blocks"]):
        W = Weighted(probs[k])
        kb = fp32_op_bound(probs[k])
        Wa = [abs(M) for M in W.At]
        for s in range(big.N):
            v = V[s, c0:c0 + n]
            ref = W.normal_apply(s, v, 1.1)
            mag = Wa[s].T @ (Wa[s] @ np.abs(v)) + 0.55 * np.abs(v)
            assert np.all(np.abs(U[s, c0:c0 + n] - ref) <= kb * mag + 1e-300), (k, s)
        xs = lsq_box(W)
        fs = W.f(xs)
        assert (W.f(z[c0:c0 + n]) - fs) / fs <= 1e-6, (k, info)


def test_wide_plan_gets_a_ring_that_fits(rpt):
    # 14,000 spots: the spot vector and the 64-bit accumulator take 168 KB of
    # shared memory, so the default 2 x 3072-block-column ring does not fit beside them
    prob = random_problem(34, m=600, n=14000, N=2, mean_row=30.0, long_rows=0)
    W = Weighted(prob)
    rng = np.random.default_rng(9)
    V = rng.uniform(0.0, 1.0, size=(prob.N, prob.n))
    with plan_of(rpt, prob) as P:
        st = P.stats()
        U = P.apply_normal(V, 0.0)
    assert st["row_path"] == 4 and (st["chunk_entries"], st["stages"]) != (3072, 2)
    k = fp32_op_bound(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], 0.0)
        Aa = abs(W.At[s])
        assert np.all(np.abs(U[s] - ref) <= k * (Aa.T @ (Aa @ V[s])) + 1e-300)
