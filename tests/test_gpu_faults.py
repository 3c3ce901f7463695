"""Failure detection without a GPU fault: failures are made on the host and the
library must report them and stay usable.

* A forced wait timeout: with the testing hook rpt_device_opts.inject_timeout
  the bulk-copy rings' producer (CSR and bundled rings) issues no copy, every
  consumer wait runs out after its one-second bound, the kernel sets the plan's
  error word and returns; the call reports RPT_TIMEOUT, and the context keeps
  working.
* Out of device memory: rpt_device_opts.device_mem_cap caps a plan's
  allocations, so plan creation fails with RPT_ENOMEM instead of exhausting the
  device.
"""
import numpy as np
import pytest

from oracle import Weighted
from synthetic import random_problem

from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def _prob():
    return random_problem(51, m=400, n=50, N=2, mean_row=8.0)


@pytest.mark.parametrize("path", [2, 4])
def test_injected_wait_timeout_is_reported_and_the_context_survives(rpt, path):
    prob = _prob()
    V = np.random.default_rng(2).uniform(0.0, 1.0, size=(prob.N, prob.n))
    with plan_of(rpt, prob, row_path=path, inject_timeout=1) as P:
        with pytest.raises(rpt.RptError) as e:
            P.apply_normal(V, 0.0)
        assert e.value.status == rpt.TIMEOUT
        with pytest.raises(rpt.RptError) as e:
            P.admm_bb_solve(max_iter=1, cg_max=1, use_graph=0)
        assert e.value.status == rpt.TIMEOUT
    W = Weighted(prob)
    k = fp32_op_bound(prob)
    with plan_of(rpt, prob, row_path=path) as P:
        U = P.apply_normal(V, 0.0)
    for s in range(prob.N):
        Aa = abs(W.At[s])
        assert np.all(np.abs(U[s] - W.normal_apply(s, V[s], 0.0)) <= k * (Aa.T @ (Aa @ V[s])) + 1e-300)


def test_device_memory_cap_gives_enomem(rpt):
    prob = _prob()
    with pytest.raises(rpt.RptError) as e:
        plan_of(rpt, prob, device_mem_cap=100000)
    assert e.value.status == rpt.ENOMEM
    with plan_of(rpt, prob) as P:
        assert P.stats()["nnz"] == sum(int(v.size) for v in prob.val)
