"""The allocation-free operator entry point (rpt_normal_apply_noalloc).

It serves callers that cannot allocate device memory and therefore cannot
create a plan: their CSR matrix and vectors already live in device memory they
own.  This test hands it caller-owned device arrays and checks its output
against the plan-based operator (rpt_apply_normal) on the same scenario, within
the float32 error bound the operator tests use, on two calls in a row (the
second with a different vector, so stale scratch contents would show).
"""
import numpy as np
import pytest

from synthetic import random_problem
from oracle import Weighted
from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound

pytestmark = pytest.mark.gpu


def test_noalloc_operator_matches_plan_operator():
    rpt = gpu_lib()
    import torch
    prob = random_problem(41, m=900, n=150, N=1, mean_row=20.0, long_rows=4, empty_frac=0.2)
    W = Weighted(prob)
    dev = torch.device("cuda:0")
    # caller-owned device arrays
    rp = torch.tensor(prob.row_ptr[0], dtype=torch.int32, device=dev)
    ci = torch.tensor(prob.col_idx[0], dtype=torch.int32, device=dev)
    va = torch.tensor(prob.val[0], dtype=torch.float32, device=dev)
    w = torch.tensor(prob.voxel_w.astype(np.float32), device=dev)
    v = torch.empty(prob.n, dtype=torch.float32, device=dev)
    u = torch.empty(prob.n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(3)
    k = fp32_op_bound(prob)
    Aa = abs(W.At[0])
    with plan_of(rpt, prob) as P:
        for call, rho in enumerate((2.5, 0.75)):
            V = rng.normal(size=prob.n) * rng.uniform(0.5, 3.0, size=prob.n)
            ref = P.apply_normal(V[None, :], rho)[0]
            v.copy_(torch.tensor(V.astype(np.float32)))
            rpt.normal_apply_noalloc(prob.m, prob.n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), w.data_ptr(),
                                     v.data_ptr(), rho, u.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize(dev)
            got = u.cpu().numpy().astype(np.float64)
            mag = Aa.T @ (Aa @ np.abs(V)) + 0.5 * rho * np.abs(V)
            err = np.abs(got - ref)
            assert np.all(err <= 2.0 * k * mag + 1e-30), (call, float(np.max(err / np.maximum(mag, 1e-30))))


def test_noalloc_rejects_bad_sizes():
    rpt = gpu_lib()
    with pytest.raises(rpt.RptError) as e:
        rpt.normal_apply_noalloc(10, 9000, 1, 1, 1, 1, 1, 1.0, 1)
    assert e.value.status == rpt.EUNSUPPORTED
    with pytest.raises(rpt.RptError) as e:
        rpt.normal_apply_noalloc(0, 10, 1, 1, 1, 1, 1, 1.0, 1)
    assert e.value.status == rpt.EINVAL
