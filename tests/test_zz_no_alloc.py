"""The allocation-free operator entry point (rpt_normal_apply_noalloc).

It serves callers that cannot allocate device memory and therefore cannot
create a plan: their CSR matrix and vectors already live in device memory they
own (a pool or framework that owns all device memory, or a loop that must not
block on the allocator).  These tests hand it caller-owned device arrays and
check its output against the float64 oracle's scenario operator
(oracle.Weighted.normal_apply, App. A) element by element, within the float32
bound of the operator tests, on consecutive calls (each with a different
vector, so stale scratch contents would show).  They also check that the calls
leave the device's free memory and the caller's allocator untouched, exercise
the largest supported spot count (8192, which needs more than the default 48 KB
of shared memory), and the documented skipping of column indices outside
[0, n).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from synthetic import random_problem
from oracle import Weighted
from tests.gpu_util import gpu_lib, fp32_op_bound

pytestmark = pytest.mark.gpu


def _device_arrays(torch, dev, rp, ci, va, w, n):
    return (torch.tensor(rp, dtype=torch.int32, device=dev), torch.tensor(ci, dtype=torch.int32, device=dev),
            torch.tensor(va, dtype=torch.float32, device=dev), torch.tensor(w.astype(np.float32), device=dev),
            torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.float32, device=dev))


def _call(rpt, torch, dev, m, n, arrs, V, rho):
    rp, ci, va, w, v, u = arrs
    v.copy_(torch.tensor(V.astype(np.float32)))
    stream = torch.cuda.current_stream(dev)
    rpt.normal_apply_noalloc(m, n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), w.data_ptr(), v.data_ptr(), rho,
                             u.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    return u.cpu().numpy().astype(np.float64)


def test_noalloc_operator_matches_oracle_and_allocates_nothing():
    rpt = gpu_lib()
    import torch
    prob = random_problem(41, m=900, n=150, N=1, mean_row=20.0, long_rows=4, empty_frac=0.2)
    W = Weighted(prob)
    dev = torch.device("cuda:0")
    arrs = _device_arrays(torch, dev, prob.row_ptr[0], prob.col_idx[0], prob.val[0], prob.voxel_w, prob.n)
    rng = np.random.default_rng(3)
    k = fp32_op_bound(prob)
    Aa = abs(W.At[0])
    free0 = alloc0 = None
    for call, rho in enumerate((2.5, 0.75, 4.0)):
        V = rng.normal(size=prob.n) * rng.uniform(0.5, 3.0, size=prob.n)
        got = _call(rpt, torch, dev, prob.m, prob.n, arrs, V, rho)
        ref = W.normal_apply(0, V, rho)
        mag = Aa.T @ (Aa @ np.abs(V)) + 0.5 * rho * np.abs(V)
        err = np.abs(got - ref)
        assert np.all(err <= k * mag + 1e-30), (call, float(np.max(err / np.maximum(mag, 1e-30))))
        free, _ = torch.cuda.mem_get_info(dev)
        alloc = torch.cuda.memory_allocated(dev)
        if call == 0:
            # the first call may load the library's kernels onto the device; after
            # it, calls must not change the device's free memory or torch's allocator
            free0, alloc0 = free, alloc
        else:
            assert free == free0 and alloc == alloc0, (call, free0 - free, alloc - alloc0)


def test_noalloc_at_the_spot_limit_and_with_out_of_range_columns():
    rpt = gpu_lib()
    import torch
    dev = torch.device("cuda:0")
    n, m = 8192, 300
    rng = np.random.default_rng(7)
    lens = rng.integers(0, 60, size=m)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    va = rng.uniform(0.0, 2.0, size=rp[-1]).astype(np.float32)
    # a few entries point outside [0, n): the call skips them
    bad = rng.choice(rp[-1], size=25, replace=False)
    ci[bad[:12]] = n + rng.integers(0, 1000, size=12)
    ci[bad[12:]] = -1 - rng.integers(0, 1000, size=13)
    w = rng.uniform(0.1, 10.0, size=m)
    keep = (ci >= 0) & (ci < n)
    rows = np.repeat(np.arange(m), lens)
    A = sp.csr_matrix((va[keep].astype(np.float64), (rows[keep], ci[keep])), shape=(m, n))
    Aa = abs(A)
    L = int(lens.max())
    K = int(np.bincount(ci[keep], minlength=n).max())
    kf = (L + K + 8) * float(np.finfo(np.float32).eps)
    arrs = _device_arrays(torch, dev, rp, ci, va, w, n)
    for call, rho in enumerate((1.5, 0.0)):
        V = rng.normal(size=n)
        got = _call(rpt, torch, dev, m, n, arrs, V, rho)
        ref = A.T @ (w * (A @ V)) + 0.5 * rho * V
        mag = Aa.T @ (w * (Aa @ np.abs(V))) + 0.5 * rho * np.abs(V)
        assert np.all(np.abs(got - ref) <= kf * mag + 1e-30), call


def test_noalloc_rejects_bad_sizes():
    rpt = gpu_lib()
    with pytest.raises(rpt.RptError) as e:
        rpt.normal_apply_noalloc(10, 9000, 1, 1, 1, 1, 1, 1.0, 1)
    assert e.value.status == rpt.EUNSUPPORTED
    with pytest.raises(rpt.RptError) as e:
        rpt.normal_apply_noalloc(0, 10, 1, 1, 1, 1, 1, 1.0, 1)
    assert e.value.status == rpt.EINVAL
