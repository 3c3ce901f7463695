"""Helpers for the GPU tests (test infrastructure)."""
import numpy as np
import pytest

EPS32 = float(np.finfo(np.float32).eps)


def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_14568_gb300 import build as build_mod
    from paper_2304_14568_gb300 import rpt
    build_mod.build()
    return rpt


def plan_of(rpt, prob, **kw):
    return rpt.Plan.from_problem(prob, **kw)


def max_row_len(prob):
    return max(int(np.diff(rp).max(initial=0)) for rp in prob.row_ptr)


def max_col_count(prob):
    return max(int(np.bincount(ci, minlength=prob.n).max(initial=0)) for ci in prob.col_idx)


def fp32_op_bound(prob):
    """Error factor of a float32 dot (length <= L) followed by a float32 scatter
    (<= K terms per column) and a few roundings: (L + K + 8) eps32."""
    return (max_row_len(prob) + max_col_count(prob) + 8) * EPS32
