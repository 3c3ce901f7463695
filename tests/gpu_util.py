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


def fixed_point_slack(prob, s, v, resid=False, value_scale=1.0):
    """Absolute slack of the bundled path's 64-bit fixed-point scatter, per spot
    column of scenario s: each contribution is rounded to a resolution of at most
    bound * 2^-59, bound = K_s max|v| (+ P_s with the prescription term), where
    K_s = max_c sum_i c_s w_i |a_ic| ||a_i||_1 and P_s = max_c sum_i c_s w_i |a_ic| p_i;
    the rounding error of one contribution is at most half of that, and column c
    takes one contribution per stored block column, at most its entry count.
    value_scale > 1 loosens it for quantised values (bounds taken on codes)."""
    import scipy.sparse as sp
    c = 1.0 if prob.scen_weight is None else float(prob.scen_weight[s])
    A = abs(prob.csr(s))
    w = c * prob.voxel_w
    l1 = np.asarray(A.sum(axis=1)).ravel()
    K = A.T @ (w * l1)
    bound = float(K.max(initial=0.0)) * float(np.max(np.abs(v), initial=0.0))
    if resid:
        bound += float((A.T @ (w * prob.presc)).max(initial=0.0))
    cnt = np.bincount(prob.col_idx[s], minlength=prob.n).astype(float)
    return cnt * bound * 2.0 ** -60 * value_scale
