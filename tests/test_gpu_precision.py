"""Reduced-precision storage forms on the GPU against the oracle.

Values stored as bfloat16 or FP8-e4m3 codes with per-column FP32 scales, and
column indices stored as uint16.  The oracle applies the same storage
definition (oracle/quantize.py) and evaluates the method in float64 on the
dequantised matrices; the GPU must match that within the float32 bound of the
plain path.  The error of a quantised plan against the original (float32)
problem is a property of the storage form, not of the kernels; it is stated per
result and bounded loosely.
"""
import numpy as np
import pytest

from oracle import Weighted, lsq_box, certificates
from oracle.quantize import quantised_problem
from synthetic import random_problem, config_tiny_plain

from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound, fixed_point_slack

pytestmark = pytest.mark.gpu

VF = {"f32": 0, "bf16": 1, "fp8": 2}
FORMATS = [("bf16", 32), ("bf16", 16), ("fp8", 32), ("fp8", 16), ("f32", 16)]


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def _abs_W(W):
    class A:
        pass
    a = A()
    a.At = [abs(M) for M in W.At]
    a.pt = [np.abs(p) for p in W.pt]
    return a


@pytest.mark.parametrize("path", [1, 2, 3, 4])
@pytest.mark.parametrize("fmt,iw", FORMATS)
def test_operator_gradient_objective_on_dequantised_matrix(rpt, fmt, iw, path):
    prob = random_problem(11, m=700, n=90, N=3, mean_row=14.0, long_rows=2, scen_weight=True)
    W = Weighted(prob if fmt == "f32" else quantised_problem(prob, fmt))
    Wa = _abs_W(W)
    k = fp32_op_bound(prob)
    rng = np.random.default_rng(5)
    V = rng.normal(size=(prob.N, prob.n))
    x = rng.uniform(0.0, 4.0, size=prob.n)
    with plan_of(rpt, prob, value_format=VF[fmt], index_width=iw, row_path=path) as P:
        U = P.apply_normal(V, 1.3)
        g, f = P.gradient(x)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], 1.3)
        mag = Wa.At[s].T @ (Wa.At[s] @ np.abs(V[s])) + 0.65 * np.abs(V[s])
        # bundled path: fixed-point slack, its bound taken on codes (scales up to 2^20 apart)
        slack = fixed_point_slack(prob, s, V[s], value_scale=2.0 ** 20) if path == 4 else 0.0
        assert np.all(np.abs(U[s] - ref) <= k * mag + slack + 1e-300), (fmt, iw, path, s)
    gmag = sum(2.0 * (Wa.At[s].T @ (Wa.At[s] @ np.abs(x) + Wa.pt[s])) for s in range(prob.N))
    gslack = (sum(2.0 * fixed_point_slack(prob, s, x, resid=True, value_scale=2.0 ** 20) for s in range(prob.N))
              if path == 4 else 0.0)
    assert np.all(np.abs(g - W.grad(x)) <= k * gmag + gslack + 1e-300)
    fmag = sum(float(np.sum((Wa.At[s] @ np.abs(x) + Wa.pt[s]) ** 2)) for s in range(prob.N))
    assert abs(f - W.f(x)) <= 2 * k * fmag


@pytest.fixture(scope="module")
def tiny():
    prob = config_tiny_plain(0)
    W0 = Weighted(prob)
    x0 = lsq_box(W0)
    return prob, W0, W0.f(x0)


# loose bounds on the storage form's own error (objective of the quantised
# optimum on the original problem, relative to the original optimum)
FORM_BOUND = {"bf16": 1e-3, "fp8": 5e-2}


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_quantised_solve_reaches_the_dequantised_optimum(rpt, tiny, fmt):
    prob, W0, f0 = tiny
    Wq = Weighted(quantised_problem(prob, fmt))
    xq = lsq_box(Wq)
    fq = Wq.f(xq)
    with plan_of(rpt, prob, value_format=VF[fmt], index_width=16) as P:
        z, info = P.admm_bb_solve(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert np.all(z >= prob.lb) and np.all(z <= prob.ub)
    # parity: the GPU optimum of the quantised plan is the oracle's optimum of the dequantised problem
    assert (Wq.f(z) - fq) / fq <= 1e-6, ((Wq.f(z) - fq) / fq, info)
    assert info["f"] == pytest.approx(Wq.f(z), rel=1e-6)
    assert certificates(Wq, z)["pg"] < 1e-3
    # the storage form's error against the float32 problem, stated
    err = (W0.f(z) - f0) / f0
    print(f"{fmt}: objective of the quantised optimum on the original problem: +{err:.3e} relative")
    assert 0.0 <= err + 1e-9 and err <= FORM_BOUND[fmt]
