"""Parity at the benchmark's full size: the realistic workload (13 scenarios,
299,088 voxels, 5,000 spots, 126.9M stored entries) in the launch
configuration bench.py times (the library's default row path).  The oracle
evaluates every output here (a few float64 sparse products per scenario), so
the comparison is element by element with the float32 bound of the plain
path; the solve is checked against the oracle's exact optimum (stored by
tests/golden/make_realistic_golden.py) and its optimality certificate."""
import json
import os

import numpy as np
import pytest

from oracle import Weighted, certificates
from synthetic import config_realistic

from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GOLD = os.path.join(os.path.dirname(__file__), "golden", "realistic_seed0_oracle.json")


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


@pytest.fixture(scope="module")
def big(rpt):
    prob = config_realistic(0, workers=min(16, os.cpu_count() or 1))
    W = Weighted(prob)
    P = plan_of(rpt, prob)
    yield prob, W, P
    P.close()


def test_plan_is_the_benchmarked_configuration(big):
    prob, W, P = big
    st = P.stats()
    assert st["row_path"] == 4 and st["nnz"] == sum(int(v.size) for v in prob.val)
    assert st["m_active"] == 85495 and prob.n == 5000 and prob.N == 13


def test_operator_every_output(big):
    prob, W, P = big
    rng = np.random.default_rng(21)
    V = rng.uniform(0.0, 5.0, size=(prob.N, prob.n))
    rho = 1826.0
    U = P.apply_normal(V, rho)
    k = fp32_op_bound(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], rho)
        Aa = abs(W.At[s])
        mag = Aa.T @ (Aa @ V[s]) + 0.5 * rho * V[s]            # V >= 0
        err = np.abs(U[s] - ref)
        assert np.all(err <= k * mag), (s, float((err / mag).max()), k)


def test_gradient_objective_every_output(big):
    prob, W, P = big
    x = np.random.default_rng(22).uniform(0.0, 6.0, size=prob.n)
    g, f = P.gradient(x)
    k = fp32_op_bound(prob)
    gref = W.grad(x)
    gmag = sum(2.0 * (abs(W.At[s]).T @ (abs(W.At[s]) @ x + W.pt[s])) for s in range(prob.N))
    assert np.all(np.abs(g - gref) <= k * gmag)
    fmag = sum(float(np.sum((abs(W.At[s]) @ x + W.pt[s]) ** 2)) for s in range(prob.N))
    assert abs(f - W.f(x)) <= 2 * k * fmag
    assert abs(P.objective(x) - W.f(x)) <= 2 * k * fmag


def test_benchmark_solve_reaches_the_oracle_optimum(big):
    prob, W, P = big
    z, info = P.admm_bb_solve()                               # the benchmark's step: eps 1e-4
    assert info["status"] == 0
    assert np.all(z >= prob.lb) and np.all(z <= prob.ub)
    fz = W.f(z)
    assert info["f"] == pytest.approx(fz, rel=1e-5)
    c = certificates(W, z)
    assert c["pg"] < 1e-2, c
    if not os.path.exists(GOLD):
        pytest.skip("no stored oracle optimum")
    g = json.load(open(GOLD))
    assert g["value_sum"] == pytest.approx(float(sum(float(np.sum(v.astype(np.float64))) for v in prob.val)),
                                           rel=1e-12)
    fstar = g["f_star"]
    # eps = 1e-4 on the residuals of Eq. 9 leaves a small objective gap
    assert fstar <= fz * (1 + 1e-9) and (fz - fstar) / fstar <= 1e-4, ((fz - fstar) / fstar)
    # the oracle's float64 run with the same parameters takes about as many iterations
    if "admm_cg" in g:
        ref_it = g["admm_cg"]["iterations"]
        assert abs(info["iterations"] - ref_it) <= 0.1 * ref_it + 5, (info["iterations"], ref_it)


def test_cached_factor_solve_reaches_the_oracle_optimum(rpt, big):
    prob, W, P = big
    z, info = P.admm_bb_solve(subproblem=rpt.SUB_CHOL)
    assert info["status"] == 0 and info["setup_seconds"] > 0
    assert np.all(z >= prob.lb) and np.all(z <= prob.ub)
    fz = W.f(z)
    assert info["f"] == pytest.approx(fz, rel=1e-5)
    assert certificates(W, z)["pg"] < 1e-2
    if not os.path.exists(GOLD):
        pytest.skip("no stored oracle optimum")
    g = json.load(open(GOLD))
    fstar = g["f_star"]
    assert fstar <= fz * (1 + 1e-9) and (fz - fstar) / fstar <= 1e-4, ((fz - fstar) / fstar)
    if "admm_chol" in g:                         # the oracle's float64 Cholesky run: same iteration count
        ref_it = g["admm_chol"]["iterations"]
        assert abs(info["iterations"] - ref_it) <= 0.05 * ref_it + 3, (info["iterations"], ref_it)


@pytest.mark.parametrize("sub", ["cg", "chol"])
def test_tight_tolerance_objective_and_dose(rpt, big, sub):
    """At eps = 1e-7 (the tightest decade the float32 passes reach) the
    full-size solve with CG x-updates meets the stated 1e-6 on the objective
    gap and on the stacked weighted dose D = [A~_1 z; ...; A~_N z] against the
    stored exact optimum z* (measured: 1.9e-11 and 5.2e-7 after 4000
    iterations).  With float atomics the residuals of Eq. 9 can hover just
    above eps at this size while the iterate already meets both tolerances, so
    the status is not asserted (as at tight eps on the small configurations);
    the iteration cap bounds the run.
    The cached factor applies a float32 B_s^-1 whose own relative error is about
    cond(B_s) eps_32 (cond(B_s) = 124 on scenario 0 of this plan; a float32
    Cholesky inverse of it is off by 4.6e-6 in the 2-norm, measured on the CPU),
    so its x-updates carry a relative error near 1e-6 that does not shrink with
    the iteration: the objective still meets 1e-6 (measured 2.9e-8) but the
    dose stops at its floor (measured 2.0e-5), asserted with room for the
    run-to-run variation of the float atomics that form B_s."""
    prob, W, P = big
    g = json.load(open(GOLD)) if os.path.exists(GOLD) else {}
    if "z_star" not in g:
        pytest.skip("no stored oracle optimum")
    kw = dict(subproblem=rpt.SUB_CHOL) if sub == "chol" else {}
    z, info = P.admm_bb_solve(eps_abs=1e-7, eps_rel=1e-7, max_iter=4000, **kw)
    assert info["status"] in (0, 1), info                 # converged or at the cap
    assert np.all(z >= prob.lb) and np.all(z <= prob.ub)
    zs = np.asarray(g["z_star"])
    fz, fstar = W.f(z), g["f_star"]
    Ds = W.stacked_weighted_dose(zs)
    assert np.linalg.norm(Ds) == pytest.approx(g["dose_norm_star"], rel=1e-12)
    rel_dose = float(np.linalg.norm(W.stacked_weighted_dose(z) - Ds) / np.linalg.norm(Ds))
    print(f"full size {sub}: status {info['status']} iterations {info['iterations']} "
          f"objective gap {(fz - fstar) / fstar:.2e} dose error {rel_dose:.2e} "
          f"r_prim/eps_prim {info['r_prim'] / info['eps_prim']:.2f}")
    assert fstar <= fz * (1 + 1e-12) and (fz - fstar) / fstar <= 1e-6
    assert rel_dose <= (1e-6 if sub == "cg" else 1e-4), rel_dose
