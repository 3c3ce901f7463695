"""Pins for the dose-constraint extension of the oracle (Sec. 4: ADMM takes
linear constraints such as maximum and mean dose; the formulation is a reading).

The exact constrained optimum comes from active-set enumeration, itself checked
against a library solver (SLSQP); the ADMM iteration must reach it, with its
dose-block duals equal to the KKT multipliers, and must reduce to ADMM-BB when
there are no constraint rows."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import minimize

from oracle import Weighted, admm_bb, kkt_bruteforce, lipschitz
from oracle.dose_constraints import DoseConstraint, constraint_rows, admm_bb_constrained, kkt_bruteforce_lin
from synthetic import from_dense
from tests.test_oracle_pins import _tiny_dense

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _slsqp(W, G, h):
    res = minimize(W.f, W.proj(np.full(W.n, 0.5)), jac=W.grad, method="SLSQP",
                   bounds=list(zip(W.lb, W.ub)),
                   constraints=[{"type": "ineq", "fun": lambda x: h - G @ x, "jac": lambda x: -G}],
                   options={"ftol": 1e-12, "maxiter": 2000})
    assert res.success, res.message
    return res


def _case(kind_set, seed):
    P = _tiny_dense(seed, m=12, n=4, N=2, lb=0.0, ub=6.0, sw=True)
    W = Weighted(P)
    x0 = kkt_bruteforce(W)
    dose = np.array([W.dose(s, x0) for s in range(W.N)])
    cons = []
    if "max" in kind_set:
        cons.append(DoseConstraint("max", np.array([0, 1]), 0.8 * float(dose[:, [0, 1]].max())))
    if "mean" in kind_set:
        cons.append(DoseConstraint("mean", np.arange(2, 7), 0.9 * float(dose[:, 2:7].mean(axis=1).max())))
    if "min" in kind_set:
        cons.append(DoseConstraint("min", np.array([8, 9]), 1.15 * float(dose[:, [8, 9]].min())))
    return P, W, cons


CASES = [(("max", "mean"), 31), (("min",), 32), (("max", "min"), 33)]


def test_mean_row_is_the_mean_dose_and_kinds_have_their_sign():
    P, W, cons = _case(("max", "mean", "min"), 30)
    G, h = constraint_rows(W, cons)
    x = np.random.default_rng(0).uniform(0.0, 3.0, size=W.n)
    for s in range(W.N):
        dose = W.dose(s, x)
        gx = G[s] @ x
        np.testing.assert_allclose(gx[:2], dose[[0, 1]], rtol=1e-14)          # max rows: dose itself
        assert gx[2] == pytest.approx(dose[2:7].mean(), rel=1e-14)           # mean row
        np.testing.assert_allclose(gx[3:5], -dose[[8, 9]], rtol=1e-14)       # min rows: negated dose
        np.testing.assert_allclose(h[s], [cons[0].limit] * 2 + [cons[1].limit] + [-cons[2].limit] * 2)


@pytest.mark.parametrize("kinds,seed", CASES)
def test_bruteforce_matches_library_slsqp_and_constraints_bind(kinds, seed):
    P, W, cons = _case(kinds, seed)
    G, h = constraint_rows(W, cons)
    Ga, ha = sp.vstack(G).toarray(), np.concatenate(h)
    xb, lam = kkt_bruteforce_lin(W, Ga, ha)
    res = _slsqp(W, Ga, ha)
    xs = res.x
    np.testing.assert_allclose(xb, xs, rtol=1e-6, atol=1e-7)
    if getattr(res, "multipliers", None) is not None:         # the library's multipliers, where it reports them
        np.testing.assert_allclose(lam, np.asarray(res.multipliers)[:len(lam)], rtol=1e-5, atol=1e-6)
    assert W.f(xb) <= W.f(xs) * (1 + 1e-10)
    assert np.all(Ga @ xb <= ha + 1e-9 * (1 + np.abs(ha)))
    assert lam.max() > 1e-6                                   # at least one limit binds
    assert W.f(xb) > W.f(kkt_bruteforce(W)) * (1 + 1e-9)      # and costs objective


@pytest.mark.parametrize("kinds,seed", CASES)
def test_constrained_admm_reaches_the_exact_optimum_and_multipliers(kinds, seed):
    P, W, cons = _case(kinds, seed)
    G, h = constraint_rows(W, cons)
    Ga, ha = sp.vstack(G).toarray(), np.concatenate(h)
    xb, lam = kkt_bruteforce_lin(W, Ga, ha)
    r = admm_bb_constrained(W, cons, eps_abs=1e-11, eps_rel=1e-11, max_iter=200000)
    assert r["status"] == "converged", r["iterations"]
    z = r["z"]
    assert (W.f(z) - W.f(xb)) / W.f(xb) == pytest.approx(0.0, abs=1e-8)
    np.testing.assert_allclose(z, xb, rtol=1e-6, atol=1e-6 * np.abs(xb).max())
    assert np.all(Ga @ z <= ha + 1e-6 * (1 + np.abs(ha)))
    mu = np.concatenate(r["mu"])
    np.testing.assert_allclose(mu, lam, rtol=1e-4, atol=1e-6 * max(1.0, lam.max()))
    # projected stationarity with the multipliers: z = P(z - (grad f + G' mu)/L)
    L = lipschitz(W)
    gl = W.grad(z) + Ga.T @ mu
    np.testing.assert_allclose(z, W.proj(z - gl / L), atol=1e-7 * max(1.0, np.abs(z).max()))


def test_no_constraint_rows_is_admm_bb_step_for_step():
    P = _tiny_dense(34, m=13, n=5, N=3, lb=0.0, ub=1.2, sw=True)
    W = Weighted(P)
    for k in (1, 2, 5, 20):
        a = admm_bb(W, rho=0.9, max_iter=k, eps_abs=0.0, eps_rel=0.0, subproblem="chol")
        b = admm_bb_constrained(W, [], rho=0.9, max_iter=k, eps_abs=0.0, eps_rel=0.0)
        np.testing.assert_allclose(b["z"], a["z"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(b["x"], a["x"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(b["y"], a["y"], rtol=1e-12, atol=1e-14)
        assert b["r_prim"] == pytest.approx(a["r_prim"], rel=1e-12)
        assert b["r_dual"] == pytest.approx(a["r_dual"], rel=1e-12)


def test_inactive_limits_leave_the_optimum_unchanged():
    P, W, cons = _case(("max", "mean"), 35)
    loose = [DoseConstraint(c.kind, c.voxels, 1e3) for c in cons]
    r = admm_bb_constrained(W, loose, eps_abs=1e-11, eps_rel=1e-11, max_iter=200000)
    x0 = kkt_bruteforce(W)
    assert r["status"] == "converged"
    np.testing.assert_allclose(r["z"], x0, rtol=1e-6, atol=1e-7)
    assert np.abs(np.concatenate(r["mu"])).max() <= 1e-9


def test_hand_worked_constrained_iterates():
    """One spot, one voxel, dose limit below the unconstrained optimum: the
    iterates of the dose block (x, v, mu) and both residuals, worked by hand."""
    g = json.load(open(os.path.join(GOLD, "hand_admm_dose_1x1.json")))
    pr = g["problem"]
    W = Weighted(from_dense(pr["A"], pr["w"], pr["p"], pr["lb"], pr["ub"]))
    cons = [DoseConstraint(c["kind"], np.array(c["voxels"]), c["limit"]) for c in pr["constraints"]]
    prm = g["params"]
    for k, it in enumerate(g["iterates"], start=1):
        r = admm_bb_constrained(W, cons, rho=prm["rho"], sigma=prm["sigma"], max_iter=k,
                                eps_abs=0.0, eps_rel=0.0)
        assert r["x"][0][0] == pytest.approx(it["x"], rel=1e-14)
        assert r["z"][0] == pytest.approx(it["z"], rel=1e-14)
        assert r["v"][0][0] == pytest.approx(it["v"], rel=1e-14)
        assert r["mu"][0][0] == pytest.approx(it["mu"], rel=1e-14, abs=1e-15)
        assert r["r_prim"] == pytest.approx(it["r_prim"], rel=1e-13, abs=1e-15)
        assert r["r_dual"] == pytest.approx(it["r_dual"], rel=1e-13)
    r = admm_bb_constrained(W, cons, rho=prm["rho"], sigma=prm["sigma"], max_iter=10000,
                            eps_abs=1e-13, eps_rel=1e-13)
    assert r["status"] == "converged"
    assert r["z"][0] == pytest.approx(g["optimum"]["x"], rel=1e-10)
    assert r["f"] == pytest.approx(g["optimum"]["f"], rel=1e-10)
    assert r["mu"][0][0] == pytest.approx(g["optimum"]["mu"], rel=1e-8)
