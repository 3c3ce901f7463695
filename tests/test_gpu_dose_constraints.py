"""Linear dose constraints on the GPU (rpt_admm_bb_solve_constrained; paper
Sec. 4) against the float64 oracle (oracle.dose_constraints): the hand-worked
iterates, the oracle's iterates step by step, the exact constrained optimum by
active-set enumeration with its multipliers, and a limit on an organ at risk of
the tiny phantom.

Tolerances.  The GPU's x-update is the float32 cached inverse of
B_s + (sigma/2) G_s'G_s (relative error about n cond(B_s) eps32 per solve, as for
the plain cached-factor solver); the constraint rows and the dose-block updates
are float64.  That error sets a floor under the residuals of Eq. 9: at
eps = 1e-8 the primal residual of these cases stalls above eps_prim (the oracle
with its Cholesky solves replaced by a float32 inverse stalls the same way), and
1e-7 is the tightest decade reached; there the float32-inverse iteration ends
within 3e-7 of the optimum's objective and 4e-7 of each limit."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import Weighted, kkt_bruteforce, default_rho
from oracle.dose_constraints import DoseConstraint, constraint_rows, admm_bb_constrained, kkt_bruteforce_lin
from synthetic import from_dense, config_tiny_plain

from tests.gpu_util import gpu_lib, plan_of
from tests.test_oracle_pins import _tiny_dense

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
KIND = {"max": 0, "min": 1, "mean": 2}


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def _lib_cons(cons):
    return [(KIND[c.kind], np.asarray(c.voxels), c.limit) for c in cons]


def _case(kind_set, seed):
    P = _tiny_dense(seed, m=12, n=4, N=2, lb=0.0, ub=6.0, sw=True)
    W = Weighted(P)
    x0 = kkt_bruteforce(W)
    dose = np.array([W.dose(s, x0) for s in range(W.N)])
    cons = []
    if "max" in kind_set:
        # with all three kinds one maximum voxel, so that the rows stay within the
        # enumeration's limit of 8 (max 2 + mean 2 + min 4 over the 2 scenarios)
        vox = np.array([0]) if len(kind_set) == 3 else np.array([0, 1])
        cons.append(DoseConstraint("max", vox, 0.8 * float(dose[:, vox].max())))
    if "mean" in kind_set:
        cons.append(DoseConstraint("mean", np.arange(2, 7), 0.9 * float(dose[:, 2:7].mean(axis=1).max())))
    if "min" in kind_set:
        cons.append(DoseConstraint("min", np.array([8, 9]), 1.15 * float(dose[:, [8, 9]].min())))
    return P, W, cons


CASES = [(("max", "mean"), 31), (("min",), 32), (("max", "min"), 33), (("max", "mean", "min"), 30)]


def test_hand_worked_constrained_iterates(rpt):
    g = json.load(open(os.path.join(GOLD, "hand_admm_dose_1x1.json")))
    pr = g["problem"]
    prob = from_dense(pr["A"], pr["w"], pr["p"], pr["lb"], pr["ub"])
    cons = [(KIND[c["kind"]], c["voxels"], c["limit"]) for c in pr["constraints"]]
    prm = g["params"]
    with plan_of(rpt, prob) as P:
        for k, it in enumerate(g["iterates"], start=1):
            x, mu, info = P.admm_bb_solve_constrained(cons, sigma=prm["sigma"], rho=prm["rho"], max_iter=k,
                                                      eps_abs=0.0, eps_rel=0.0)
            z, X, Y = P.state_get()
            assert info["iterations"] == k
            assert X[0] == pytest.approx(it["x"], rel=1e-6)
            assert z[0] == pytest.approx(it["z"], rel=1e-6)
            assert mu[0, 0] == pytest.approx(it["mu"], rel=1e-5, abs=1e-6)
            assert info["r_prim"] == pytest.approx(it["r_prim"], rel=1e-5, abs=1e-6)
            assert info["r_dual"] == pytest.approx(it["r_dual"], rel=1e-5)
        x, mu, info = P.admm_bb_solve_constrained(cons, sigma=prm["sigma"], rho=prm["rho"], max_iter=10000,
                                                  eps_abs=1e-8, eps_rel=1e-8)
    assert info["status"] == 0
    assert x[0] == pytest.approx(g["optimum"]["x"], rel=1e-6)
    assert mu[0, 0] == pytest.approx(g["optimum"]["mu"], rel=1e-5)


@pytest.mark.parametrize("path", [2, 4])
@pytest.mark.parametrize("kinds,seed", CASES)
def test_iterates_match_the_oracle(rpt, kinds, seed, path):
    """z, x_s, y_s and the dose duals mu_s after k iterations against the
    oracle's float64 iteration (Cholesky subproblems), CSR and bundled layouts."""
    P, W, cons = _case(kinds, seed)
    rho = default_rho(W)
    with plan_of(rpt, P, row_path=path) as Q:
        for k in (1, 2, 4, 10):
            ref = admm_bb_constrained(W, cons, rho=rho, max_iter=k, eps_abs=0.0, eps_rel=0.0)
            x, mu, info = Q.admm_bb_solve_constrained(_lib_cons(cons), rho=rho, max_iter=k, eps_abs=0.0,
                                                      eps_rel=0.0)
            z, X, Y = Q.state_get()
            sz = max(1.0, np.abs(ref["z"]).max())
            np.testing.assert_allclose(z, ref["z"], rtol=1e-4, atol=1e-5 * sz)
            np.testing.assert_allclose(X, ref["x"], rtol=1e-4, atol=1e-5 * sz)
            np.testing.assert_allclose(Y, ref["y"], rtol=1e-3, atol=1e-4 * max(1.0, np.abs(ref["y"]).max()))
            mref = np.stack(ref["mu"])
            np.testing.assert_allclose(mu, mref, rtol=1e-3, atol=1e-4 * max(1.0, np.abs(mref).max()))
            assert info["r_prim"] == pytest.approx(ref["r_prim"], rel=1e-3, abs=1e-5 * sz)
            assert info["r_dual"] == pytest.approx(ref["r_dual"], rel=1e-3, abs=1e-5 * rho * sz)


@pytest.mark.parametrize("kinds,seed", CASES)
def test_reaches_the_exact_constrained_optimum(rpt, kinds, seed):
    """The converged plan against active-set enumeration: objective to 1e-6,
    every limit met to 1e-6 of its size, duals equal to the KKT multipliers."""
    P, W, cons = _case(kinds, seed)
    G, h = constraint_rows(W, cons)
    Ga, ha = sp.vstack(G).toarray(), np.concatenate(h)
    xb, lam = kkt_bruteforce_lin(W, Ga, ha)
    with plan_of(rpt, P) as Q:
        z, mu, info = Q.admm_bb_solve_constrained(_lib_cons(cons), eps_abs=1e-7, eps_rel=1e-7, max_iter=100000)
    assert info["status"] == 0, info
    assert abs(W.f(z) - W.f(xb)) / W.f(xb) <= 1e-6
    assert np.all(Ga @ z <= ha + 1e-6 * (1 + np.abs(ha)))
    np.testing.assert_allclose(mu.ravel(), lam, rtol=1e-3, atol=1e-5 * max(1.0, lam.max()))


def test_organ_at_risk_limit_on_the_phantom(rpt):
    """A maximum-dose limit on the organ at risk of the tiny phantom (13
    scenarios, 200 spots): the robust plan keeps every scenario's OAR dose under
    the limit, costs objective against the unconstrained plan, and matches the
    oracle's constrained solve."""
    prob = config_tiny_plain(0)
    W = Weighted(prob)
    oar = np.flatnonzero(prob.labels == 2)
    with plan_of(rpt, prob) as P:
        z0, i0 = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, subproblem=rpt.SUB_CHOL)
        d0 = max(float(W.dose(s, z0)[oar].max()) for s in range(prob.N))
        limit = 0.7 * d0
        z, mu, info = P.admm_bb_solve_constrained([(rpt.DOSE_MAX, oar, limit)], eps_abs=1e-6, eps_rel=1e-6,
                                                  max_iter=50000)
    assert info["status"] == 0, info
    dmax = max(float(W.dose(s, z)[oar].max()) for s in range(prob.N))
    assert dmax <= limit * (1 + 1e-3), (dmax, limit)
    assert W.f(z) > W.f(z0)
    ref = admm_bb_constrained(W, [DoseConstraint("max", oar, limit)], eps_abs=1e-6, eps_rel=1e-6,
                              max_iter=50000)
    assert ref["status"] == "converged"
    assert abs(W.f(z) - ref["f"]) / ref["f"] <= 1e-5
    assert np.all(mu >= -1e-9 * np.abs(mu).max())
