"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each test fixes the oracle to a closed form, a library routine, a brute-force
enumeration, a hand-worked example or an invariant of the paper's method, so
that a dropped term, a wrong sign or a shifted index in the oracle fails here.
"""
import json
import math
import os

import numpy as np
import pytest

from synthetic import from_dense, random_problem, config_tiny_plain
from oracle import (Weighted, admm_bb, pgd, kkt_bruteforce, lsq_box, certificates,
                    consensus_admm_scaled, default_rho, lipschitz)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_dense(seed, m=12, n=4, N=3, lb=0.0, ub=10.0, sw=False):
    rng = np.random.default_rng(seed)
    A = [rng.uniform(0.0, 1.0, size=(m, n)) * (rng.random((m, n)) < 0.7) for _ in range(N)]
    for Ai in A:                       # full column rank: a diagonal block
        Ai[:n, :n] += np.eye(n)
    w = rng.uniform(0.5, 3.0, size=m)
    p = np.where(rng.random(m) < 0.5, 5.0, 0.0)
    c = rng.uniform(0.3, 1.0, size=N) if sw else None
    return from_dense(A, w, p, lb, ub, scen_weight=c)


# ---------------------------------------------------------------------------
# Eq. 1, 2, 4 written as explicit sums (brute force) vs the oracle's sparse form
# ---------------------------------------------------------------------------

def test_objective_gradient_normal_op_bruteforce():
    P = random_problem(3, m=9, n=5, N=2, mean_row=3.0, scen_weight=True)
    W = Weighted(P)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 3, size=P.n)
    v = rng.normal(size=P.n)
    f_bf, g_bf = 0.0, np.zeros(P.n)
    for s in range(P.N):
        cs = P.scen_weight[s]
        A = P.csr(s).toarray()
        u_bf = np.zeros(P.n)
        for i in range(P.m):
            dot = sum(A[i, j] * x[j] for j in range(P.n))
            f_bf += cs * P.voxel_w[i] * (dot - P.presc[i]) ** 2              # Eq. 1
            for j in range(P.n):
                g_bf[j] += 2.0 * cs * P.voxel_w[i] * A[i, j] * (dot - P.presc[i])   # Eq. 4
            av = sum(A[i, j] * v[j] for j in range(P.n))
            for j in range(P.n):
                u_bf[j] += cs * P.voxel_w[i] * A[i, j] * av
        rho = 1.7
        np.testing.assert_allclose(W.normal_apply(s, v, rho), u_bf + 0.5 * rho * v, rtol=1e-12, atol=1e-12)
    assert W.f(x) == pytest.approx(f_bf, rel=1e-13)
    np.testing.assert_allclose(W.grad(x), g_bf, rtol=1e-12, atol=1e-10)


def test_default_rho_and_lipschitz_against_dense_linear_algebra():
    P = _tiny_dense(1, m=10, n=6, N=3)
    W = Weighted(P)
    H = W.hessian_dense()
    G = [(W.At[s].T @ W.At[s]).toarray() for s in range(P.N)]
    assert default_rho(W) == pytest.approx(2.0 * np.mean([np.trace(g) for g in G]) / P.n, rel=1e-13)
    lam = np.linalg.eigvalsh(H).max()          # library eigensolver
    assert lipschitz(W, iters=200) == pytest.approx(lam, rel=1e-8)


# ---------------------------------------------------------------------------
# exact optimum: closed forms, library routines, enumeration
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lb,ub,where", [(0.0, 10.0, "free"), (2.0, 10.0, "lb"), (0.0, 0.5, "ub")])
def test_scalar_closed_form(lb, ub, where):
    """n = 1: x* = clamp(sum c_s w_i a_i p_i / sum c_s w_i a_i^2, lb, ub)."""
    rng = np.random.default_rng(7)
    m, N = 6, 3
    A = [rng.uniform(0.1, 1.0, size=(m, 1)) for _ in range(N)]
    w = rng.uniform(0.5, 2.0, size=m)
    p = rng.uniform(0.0, 2.0, size=m)
    c = rng.uniform(0.3, 1.0, size=N)
    num = sum(c[s] * np.sum(w * A[s][:, 0] * p) for s in range(N))
    den = sum(c[s] * np.sum(w * A[s][:, 0] ** 2) for s in range(N))
    xs = min(max(num / den, lb), ub)
    P = from_dense(A, w, p, lb, ub, scen_weight=c)
    # float32 storage of A: rebuild the closed form from the stored values
    Af = [P.csr(s).toarray() for s in range(N)]
    num = sum(c[s] * np.sum(w * Af[s][:, 0] * p) for s in range(N))
    den = sum(c[s] * np.sum(w * Af[s][:, 0] ** 2) for s in range(N))
    xs = min(max(num / den, lb), ub)
    if where == "free":
        assert lb < xs < ub
    W = Weighted(P)
    assert kkt_bruteforce(W)[0] == pytest.approx(xs, rel=1e-12)
    assert lsq_box(W)[0] == pytest.approx(xs, rel=1e-9, abs=1e-12)
    r = admm_bb(W, eps_abs=1e-12, eps_rel=1e-12, max_iter=5000)
    assert r["z"][0] == pytest.approx(xs, rel=1e-8, abs=1e-10)
    r = admm_bb(W, eps_abs=1e-12, eps_rel=1e-12, max_iter=5000, subproblem="cg")
    assert r["z"][0] == pytest.approx(xs, rel=1e-8, abs=1e-10)
    r = pgd(W, tol_rel_df=1e-15, max_iter=5000)
    assert r["x"][0] == pytest.approx(xs, rel=1e-7, abs=1e-9)


def test_unconstrained_matches_lstsq():
    """No active bound: x* solves the stacked least squares (numpy.linalg.lstsq)."""
    P = _tiny_dense(2, m=15, n=5, N=4, lb=-np.inf, ub=np.inf, sw=True)
    W = Weighted(P)
    A, b = W.stacked()
    x_ls = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]
    r = admm_bb(W, eps_abs=1e-13, eps_rel=1e-13, max_iter=20000)
    np.testing.assert_allclose(r["z"], x_ls, rtol=1e-8, atol=1e-9)
    r = pgd(W, tol_rel_df=1e-16, max_iter=100000)
    np.testing.assert_allclose(r["x"], x_ls, rtol=1e-5, atol=1e-6)
    # paper-literal z-update coincides with the standard one when no bound is active
    rl = admm_bb(W, eps_abs=1e-13, eps_rel=1e-13, max_iter=20000, zmode="lit")
    np.testing.assert_allclose(rl["z"], x_ls, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bruteforce_kkt_vs_library_bvls_vs_admm_vs_pgd(seed):
    P = _tiny_dense(10 + seed, m=14, n=6, N=3, lb=0.0, ub=1.5, sw=(seed % 2 == 1))
    W = Weighted(P)
    xb = kkt_bruteforce(W)
    xl = lsq_box(W)
    np.testing.assert_allclose(xl, xb, atol=1e-9)
    c = certificates(W, xb)
    assert c["pg"] < 1e-12 and c["kkt"] < 1e-11 and c["infeas"] == 0.0
    fstar = W.f(xb)
    for sub in ("chol", "cg"):
        r = admm_bb(W, eps_abs=1e-11, eps_rel=1e-11, max_iter=20000, subproblem=sub)
        assert r["status"] == "converged"
        assert abs(r["f"] - fstar) <= 1e-9 * fstar
        np.testing.assert_allclose(r["z"], xb, atol=1e-6)
    r = pgd(W, tol_rel_df=1e-15, max_iter=200000)
    assert abs(r["f"] - fstar) <= 1e-8 * fstar


def test_tiny_plain_config_admm_matches_library_optimum():
    P = config_tiny_plain(0).subset_scenarios([0, 1, 7])
    W = Weighted(P)
    xs = lsq_box(W)
    fstar = W.f(xs)
    c = certificates(W, xs)
    assert c["pg"] < 1e-9
    r = admm_bb(W, rho=0.3 * default_rho(W), eps_abs=1e-7, eps_rel=1e-7, max_iter=5000)
    assert r["status"] == "converged"
    assert (r["f"] - fstar) / fstar < 1e-8
    assert certificates(W, r["z"])["pg"] < 1e-5


# ---------------------------------------------------------------------------
# the x-subproblem (App. A): normal equations vs the stacked least squares
# ---------------------------------------------------------------------------

def test_subproblem_normal_equations_vs_stacked_lstsq():
    P = _tiny_dense(4, m=11, n=5, N=2, sw=True)
    W = Weighted(P)
    rho = 0.7
    rng = np.random.default_rng(1)
    z = rng.uniform(0, 2, size=P.n)
    y = rng.normal(size=(P.N, P.n))
    r = admm_bb(W, rho=rho, z0=z, y0=y, max_iter=1, bb="off")
    for s in range(P.N):
        At = W.At[s].toarray()
        Astk = np.vstack([At, math.sqrt(rho / 2.0) * np.eye(P.n)])
        bstk = np.concatenate([W.pt[s], math.sqrt(rho / 2.0) * (z - y[s] / rho)])
        xs = np.linalg.lstsq(Astk, bstk, rcond=None)[0]
        np.testing.assert_allclose(r["x"][s], xs, rtol=1e-11, atol=1e-12)
        # and it minimises f_s(x) + rho/2 ||x - z + y/rho||^2 (Eq. 6): gradient zero
        g = W.grad_s(s, xs) + rho * (xs - z + y[s] / rho)
        assert np.abs(g).max() < 1e-9


# ---------------------------------------------------------------------------
# the iteration (Sec. 2.2): hand-worked example and textbook ADMM
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precond", [False, True])
def test_cg_subproblem_solver_matches_dense_solve_within_n_steps(precond):
    """The oracle's (preconditioned) conjugate gradients on B_s x = c: in exact
    arithmetic CG ends within n steps, so with n = 6 and 8 steps allowed it
    must reach the dense solve to rounding, from any warm start."""
    from oracle.admm_bb import _cg
    P = _tiny_dense(12, m=14, n=6, N=2, sw=True)
    W = Weighted(P)
    rho = 0.8
    rng = np.random.default_rng(3)
    for s in range(P.N):
        B = W.B_dense(s, rho)
        c = rng.normal(size=P.n)
        x0 = rng.normal(size=P.n)
        minv = 1.0 / np.diag(B) if precond else None
        x, its = _cg(W, s, rho, c, x0.copy(), lambda r0: 1e-13 * r0, 8, minv)
        np.testing.assert_allclose(x, np.linalg.solve(B, c), rtol=1e-10, atol=1e-12)
        assert 1 <= its <= 8
        # the warm start counts: starting at the solution needs no step
        x2, its2 = _cg(W, s, rho, c, np.linalg.solve(B, c), lambda r0: max(1e-13 * r0, 1e-12), 8, minv)
        assert its2 == 0


def test_hand_worked_iterates():
    g = json.load(open(os.path.join(GOLD, "hand_admm_bb_2x1.json")))
    pr = g["problem"]
    P = from_dense(pr["A"], pr["w"], pr["p"], pr["lb"], pr["ub"])
    W = Weighted(P)
    rho = g["params"]["rho"]
    for k, it in enumerate(g["iterates"], start=1):
        r = admm_bb(W, rho=rho, max_iter=k, eps_abs=0.0, eps_rel=0.0)
        np.testing.assert_allclose(r["x"], it["x"], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(r["z"], it["z"], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(r["y"], it["y"], rtol=1e-13, atol=1e-13)
        assert r["step"] == pytest.approx(it["step"], rel=1e-12)
        if "r_prim" in it:
            assert r["r_prim"] == pytest.approx(it["r_prim"], rel=1e-14)
            assert r["r_dual"] == pytest.approx(it["r_dual"], rel=1e-14)
    r = admm_bb(W, rho=rho, eps_abs=1e-14, eps_rel=1e-14, max_iter=10000)
    assert r["z"][0] == pytest.approx(g["optimum"]["x"][0], rel=1e-10)
    assert r["f"] == pytest.approx(g["optimum"]["f"], rel=1e-10)


def test_hand_worked_per_scenario_bb_iterates():
    """Eq. 8 applied per scenario on a 2-scenario example whose bound binds, so
    that the two scenarios' steps differ (4 and 10 at k = 2)."""
    g = json.load(open(os.path.join(GOLD, "hand_admm_bb_scen_2x1.json")))
    pr = g["problem"]
    W = Weighted(from_dense(pr["A"], pr["w"], pr["p"], pr["lb"], pr["ub"]))
    rho = g["params"]["rho"]
    for k, it in enumerate(g["iterates"], start=1):
        r = admm_bb(W, rho=rho, max_iter=k, eps_abs=0.0, eps_rel=0.0, bb_per_scenario=True)
        np.testing.assert_allclose(r["x"], it["x"], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(r["z"], it["z"], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(r["y"], it["y"], rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(r["steps"], it["steps"], rtol=1e-12)
        assert r["step"] == pytest.approx(float(np.mean(it["steps"])), rel=1e-12)
        if "r_prim" in it:
            assert r["r_prim"] == pytest.approx(it["r_prim"], rel=1e-14, abs=1e-15)
            assert r["r_dual"] == pytest.approx(it["r_dual"], rel=1e-14, abs=1e-15)
    r = admm_bb(W, rho=rho, max_iter=100, eps_abs=1e-12, eps_rel=1e-12, bb_per_scenario=True)
    assert r["status"] == "converged" and r["iterations"] == 4
    assert r["f"] == pytest.approx(g["optimum"]["f"], rel=1e-14)
    # the global rule differs at k = 2 on the same example
    rg = admm_bb(W, rho=rho, max_iter=3, eps_abs=0.0, eps_rel=0.0)
    assert rg["step"] == pytest.approx(0.29624 / 0.067124, rel=1e-12)


@pytest.mark.parametrize("N,bb", [(1, "paper"), (1, "guarded"), (3, "off")])
def test_per_scenario_bb_reduces_to_global(N, bb):
    """With one scenario, or with the BB step off, the per-scenario rule is the global one."""
    P = _tiny_dense(8, m=15, n=5, N=N, lb=0.0, ub=1.0, sw=True)
    W = Weighted(P)
    for k in (1, 2, 5, 20):
        a = admm_bb(W, rho=1.1, max_iter=k, eps_abs=0.0, eps_rel=0.0, bb=bb)
        b = admm_bb(W, rho=1.1, max_iter=k, eps_abs=0.0, eps_rel=0.0, bb=bb, bb_per_scenario=True)
        np.testing.assert_allclose(b["y"], a["y"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(b["z"], a["z"], rtol=1e-12, atol=1e-14)


def test_per_scenario_bb_reaches_the_optimum():
    P = _tiny_dense(9, m=16, n=6, N=4, lb=0.0, ub=0.8, sw=True)
    W = Weighted(P)
    xs = kkt_bruteforce(W)
    r = admm_bb(W, eps_abs=1e-12, eps_rel=1e-12, max_iter=20000, bb_per_scenario=True)
    assert r["status"] == "converged"
    assert r["f"] == pytest.approx(W.f(xs), rel=1e-10)
    assert len(set(np.round(r["steps"], 12))) > 1          # the steps did differ


def test_bb_off_equals_textbook_scaled_consensus_admm():
    P = _tiny_dense(5, m=13, n=5, N=3, lb=0.0, ub=1.2, sw=True)
    W = Weighted(P)
    rho = 0.9
    ref = consensus_admm_scaled(W, rho, iters=25)
    for k in (1, 2, 7, 25):
        r = admm_bb(W, rho=rho, max_iter=k, bb="off", eps_abs=0.0, eps_rel=0.0)
        np.testing.assert_allclose(r["z"], ref["z_hist"][k - 1], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r["y"], ref["y"], rtol=1e-9, atol=1e-10)


def test_fixed_point_dual_is_negative_scenario_gradient():
    """At the Z-STD fixed point y_s = -grad f_s(z*) and z* = P(z* - grad f(z*)/(N rho))."""
    P = _tiny_dense(6, m=14, n=5, N=3, lb=0.0, ub=1.0)
    W = Weighted(P)
    rho = 1.3
    r = admm_bb(W, rho=rho, eps_abs=1e-13, eps_rel=1e-13, max_iter=50000, bb="off")
    z = r["z"]
    for s in range(P.N):
        np.testing.assert_allclose(r["y"][s], -W.grad_s(s, z), rtol=1e-7, atol=1e-7)
    np.testing.assert_allclose(z, W.proj(z - W.grad(z) / (P.N * rho)), atol=1e-9)


def test_z_stays_in_box_and_literal_zupdate_can_stall():
    P = config_tiny_plain(0).subset_scenarios([0, 3, 8])
    W = Weighted(P)
    xs = lsq_box(W)
    fstar = W.f(xs)
    rho = 0.3 * default_rho(W)
    r = admm_bb(W, rho=rho, eps_abs=1e-7, eps_rel=1e-7, max_iter=2000, record=False)
    assert np.all(r["z"] >= W.lb) and np.all(r["z"] <= W.ub)
    rl = admm_bb(W, rho=rho, eps_abs=1e-7, eps_rel=1e-7, max_iter=2000, zmode="lit")
    assert np.all(rl["z"] >= W.lb) and np.all(rl["z"] <= W.ub)
    # with bounds active, the printed update's limit is not the optimum (reported)
    gap_lit = (rl["f"] - fstar) / fstar
    gap_std = (r["f"] - fstar) / fstar
    assert gap_std < 1e-7
    assert gap_lit > 100 * max(gap_std, 1e-12)


# ---------------------------------------------------------------------------
# PGD (Sec. 2.1, Eq. 3 read as sufficient decrease)
# ---------------------------------------------------------------------------

def test_pgd_monotone_and_armijo_holds():
    P = _tiny_dense(8, m=20, n=7, N=3, lb=0.0, ub=1.0)
    W = Weighted(P)
    r = pgd(W, tol_rel_df=1e-12, max_iter=400, record=True)
    fs = [h["f"] for h in r["history"]]
    assert all(b <= a for a, b in zip(fs, fs[1:]))
    # one step by hand: the accepted point satisfies sufficient decrease
    x0 = W.proj(np.zeros(P.n))
    g = W.grad(x0)
    r1 = pgd(W, max_iter=1, tol_rel_df=0.0)
    assert W.f(r1["x"]) <= W.f(x0) + 1e-4 * float(g @ (r1["x"] - x0)) + 1e-12
    # a step of 1/L from x0 is always accepted (descent lemma), so the first
    # accepted step is >= gamma^j * alpha >= 1/(2L) with alpha = 4/L
    L = lipschitz(W)
    t = r1["history"][0]["step"] if r1["history"] else None
    r1 = pgd(W, max_iter=1, tol_rel_df=0.0, record=True)
    assert r1["history"][0]["step"] >= 0.5 / L


@pytest.mark.parametrize("seed,ub", [(41, 3.0), (42, 3.0), (60, 20.0), (61, 100.0)])
def test_projected_newton_matches_bruteforce_and_library_bvls(seed, ub):
    """box_qp_newton (used for the full-size optimum) against KKT enumeration
    (n = 8) and against the library's BVLS on a case with free variables and
    both kinds of active bounds."""
    from oracle import box_qp_newton
    small = random_problem(seed, m=300, n=8, N=2, mean_row=4.0, ub=ub)
    Ws = Weighted(small)
    a, b = kkt_bruteforce(Ws), box_qp_newton(Ws)
    assert abs(Ws.f(a) - Ws.f(b)) <= 1e-12 * Ws.f(a) and np.abs(a - b).max() <= 1e-9
    prob = random_problem(seed, m=2000, n=120, N=3, mean_row=10.0, ub=ub)
    W = Weighted(prob)
    a, b = lsq_box(W), box_qp_newton(W)
    assert abs(W.f(a) - W.f(b)) <= 1e-12 * W.f(a) and np.abs(a - b).max() <= 1e-8
    assert certificates(W, b)["pg"] <= 1e-12
