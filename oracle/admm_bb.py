"""ADMM with Barzilai-Borwein dual step, float64 (oracle; test use only).

Sec. 2.2.  Consensus form (Eq. 5): minimise sum_s f_s(x_s) s.t. x_s = z,
z in the box.  Each iteration k:
  1. x_s^{k+1} = argmin f_s(x) + (rho/2)||x - z^k + y_s^k/rho||^2      (Eq. 6)
     = solution of B_s x = c_s^k,  B_s = A~_s^T A~_s + (rho/2) I,
       c_s^k = A~_s^T p~ + (rho/2)(z^k - y_s^k/rho)                  (App. A)
  2. z^{k+1} = P_box(mean_s(x_s^{k+1} + y_s^k/rho))   [zmode "std"]
     or       P_box(mean_s x_s^{k+1})                 [zmode "lit", as printed]
  3. y_s^{k+1} = y_s^k + step_k (x_s^{k+1} - z^{k+1})                   (Eq. 7)
     step_k = BB value beta^k = -dd'dy/||dd||^2 if it is > 0, else rho   (Eq. 8)
     dd = d^{k+1} - d^k with d = x - 1(x)z, dy = y^k - y^{k-1}
     (bb_per_scenario: the same rule applied to each scenario's own blocks
     dd_s, dy_s, giving one step beta_s^k per scenario)
  4. stop when ||r_prim|| <= eps_prim and ||r_dual|| <= eps_dual          (Eq. 9)
     r_prim = x^{k+1} - 1(x)z^{k+1},  r_dual = 1(x) rho (z^{k+1} - z^k),
     eps_prim = eps_abs sqrt(Nn) + eps_rel max(||x||, sqrt(N)||z||),
     eps_dual = eps_abs sqrt(Nn) + eps_rel ||y||.
Optionally combined (AND) with a relative objective-change test (Sec. 2.3).

Readings (the paper is silent): z^0 = P(z0) (default 0), y^0 = y0 (default 0),
x_s^0 = z^0; the BB step needs y^{k-1}, so the first iteration uses rho; the
step must be finite and > 0, else rho; bb="guarded" clamps it to
[rho/kappa, kappa*rho]; bb="off" always uses rho.  Eq. 8 is written over the
concatenated vectors, so one global step is the default; per-scenario steps
are an option (a reading, not the paper's rule).  The returned "step" is the
global step, or the mean of the per-scenario steps ("steps" holds them all).

The subproblem is solved either with a Cholesky factor of B_s computed once
(App. A, the paper's method) or by conjugate gradients warm-started from
x_s^k (a reading: the paper only uses the factor), optionally with the
Jacobi preconditioner M = diag(B_s).  CG on scenario s stops
when ||c_s - B_s x|| <= tol_s with
    k = 0:  tol_s = eta0 ||r0_s||,  r0_s = c_s - B_s x_s^0 (the first residual)
    k >= 1: tol_s = max(theta (rho/2) max(r_prim^k, eps_prim^k) / sqrt(N),
                        min(floor_rel ||r0_s||, (rho/2) eps_prim^k / sqrt(N)))
Since ||x_err|| <= 2 ||residual|| / rho, the subproblem error stays a
fraction theta of the primal residual.  The floor saves steps on a
subproblem that is already accurate, but it is capped at the accuracy that
Eq. 9 needs: summed over the scenarios, a subproblem error of up to eps_prim.
An uncapped floor (floor_rel ||r0_s|| above that) leaves the x-updates less
accurate than the stopping rule asks, and the iteration stalls above eps.
"""
from __future__ import annotations

import math
import time

import numpy as np
import scipy.linalg as sla

from .problem import Weighted


def _cg(W, s, rho, c, x, tol_fn, kmax, minv=None):
    """Preconditioned conjugate gradients (Hestenes-Stiefel) on B_s x = c from the
    warm start x, with M^{-1} = diag(minv) (None: no preconditioner); stopped when
    the residual norm ||c - B_s x|| <= tol_fn(||initial residual||)."""
    r = c - W.normal_apply(s, x, rho)
    tol = tol_fn(float(np.linalg.norm(r)))
    if float(np.linalg.norm(r)) <= tol:
        return x, 0
    z = r if minv is None else minv * r
    gam = float(r @ z)
    p = z.copy()
    it = 0
    for it in range(1, kmax + 1):
        u = W.normal_apply(s, p, rho)
        alpha = gam / float(p @ u)
        x = x + alpha * p
        r = r - alpha * u
        if float(np.linalg.norm(r)) <= tol:
            break
        z = r if minv is None else minv * r
        gnew = float(r @ z)
        p = z + (gnew / gam) * p
        gam = gnew
    return x, it


def admm_bb(prob_or_w, rho=None, eps_abs=1e-4, eps_rel=1e-4, max_iter=1000,
            subproblem="chol", bb="paper", zmode="std", bb_kappa=10.0,
            z0=None, y0=None, tol_obj=math.inf, cg_theta=0.15, cg_eta0=1e-2,
            cg_floor_rel=0.0, cg_max=200, cg_precond="jacobi", record=False, record_f=False,
            bb_per_scenario=False, xupdate=None):
    """xupdate: optional callable (z, y) -> x [N, n] that performs step 1 with
    the cached factors held elsewhere (oracle.parallel: the scenario subproblems
    on worker processes, as the paper ran them); only with subproblem="chol"."""
    if xupdate is not None and subproblem != "chol":
        raise ValueError("xupdate replaces the cached-factor x-update only")
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    N, n = W.N, W.n
    if rho is None:
        from .problem import default_rho
        rho = default_rho(W)
    t0 = time.perf_counter()
    b = [W.b(s) for s in range(N)]
    if subproblem == "chol" and xupdate is None:
        fac = [sla.cho_factor(W.B_dense(s, rho), lower=False) for s in range(N)]
    minv = [None] * N
    if subproblem == "cg" and cg_precond == "jacobi":
        # Jacobi preconditioner: diag(B_s) = diag(A~_s^T A~_s) + rho/2
        minv = [1.0 / (np.asarray(W.At[s].multiply(W.At[s]).sum(axis=0)).ravel() + 0.5 * rho)
                for s in range(N)]
    z = W.proj(np.zeros(n) if z0 is None else np.asarray(z0, float).copy())
    y = np.zeros((N, n)) if y0 is None else np.asarray(y0, float).reshape(N, n).copy()
    x = np.tile(z, (N, 1))
    d_prev = x - z[None, :]
    y_prev = None
    rp_prev, ep_prev = None, None
    r0 = np.zeros(N)
    f_prev = W.f(z) if math.isfinite(tol_obj) else None
    hist = []
    status = "not_converged"
    cg_total = 0
    it = 0
    step = rho
    steps = np.full(N, rho)
    for k in range(max_iter):
        # 1. scenario subproblems
        xn = np.empty_like(x)
        if xupdate is not None:
            xn[:] = xupdate(z, y)
        for s in range(N if xupdate is None else 0):
            c = b[s] + 0.5 * rho * (z - y[s] / rho)
            if subproblem == "chol":
                xn[s] = sla.cho_solve(fac[s], c)
            else:
                if rp_prev is None:
                    def tol_fn(r0n, s=s):
                        r0[s] = r0n
                        return cg_eta0 * r0n
                else:
                    def tol_fn(r0n, s=s):
                        return max(cg_theta * 0.5 * rho * max(rp_prev, ep_prev) / math.sqrt(N),
                                   min(cg_floor_rel * r0[s], 0.5 * rho * ep_prev / math.sqrt(N)))
                xn[s], kk = _cg(W, s, rho, c, x[s].copy(), tol_fn, cg_max, minv[s])
                cg_total += kk
        # 2. consensus projection
        if zmode == "std":
            zn = W.proj(np.mean(xn + y / rho, axis=0))
        elif zmode == "lit":
            zn = W.proj(np.mean(xn, axis=0))
        else:
            raise ValueError(zmode)
        # 3. BB step and dual update
        d = xn - zn[None, :]

        def bb_step(dd, dy):
            st = rho
            if bb != "off" and y_prev is not None:
                den = float(dd @ dd)
                if den > 0.0:
                    beta = -float(dd @ dy) / den
                    if math.isfinite(beta) and beta > 0.0:
                        st = beta
                        if bb == "guarded":
                            st = min(max(st, rho / bb_kappa), bb_kappa * rho)
            return st

        if bb_per_scenario:
            steps = np.array([bb_step(d[s] - d_prev[s], None if y_prev is None else y[s] - y_prev[s])
                              for s in range(N)])
            step = float(np.mean(steps))
            yn = y + steps[:, None] * d
        else:
            step = bb_step((d - d_prev).ravel(), None if y_prev is None else (y - y_prev).ravel())
            steps = np.full(N, step)
            yn = y + step * d
        # 4. residuals and stopping rule
        r_prim = float(np.linalg.norm(d))
        r_dual = math.sqrt(N) * rho * float(np.linalg.norm(zn - z))
        xnorm = float(np.linalg.norm(xn))
        eps_prim = eps_abs * math.sqrt(N * n) + eps_rel * max(xnorm, math.sqrt(N) * float(np.linalg.norm(zn)))
        eps_dual = eps_abs * math.sqrt(N * n) + eps_rel * float(np.linalg.norm(yn))
        ok = r_prim <= eps_prim and r_dual <= eps_dual
        if math.isfinite(tol_obj):
            fz = W.f(zn)
            ok = ok and abs(f_prev - fz) <= tol_obj * max(abs(fz), 1e-300)
            f_prev = fz
        if record:
            hist.append(dict(k=k + 1, t=time.perf_counter() - t0, r_prim=r_prim, r_dual=r_dual,
                             eps_prim=eps_prim, eps_dual=eps_dual, step=step, cg=cg_total,
                             f=W.f(zn) if record_f else None))
        y_prev, y = y, yn
        x, z, d_prev = xn, zn, d
        rp_prev, ep_prev = r_prim, eps_prim
        it = k + 1
        if not (math.isfinite(r_prim) and math.isfinite(r_dual)):
            status = "diverged"
            break
        if ok:
            status = "converged"
            break
    return dict(z=z, x=x, y=y, iterations=it, status=status, rho=rho, step=step, steps=steps,
                r_prim=r_prim, r_dual=r_dual, eps_prim=eps_prim, eps_dual=eps_dual,
                cg_iterations=cg_total, f=W.f(z), history=hist,
                seconds=time.perf_counter() - t0)
