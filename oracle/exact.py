"""Exact optimum of the box-constrained weighted least squares (oracle; test use only).

f(x) = sum_s ||A~_s x - p~_s||^2 = x^T H x / 2 + g0^T x + const with
H = 2 sum_s A~_s^T A~_s and g0 = -2 sum_s A~_s^T p~_s (Sec. 2.1, Eq. 2; App. A).
The minimiser over lb <= x <= ub satisfies the KKT conditions
    grad_j >= 0 where x_j = lb_j,  grad_j <= 0 where x_j = ub_j,  grad_j = 0 otherwise.

kkt_bruteforce: enumerate every lower/upper/free assignment (3^n, n <= 10),
    solve the free block of the normal equations, keep the point that is
    feasible and satisfies KKT.
lsq_box: scipy.optimize.lsq_linear on the stacked system (library BVLS/TRF).
box_qp_newton: the same optimum from the dense normal equations by a projected
    Newton method (Bertsekas, SIAM J. Control Optim. 20 (1982)): Newton steps on
    the variables off their bounds, gradient steps on the binding ones, Armijo
    search along the projection arc.  For plans whose stacked system is too big
    for lsq_box in reasonable time (n of a few thousand).
certificates: feasibility, projected-gradient residual and KKT signs of any x.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import lsq_linear

from .problem import Weighted


def _wrap(p):
    return p if isinstance(p, Weighted) else Weighted(p)


def kkt_bruteforce(prob_or_w, tol=1e-9):
    W = _wrap(prob_or_w)
    n = W.n
    if n > 10:
        raise ValueError("brute force is limited to n <= 10")
    H = W.hessian_dense()
    g0 = -2.0 * sum(W.At[s].T @ W.pt[s] for s in range(W.N))
    lb, ub = W.lb, W.ub
    scale = max(1.0, float(np.abs(g0).max()), float(np.abs(H).max()))
    found = []
    for assign in itertools.product((0, 1, 2), repeat=n):   # 0 lb, 1 ub, 2 free
        a = np.array(assign)
        if np.any((a == 1) & ~np.isfinite(ub)) or np.any((a == 0) & ~np.isfinite(lb)):
            continue
        x = np.where(a == 0, lb, np.where(a == 1, ub, 0.0)).astype(np.float64)
        F = a == 2
        if F.any():
            HFF = H[np.ix_(F, F)]
            rhs = -(g0[F] + H[np.ix_(F, ~F)] @ x[~F])
            try:
                x[F] = np.linalg.solve(HFF, rhs)
            except np.linalg.LinAlgError:
                continue
        g = H @ x + g0
        feas = np.all(x >= lb - tol * (1 + np.abs(lb))) and np.all(x <= ub + tol * (1 + np.abs(ub)))
        kkt = (np.all(g[a == 0] >= -tol * scale) and np.all(g[a == 1] <= tol * scale)
               and np.all(np.abs(g[F]) <= tol * scale))
        if feas and kkt:
            found.append(np.minimum(np.maximum(x, lb), ub))
    if not found:
        raise RuntimeError("no KKT point found")
    fs = [W.f(x) for x in found]
    return found[int(np.argmin(fs))]


def lsq_box(prob_or_w, method=None, tol=1e-13, max_iter=None):
    """Bounded least squares on the stacked system; returns x."""
    W = _wrap(prob_or_w)
    A, b = W.stacked()
    if method is None:
        method = "bvls" if W.n <= 400 else "trf"
    if method == "bvls":
        res = lsq_linear(A.toarray(), b, bounds=(W.lb, W.ub), method="bvls", tol=tol,
                         max_iter=max_iter)
    else:
        res = lsq_linear(A, b, bounds=(W.lb, W.ub), method="trf", tol=tol,
                         lsmr_tol="auto", max_iter=max_iter or 1000)
    return np.minimum(np.maximum(res.x, W.lb), W.ub)


def normal_equations(prob_or_w):
    """H = 2 sum_s A~_s^T A~_s (dense), g0 = -2 sum_s A~_s^T p~_s and
    c = sum_s ||p~_s||^2, so that f(x) = x^T H x / 2 + g0^T x + c."""
    W = _wrap(prob_or_w)
    H = np.zeros((W.n, W.n))
    g0 = np.zeros(W.n)
    c = 0.0
    for s in range(W.N):
        A = W.At[s].tocsr()
        H += 2.0 * (A.T @ A).toarray()
        g0 -= 2.0 * (A.T @ W.pt[s])
        c += float(W.pt[s] @ W.pt[s])
    return H, g0, c


def box_qp_newton(prob_or_w, x0=None, tol=1e-13, max_iter=500, sigma=1e-4, normal=None):
    """Minimise f over [lb, ub] by projected Newton; returns x."""
    W = _wrap(prob_or_w)
    H, g0, _ = normal if normal is not None else normal_equations(W)
    lb, ub = W.lb, W.ub
    L = float(np.abs(H).sum(axis=1).max())          # >= lambda_max(H) (Gershgorin)

    def proj(v):
        return np.minimum(np.maximum(v, lb), ub)

    def q(v):
        return 0.5 * float(v @ (H @ v)) + float(g0 @ v)

    x = proj(np.zeros(W.n) if x0 is None else np.asarray(x0, dtype=np.float64))
    for _ in range(max_iter):
        g = H @ x + g0
        w = float(np.abs(x - proj(x - g / L)).max())
        if w <= tol * max(1.0, float(np.abs(x).max())):
            break
        eps = min(1e-6, w)
        B = ((x <= lb + eps) & (g > 0)) | ((x >= ub - eps) & (g < 0))
        F = ~B
        d = np.zeros(W.n)
        if F.any():
            HFF = H[np.ix_(F, F)]
            try:
                d[F] = -np.linalg.solve(HFF, g[F])
            except np.linalg.LinAlgError:
                d[F] = -g[F] / L
        d[B] = -g[B] / L
        qx = q(x)
        a = 1.0
        for _ls in range(60):
            xn = proj(x + a * d)
            dec = -float(g[F] @ (xn - x)[F]) - float(g[B] @ (xn - x)[B])   # >= 0 predicted decrease
            if qx - q(xn) >= sigma * dec:
                break
            a *= 0.5
        x = xn
    return x


def certificates(prob_or_w, x, L=None):
    """Feasibility, projected-gradient residual and KKT-sign violations at x.

    pg = ||x - P(x - grad f(x)/L)||_inf / max(1, ||x||_inf)   (0 exactly at the optimum).
    kkt = largest sign violation of grad f, relative to ||grad f(0)||_inf.
    """
    W = _wrap(prob_or_w)
    from .problem import lipschitz
    if L is None:
        L = lipschitz(W)
    g = W.grad(x)
    g0 = np.abs(W.grad(np.zeros(W.n))).max()
    pg = float(np.abs(x - W.proj(x - g / L)).max() / max(1.0, float(np.abs(x).max())))
    span = np.where(np.isfinite(W.ub - W.lb), W.ub - W.lb, 1.0)
    at_lb = x <= W.lb + 1e-9 * span
    at_ub = x >= W.ub - 1e-9 * span
    free = ~(at_lb | at_ub)
    viol = 0.0
    if at_lb.any():
        viol = max(viol, float(np.max(np.maximum(-g[at_lb], 0.0))))
    if at_ub.any():
        viol = max(viol, float(np.max(np.maximum(g[at_ub], 0.0))))
    if free.any():
        viol = max(viol, float(np.max(np.abs(g[free]))))
    feas = float(max(np.max(W.lb - x, initial=0.0), np.max(x - W.ub, initial=0.0)))
    return dict(pg=pg, kkt=viol / max(g0, 1e-300), infeas=feas, f=W.f(x))
