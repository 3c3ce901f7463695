"""Projected gradient descent with Armijo backtracking, float64 (oracle; test use only).

Sec. 2.1: grad f(x^k) = sum_s sum_i 2 w_i a_{s,i}(a_{s,i}^T x^k - p_i)
          x^{k+1} = P_box(x^k - t_k grad f(x^k))
The step t_k starts at alpha and shrinks by gamma until the sufficient
decrease condition (Eq. 3, read as Nocedal-Wright Sec. 3.1; the printed
inequality points the wrong way)
          f(x^{k+1}) <= f(x^k) + beta grad f(x^k)^T (x^{k+1} - x^k)
holds.  Stop when |f(x^k) - f(x^{k+1})| / f(x^k) <= tol_rel_df.
Defaults (the paper gives none): alpha = 4 / L with L = 2 lambda_max(sum_s
A~_s^T A~_s), beta = 1e-4, gamma = 0.5, at most 30 trials per iteration.
"""
from __future__ import annotations

import math
import time

import numpy as np

from .problem import Weighted, lipschitz


def pgd(prob_or_w, alpha=None, beta=1e-4, gamma=0.5, tol_rel_df=1e-5, max_iter=10000,
        max_trials=30, x0=None, f_target=None, record=False):
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    t0 = time.perf_counter()
    if alpha is None:
        alpha = 4.0 / lipschitz(W)
    x = W.proj(np.zeros(W.n) if x0 is None else np.asarray(x0, float).copy())
    fx = W.f(x)
    hist = []
    status = "not_converged"
    trials_total = 0
    it = 0
    for k in range(max_iter):
        g = W.grad(x)
        t = alpha
        accepted = False
        for _ in range(max_trials):
            xt = W.proj(x - t * g)
            ft = W.f(xt)
            trials_total += 1
            if ft <= fx + beta * float(g @ (xt - x)):
                accepted = True
                break
            t *= gamma
        if not accepted:
            status = "line_search_failed"
            break
        rel = abs(fx - ft) / max(abs(fx), 1e-300)
        x, fx = xt, ft
        it = k + 1
        if record:
            hist.append(dict(k=it, t=time.perf_counter() - t0, f=fx, step=t))
        if f_target is not None and fx <= f_target:
            status = "reached_target"
            break
        if rel <= tol_rel_df:
            status = "converged"
            break
    return dict(x=x, f=fx, iterations=it, trials=trials_total, status=status, alpha=alpha,
                history=hist, seconds=time.perf_counter() - t0)
