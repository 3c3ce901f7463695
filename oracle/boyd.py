"""Textbook consensus ADMM in scaled form (Boyd et al. 2011, Sec. 7.1), float64
(oracle; test use only).

Written independently of admm_bb.py, in the scaled dual u_s = y_s / rho:
    x_s <- argmin f_s(x) + (rho/2)||x - z + u_s||^2
         = (A~_s^T A~_s + (rho/2) I)^{-1} (A~_s^T p~ + (rho/2)(z - u_s))
    z   <- P_box(mean_s(x_s + u_s))
    u_s <- u_s + x_s - z
With the BB step switched off, ADMM-BB (Sec. 2.2, z-update read as the exact
z-minimiser) is this method written with y_s = rho u_s, so both produce the
same iterates.
"""
from __future__ import annotations

import numpy as np

from .problem import Weighted


def consensus_admm_scaled(prob_or_w, rho, iters, z0=None):
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    N, n = W.N, W.n
    Minv = [np.linalg.inv(W.B_dense(s, rho)) for s in range(N)]
    q = [W.At[s].T @ W.pt[s] for s in range(N)]
    z = W.proj(np.zeros(n) if z0 is None else np.asarray(z0, float))
    u = np.zeros((N, n))
    xs = np.zeros((N, n))
    zs = []
    for _ in range(iters):
        for s in range(N):
            xs[s] = Minv[s] @ (q[s] + 0.5 * rho * (z - u[s]))
        z = W.proj((xs + u).mean(axis=0))
        u = u + xs - z[None, :]
        zs.append(z.copy())
    return dict(z=z, x=xs.copy(), y=rho * u, z_hist=zs)
