"""Linear dose constraints as extra ADMM blocks, float64 (oracle; test use only).

Sec. 4 notes that ADMM, unlike PGD, accepts any linear constraint on the plan,
for instance maximum or mean dose limits, while the paper's runs use only the
box.  The paper gives no formulation; this module fixes one (a reading) and
the exact optimum it must reach.

Problem.  minimise f(x) = sum_s ||A~_s x - p~||^2 (Eq. 2) over lb <= x <= ub
and, in every scenario s (robust limits), G_s x <= h_s, where each row of G_s
is built from the physical dose A_s (unweighted) of one constraint:
    "max"  limit on every voxel i of a set:  a_{s,i}^T x <= D
    "min"  floor on every voxel i of a set:  -a_{s,i}^T x <= -D
    "mean" limit on a set's mean dose:       (1/|S|) sum_{i in S} a_{s,i}^T x <= D

Splitting (two ADMM blocks: {x_s} and {z, v_s}).  Besides the consensus
x_s = z of Eq. 5, each scenario gets v_s = G_s x_s with v_s <= h_s and a
second dual mu_s with a fixed penalty sigma.  One iteration:
  1. x_s = argmin f_s(x) + (rho/2)||x - z + y_s/rho||^2 + (sigma/2)||G_s x - v_s + mu_s/sigma||^2
     i.e. (A~_s'A~_s + (rho/2) I + (sigma/2) G_s'G_s) x
            = A~_s'p~ + (rho/2)(z - y_s/rho) + (sigma/2) G_s'(v_s - mu_s/sigma)
  2. z   = P_box(mean_s(x_s + y_s/rho))                      (Z-STD, as in Eq. 5-7)
     v_s = min(G_s x_s + mu_s/sigma, h_s)                     (projection on v <= h)
  3. y_s += step (x_s - z), step by Eq. 8 over the consensus blocks
     mu_s += sigma (G_s x_s - v_s)
  4. stop when r_prim <= eps_prim and r_dual <= eps_dual (Eq. 9 extended to
     both constraint blocks, in the usual two-block form):
       r_prim = ||[x_s - z ; G_s x_s - v_s]_s||
       r_dual = ||[rho (z - z_prev) + sigma G_s'(v_s - v_s_prev)]_s||
       eps_prim = eps_abs sqrt(N n + K) + eps_rel max(||[x_s ; G_s x_s]_s||, ||[z ; v_s]_s||)
     (K the number of constraint rows over all scenarios; z counted once per scenario)
       eps_dual = eps_abs sqrt(N n) + eps_rel ||[y_s + G_s' mu_s]_s||
With no constraint rows this is admm_bb (Cholesky subproblem) step for step.
At a fixed point x_s = z, v_s = G_s z, mu_s >= 0 and mu_s'(G_s z - h_s) = 0, and
grad f(z) + sum_s G_s' mu_s + sum_s y_s = 0 with -sum_s y_s in the box's normal
cone: the KKT conditions of the constrained problem, mu_s its multipliers.

kkt_bruteforce_lin: the exact optimum by enumerating, for every spot,
lower/upper/free, and for every constraint row, active/inactive (n and the row
count tiny), solving the equality-constrained KKT system of each pattern and
keeping the feasible point with valid multipliers.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .problem import Weighted


@dataclass
class DoseConstraint:
    kind: str            # "max" | "min" | "mean"
    voxels: np.ndarray   # voxel (row) indices of the structure
    limit: float         # Gy


def constraint_rows(W: Weighted, cons):
    """(G_s, h_s) for every scenario: G_s sparse [K x n], h_s [K], K the same in
    every scenario (rows in the order of `cons`, voxels in the given order)."""
    G, h = [], []
    for s in range(W.N):
        A = W.A[s].tocsr()
        rows, lim = [], []
        for c in cons:
            idx = np.asarray(c.voxels, dtype=np.int64)
            if c.kind == "max":
                rows.append(A[idx])
                lim.append(np.full(len(idx), float(c.limit)))
            elif c.kind == "min":
                rows.append(-A[idx])
                lim.append(np.full(len(idx), -float(c.limit)))
            elif c.kind == "mean":
                rows.append(sp.csr_matrix(np.asarray(A[idx].sum(axis=0)) / len(idx)))
                lim.append(np.array([float(c.limit)]))
            else:
                raise ValueError(c.kind)
        if rows:
            G.append(sp.vstack(rows).tocsr())
            h.append(np.concatenate(lim))
        else:
            G.append(sp.csr_matrix((0, W.n)))
            h.append(np.zeros(0))
    return G, h


def admm_bb_constrained(prob_or_w, cons, rho=None, sigma=None, eps_abs=1e-4, eps_rel=1e-4,
                        max_iter=1000, bb="paper", bb_kappa=10.0, z0=None):
    """ADMM-BB with the dose-constraint blocks above; Cholesky subproblems.
    sigma defaults to rho (the two penalties on the same scale)."""
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    N, n = W.N, W.n
    if rho is None:
        from .problem import default_rho
        rho = default_rho(W)
    if sigma is None:
        sigma = rho
    G, h = constraint_rows(W, cons)
    K = sum(len(hs) for hs in h)
    b = [W.b(s) for s in range(N)]
    fac = []
    for s in range(N):
        B = W.B_dense(s, rho) + 0.5 * sigma * (G[s].T @ G[s]).toarray()
        fac.append(sla.cho_factor(B, lower=False))
    z = W.proj(np.zeros(n) if z0 is None else np.asarray(z0, float).copy())
    x = np.tile(z, (N, 1))
    y = np.zeros((N, n))
    v = [np.minimum(G[s] @ z, h[s]) for s in range(N)]
    mu = [np.zeros(len(h[s])) for s in range(N)]
    d_prev = x - z[None, :]
    y_prev = None
    status = "not_converged"
    step = rho
    it = 0
    for k in range(max_iter):
        # 1. scenario subproblems
        xn = np.empty_like(x)
        for s in range(N):
            c = b[s] + 0.5 * rho * (z - y[s] / rho) + 0.5 * sigma * (G[s].T @ (v[s] - mu[s] / sigma))
            xn[s] = sla.cho_solve(fac[s], c)
        # 2. second block: consensus projection and the dose variables
        zn = W.proj(np.mean(xn + y / rho, axis=0))
        Gx = [G[s] @ xn[s] for s in range(N)]
        vn = [np.minimum(Gx[s] + mu[s] / sigma, h[s]) for s in range(N)]
        # 3. duals: BB step (Eq. 8) on the consensus blocks, fixed sigma on the dose blocks
        d = xn - zn[None, :]
        step = rho
        if bb != "off" and y_prev is not None:
            dd = (d - d_prev).ravel()
            dy = (y - y_prev).ravel()
            den = float(dd @ dd)
            if den > 0.0:
                beta = -float(dd @ dy) / den
                if math.isfinite(beta) and beta > 0.0:
                    step = beta
                    if bb == "guarded":
                        step = min(max(step, rho / bb_kappa), bb_kappa * rho)
        yn = y + step * d
        mun = [mu[s] + sigma * (Gx[s] - vn[s]) for s in range(N)]
        # 4. residuals
        r_prim = math.sqrt(float(np.sum(d * d)) + sum(float(np.sum((Gx[s] - vn[s]) ** 2)) for s in range(N)))
        r_dual = math.sqrt(sum(float(np.sum((rho * (zn - z) + sigma * (G[s].T @ (vn[s] - v[s]))) ** 2))
                               for s in range(N)))
        ax = math.sqrt(float(np.sum(xn * xn)) + sum(float(g @ g) for g in Gx))
        bz = math.sqrt(N * float(zn @ zn) + sum(float(w @ w) for w in vn))
        eps_prim = eps_abs * math.sqrt(N * n + K) + eps_rel * max(ax, bz)
        aty = math.sqrt(sum(float(np.sum((yn[s] + G[s].T @ mun[s]) ** 2)) for s in range(N)))
        eps_dual = eps_abs * math.sqrt(N * n) + eps_rel * aty
        y_prev, y = y, yn
        x, z, v, mu, d_prev = xn, zn, vn, mun, d
        it = k + 1
        if not (math.isfinite(r_prim) and math.isfinite(r_dual)):
            status = "diverged"
            break
        if r_prim <= eps_prim and r_dual <= eps_dual:
            status = "converged"
            break
    return dict(z=z, x=x, y=y, v=v, mu=mu, iterations=it, status=status, rho=rho, sigma=sigma,
                step=step, r_prim=r_prim, r_dual=r_dual, eps_prim=eps_prim, eps_dual=eps_dual,
                f=W.f(z), G=G, h=h)


def kkt_bruteforce_lin(prob_or_w, G_all, h_all, tol=1e-9):
    """Exact minimiser of f over {lb <= x <= ub, G_all x <= h_all} by active-set
    enumeration (n <= 6, at most 8 rows): for every pattern solve
        [H_FF  C_F'] [x_F]   [-(g0_F + H_FA x_A)]
        [C_F   0   ] [lam] = [ h_C - C_A x_A    ]
    (C the active rows), then keep the points that are feasible, have lam >= 0
    and the right signs of the bound multipliers.  Returns (x, lam_full)."""
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    n = W.n
    Gd = np.asarray(G_all.toarray() if sp.issparse(G_all) else G_all, dtype=np.float64)
    hh = np.asarray(h_all, dtype=np.float64)
    K = Gd.shape[0]
    if n > 6 or K > 8:
        raise ValueError("brute force is limited to n <= 6 and 8 constraint rows")
    H = W.hessian_dense()
    g0 = -2.0 * sum(W.At[s].T @ W.pt[s] for s in range(W.N))
    lb, ub = W.lb, W.ub
    scale = max(1.0, float(np.abs(g0).max()), float(np.abs(H).max()))
    best = None
    for assign in itertools.product((0, 1, 2), repeat=n):   # 0 lb, 1 ub, 2 free
        a = np.array(assign)
        if np.any((a == 1) & ~np.isfinite(ub)) or np.any((a == 0) & ~np.isfinite(lb)):
            continue
        xA = np.where(a == 0, lb, np.where(a == 1, ub, 0.0)).astype(np.float64)
        F = a == 2
        nf = int(F.sum())
        for act in itertools.product((0, 1), repeat=K):
            Ci = np.flatnonzero(np.array(act, dtype=bool)) if K else np.zeros(0, dtype=int)
            nc = len(Ci)
            if nc > nf:
                continue
            x = xA.copy()
            lam = np.zeros(K)
            if nf:
                CF = Gd[np.ix_(Ci, F)]
                M = np.zeros((nf + nc, nf + nc))
                M[:nf, :nf] = H[np.ix_(F, F)]
                M[:nf, nf:] = CF.T
                M[nf:, :nf] = CF
                rhs = np.concatenate([-(g0[F] + H[np.ix_(F, ~F)] @ xA[~F]),
                                      hh[Ci] - Gd[np.ix_(Ci, ~F)] @ xA[~F]])
                try:
                    sol = np.linalg.solve(M, rhs)
                except np.linalg.LinAlgError:
                    continue
                if not np.all(np.isfinite(sol)):
                    continue
                x[F] = sol[:nf]
                lam[Ci] = sol[nf:]
            elif nc:
                continue
            gl = H @ x + g0 + Gd.T @ lam            # gradient of the Lagrangian (box terms aside)
            feas = (np.all(x >= lb - tol * (1 + np.abs(lb))) and np.all(x <= ub + tol * (1 + np.abs(ub)))
                    and np.all(Gd @ x <= hh + tol * (1 + np.abs(hh))))
            kkt = (np.all(lam >= -tol * scale) and np.all(gl[a == 0] >= -tol * scale)
                   and np.all(gl[a == 1] <= tol * scale) and np.all(np.abs(gl[F]) <= tol * scale))
            if feas and kkt:
                fx = W.f(x)
                if best is None or fx < best[0]:
                    best = (fx, np.minimum(np.maximum(x, lb), ub), lam)
    if best is None:
        raise RuntimeError("no KKT point found")
    return best[1], best[2]
