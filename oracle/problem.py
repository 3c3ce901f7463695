"""Robust weighted least squares over scenarios, float64 (oracle; test use only).

Sec. 2.1: f_s(x) = sum_i w_i (a_{s,i}^T x - p_i)^2        (Eq. 1)
          f(x)   = sum_s f_s(x),  subject to bounds on x   (Eq. 2)
          with optional scenario probabilities c_s: w_i -> c_s w_i.
Eq. 4:    grad f_s(x) = sum_i 2 w_i a_{s,i} (a_{s,i}^T x - p_i).
App. A:   A~_s = diag(sqrt(w)) A_s, p~ = diag(sqrt(w)) p, so that
          f_s(x) = ||A~_s x - p~||^2 and B_s = A~_s^T A~_s + (rho/2) I.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Weighted:
    """The weighted matrices A~_s = diag(sqrt(c_s w)) A_s and p~_s of App. A."""

    def __init__(self, prob):
        self.m, self.n, self.N = prob.m, prob.n, prob.N
        c = np.ones(prob.N) if prob.scen_weight is None else np.asarray(prob.scen_weight, float)
        w = np.asarray(prob.voxel_w, dtype=np.float64)
        p = np.asarray(prob.presc, dtype=np.float64)
        self.c = c
        self.A = []      # unweighted A_s (float64 copy of the float32 input)
        self.At = []     # weighted A~_s
        self.pt = []     # weighted p~_s
        for s in range(prob.N):
            A = prob.csr(s)
            sw = np.sqrt(c[s] * w)
            self.A.append(A)
            self.At.append(sp.diags(sw) @ A)
            self.pt.append(sw * p)
        self.lb = np.asarray(prob.lb, dtype=np.float64)
        self.ub = np.asarray(prob.ub, dtype=np.float64)
        self._b = None

    # ---- bounds ---------------------------------------------------------------
    def proj(self, x):
        """Euclidean projection onto the box [lb, ub] (the max(., 0) of Sec. 2.1/2.2)."""
        return np.minimum(np.maximum(x, self.lb), self.ub)

    # ---- objective and gradient (Eqs. 1, 2, 4) ------------------------------
    def f_s(self, s, x):
        r = self.At[s] @ x - self.pt[s]
        return float(r @ r)

    def f(self, x):
        return sum(self.f_s(s, x) for s in range(self.N))

    def grad_s(self, s, x):
        return 2.0 * (self.At[s].T @ (self.At[s] @ x - self.pt[s]))

    def grad(self, x):
        g = np.zeros(self.n)
        for s in range(self.N):
            g += self.grad_s(s, x)
        return g

    # ---- pieces of the x-subproblem (App. A) -------------------------------
    def b(self, s):
        """Constant part of c_s: A~_s^T p~_s."""
        if self._b is None:
            self._b = [self.At[k].T @ self.pt[k] for k in range(self.N)]
        return self._b[s]

    def normal_apply(self, s, v, rho=0.0):
        """B_s v = A~_s^T A~_s v + (rho/2) v."""
        return self.At[s].T @ (self.At[s] @ v) + 0.5 * rho * v

    def B_dense(self, s, rho):
        G = (self.At[s].T @ self.At[s]).toarray()
        G[np.diag_indices_from(G)] += 0.5 * rho
        return G

    # ---- doses ------------------------------------------------------------------
    def dose(self, s, x):
        """Physical dose A_s x of scenario s."""
        return self.A[s] @ x

    def stacked_weighted_dose(self, x):
        """[A~_1 x; ...; A~_N x] -- unique at the optimum when all w_i > 0."""
        return np.concatenate([self.At[s] @ x for s in range(self.N)])

    def stacked(self):
        """The stacked system [A~_1; ...; A~_N] x ~ [p~_1; ...; p~_N]."""
        return sp.vstack(self.At).tocsr(), np.concatenate(self.pt)

    def hessian_dense(self):
        """H = 2 sum_s A~_s^T A~_s (f is quadratic: f(x) = x'Hx/2 + g0'x + const)."""
        H = np.zeros((self.n, self.n))
        for s in range(self.N):
            H += 2.0 * (self.At[s].T @ self.At[s]).toarray()
        return H

    def const(self):
        return float(sum(p @ p for p in self.pt))


def default_rho(W: Weighted) -> float:
    """rho = 2 * mean_s(trace(A~_s^T A~_s) / n): (rho/2) I then equals the mean
    diagonal of A~_s^T A~_s.  The paper gives rho no value (Sec. 2.2)."""
    tr = [float(W.At[s].multiply(W.At[s]).sum()) for s in range(W.N)]
    return 2.0 * float(np.mean(tr)) / W.n


def lipschitz(W: Weighted, iters: int = 30) -> float:
    """L = 2 lambda_max(sum_s A~_s^T A~_s), by power iteration from ones/sqrt(n)."""
    v = np.ones(W.n) / np.sqrt(W.n)
    lam = 0.0
    for _ in range(iters):
        u = np.zeros(W.n)
        for s in range(W.N):
            u += W.normal_apply(s, v)
        lam = float(np.linalg.norm(u))
        if lam == 0.0:
            return 0.0
        v = u / lam
    return 2.0 * lam
