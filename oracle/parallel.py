"""ADMM-BB with cached Cholesky subproblems spread over worker processes, the
way the paper ran it (Sec. 2.3: Python multiprocessing, scenario subproblems
in parallel; App. A: B_s = A~_s^T A~_s + (rho/2) I factored once per scenario).

TEST INFRASTRUCTURE ONLY: the CPU baseline of the benchmark and its tests.
The arithmetic is that of admm_bb(subproblem="chol"): each worker owns a set of
scenarios, forms and factors their B_s once, and per iteration returns
x_s = B_s^{-1} (A~_s^T p~_s + (rho/2)(z - y_s/rho)); the z-update, the BB step,
the dual update and the stopping rule run in the calling process (admm_bb with
an xupdate callable).  Workers are started with the "spawn" method (safe after
a GPU context exists in the caller), and each worker's BLAS thread count is set
through the environment before it starts.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .admm_bb import admm_bb
from .problem import Weighted, default_rho

_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _serve(conn):
    """Worker: receive its scenarios, factor their B_s, then answer x-updates."""
    kind, rho, items = conn.recv()
    t0 = time.perf_counter()
    fac, b = [], []
    for data, indices, indptr, shape, pt in items:
        At = sp.csr_matrix((data, indices, indptr), shape=shape)
        G = (At.T @ At).toarray()
        G[np.diag_indices_from(G)] += 0.5 * rho
        fac.append(sla.cho_factor(G, lower=False, check_finite=False))
        b.append(At.T @ pt)
        del G
    conn.send(time.perf_counter() - t0)
    while True:
        msg = conn.recv()
        if msg is None:
            break
        z, ys = msg
        conn.send(np.stack([sla.cho_solve(F, bs + 0.5 * rho * (z - y / rho), check_finite=False)
                            for F, bs, y in zip(fac, b, ys)]))
    conn.close()


class ScenarioPool:
    """Worker processes that hold the cached factors of the scenario subproblems."""

    def __init__(self, W: Weighted, rho: float, workers: int, blas_threads: int):
        self.N = W.N
        self.groups = [g.tolist() for g in np.array_split(np.arange(W.N), max(1, min(workers, W.N)))]
        self.groups = [g for g in self.groups if g]
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in _BLAS_VARS}
        self.conns, self.procs = [], []
        try:
            for k in _BLAS_VARS:
                os.environ[k] = str(blas_threads)
            for g in self.groups:
                a, b = ctx.Pipe()
                p = ctx.Process(target=_serve, args=(b,), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        t0 = time.perf_counter()
        for c, g in zip(self.conns, self.groups):
            c.send(("setup", rho, [(W.At[s].data, W.At[s].indices, W.At[s].indptr, W.At[s].shape, W.pt[s])
                                   for s in g]))
        self.factor_s = max(c.recv() for c in self.conns)          # slowest worker's factor time
        self.setup_s = time.perf_counter() - t0                       # including the transfer

    def xupdate(self, z, y):
        for c, g in zip(self.conns, self.groups):
            c.send((z, y[g]))
        x = np.empty((self.N, z.size))
        for c, g in zip(self.conns, self.groups):
            x[g] = c.recv()
        return x

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()


def admm_bb_chol_parallel(prob_or_w, rho=None, workers=None, blas_threads=None, **kw):
    """admm_bb(subproblem="chol") with the scenario subproblems on `workers`
    processes (default: one per scenario, at most the usable cores) of
    `blas_threads` BLAS threads each (default: the cores shared out).  Returns
    admm_bb's result plus setup_s (transfer, forming and factoring B_s),
    factor_s, workers and blas_threads; "seconds" is the iteration time."""
    W = prob_or_w if isinstance(prob_or_w, Weighted) else Weighted(prob_or_w)
    if rho is None:
        rho = default_rho(W)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    workers = max(1, min(W.N, cores if workers is None else workers))
    blas_threads = max(1, cores // workers) if blas_threads is None else blas_threads
    pool = ScenarioPool(W, rho, workers, blas_threads)
    try:
        res = admm_bb(W, rho=rho, subproblem="chol", xupdate=pool.xupdate, **kw)
    finally:
        pool.close()
    res.update(setup_s=pool.setup_s, factor_s=pool.factor_s, workers=len(pool.groups),
               blas_threads=blas_threads, cores=cores)
    return res
