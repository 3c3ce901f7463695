"""Write tests/golden/realistic_seed0_oracle.json from the CPU oracle only.

Workload: synthetic.config_realistic(seed=0) (128x128x96 grid, ~299k voxels,
5000 spots, 13 scenarios).  Records
  * the exact box-constrained optimum z* and f* of the plan
    (oracle.exact.box_qp_newton on the dense normal equations) with its
    optimality certificates;
  * ADMM-BB with CG subproblems and the library's default parameters
    (rho = default rule, eps = 1e-4, theta 0.15, eta0 1e-2, floor 1e-6, at most
    50 steps, Jacobi): iterations and CG steps to tolerance and the objective,
    used to extrapolate the CPU timing of a bounded sample;
  * the paper's ADMM-BB with cached Cholesky subproblems (App. A) at eps = 1e-4;
  * a checksum of the generated matrices so a differing platform is noticed.
The file is rewritten after every stage.
Run: python tests/golden/make_realistic_golden.py   (about an hour, CPU only)
     python tests/golden/make_realistic_golden.py exact   (the exact stage alone,
     a few minutes; the other stages' records in the file are kept)
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def main(stages=("exact", "admm_cg", "admm_chol")):
    from synthetic import config_realistic
    from oracle import Weighted, admm_bb, default_rho, certificates, box_qp_newton
    out_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "realistic_seed0_oracle.json")
    t0 = time.time()
    prob = config_realistic(0, workers=8)
    nnz = [int(v.size) for v in prob.val]
    checksum = float(sum(float(np.sum(v.astype(np.float64))) for v in prob.val))
    W = Weighted(prob)
    rho0 = default_rho(W)
    res = {}
    if os.path.exists(out_path):
        old = json.load(open(out_path))
        if old.get("value_sum") == checksum:     # records of the same matrices are kept
            res = old
    res.update(workload="config_realistic(seed=0)", m=prob.m, n=prob.n, N=prob.N, nnz=nnz,
               value_sum=checksum, default_rho=rho0, made_by="tests/golden/make_realistic_golden.py")

    def save():
        res["total_seconds"] = time.time() - t0
        json.dump(res, open(out_path, "w"), indent=1)

    if "exact" in stages:
        t1 = time.time()
        xs = box_qp_newton(W)
        c = certificates(W, xs)
        res["exact"] = dict(method="box_qp_newton", f=W.f(xs), pg=c["pg"], kkt=c["kkt"],
                            seconds=time.time() - t1, at_lb=int((xs <= W.lb).sum()),
                            at_ub=int((xs >= W.ub).sum()))
        res["f_star"] = W.f(xs)
        # z* (unique: the Hessian has full rank) and the norm of its stacked weighted dose
        res["z_star"] = [float(v) for v in xs]
        res["dose_norm_star"] = float(np.linalg.norm(W.stacked_weighted_dose(xs)))
        save()
    if "admm_cg" in stages:
        rc = admm_bb(W, rho=rho0, eps_abs=1e-4, eps_rel=1e-4, max_iter=20000, subproblem="cg",
                     cg_theta=0.15, cg_eta0=1e-2, cg_floor_rel=1e-6, cg_max=50, cg_precond="jacobi")
        res["admm_cg"] = dict(eps=1e-4, iterations=rc["iterations"], cg_iterations=rc["cg_iterations"],
                              status=rc["status"], f=rc["f"], seconds=rc["seconds"])
        save()
    if "admm_chol" in stages:
        r4 = admm_bb(W, rho=rho0, eps_abs=1e-4, eps_rel=1e-4, max_iter=20000, subproblem="chol")
        res["admm_chol"] = dict(eps=1e-4, iterations=r4["iterations"], status=r4["status"], f=r4["f"],
                                seconds=r4["seconds"])
        save()

if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ("exact", "admm_cg", "admm_chol"))
