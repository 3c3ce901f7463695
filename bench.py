#!/usr/bin/env python
"""Benchmark: ADMM-BB time-to-tolerance on the realistic robust-planning workload.

Workload: 128x128x96 grid (2.5 mm), ~299k voxels, 5000 spots from 3 beams, 13
uncertainty scenarios, ~2000 entries per spot column (~127M entries, CSR int32
indices + float32 values, ~1.02 GB); ADMM-BB to the Eq. 9 residual rule at
eps_abs = eps_rel = 1e-4 from a cold start.  One step = one full solve with the
plan resident in HBM.  The matrices (1 GB) are larger than L2 (129 MB), so no
explicit L2 flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADMM-BB time-to-tolerance (s), SpMV GB/s vs HBM peak: plain vs mixed/learned"
WORKLOAD = "realistic: 128x128x96 grid, 299k voxels, 5000 spots, 13 scenarios, ~2000 nnz/spot, F32+int32 CSR"


def max_over_ranks(value, world, device=None):
    """The largest of every rank's value (a step time is max-reduced across the
    job); world 1: the value itself.  device: where the reduction tensor lives
    (the rank's GPU with NCCL, None for the CPU with gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _golden_fstar():
    """The oracle's exact optimum of the benchmark workload (seed 0), if stored."""
    path = os.path.join(ROOT, "tests", "golden", "realistic_seed0_oracle.json")
    try:
        return json.load(open(path))["f_star"]
    except Exception:
        return None


def _workload(seed, workers):
    from synthetic import config_realistic
    return config_realistic(seed=seed, workers=workers)


def cpu_baseline(prob, budget_s=20.0):
    """The paper's own CPU method, timed to completion on the host cores: the
    oracle's ADMM-BB with cached-Cholesky subproblems (App. A) spread over worker
    processes, one or more scenarios each (Sec. 2.3: Python multiprocessing),
    BLAS threads shared out among the workers; eps_abs = eps_rel = 1e-4, the
    library's default rho, cold start.  value = forming and factoring B_s (in the
    workers, in parallel) + the iterations to tolerance.  budget_s is unused:
    the solve is run in full (about half a minute on 16 cores)."""
    from oracle import Weighted, default_rho
    from oracle.parallel import admm_bb_chol_parallel
    t0 = time.perf_counter()
    W = Weighted(prob)
    t_w = time.perf_counter() - t0
    res = admm_bb_chol_parallel(W, rho=default_rho(W), eps_abs=1e-4, eps_rel=1e-4, max_iter=20000)
    total = res["setup_s"] + res["seconds"]
    return {"value": total, "unit": "s", "cores": res["cores"], "kind": "oracle",
            "sample": (f"complete solve, not a sample: oracle ADMM-BB with cached-Cholesky subproblems on "
                       f"{res['workers']} worker processes x {res['blas_threads']} BLAS threads, "
                       f"{res['iterations']} iterations to eps 1e-4 ({res['status']}); setup (transfer, "
                       f"form and factor B_s) {res['setup_s']:.1f} s + iterations {res['seconds']:.1f} s"),
            "iterations": res["iterations"], "setup_s": round(res["setup_s"], 2),
            "iterate_s": round(res["seconds"], 2), "workers": res["workers"], "blas_threads": res["blas_threads"],
            "weighting_s": round(t_w, 2), "f": res["f"]}


def cpu_one_core_sample(prob, iters=20):
    """The same method on one core (one worker, one BLAS thread), as a bounded
    sample: scenario 0 is formed and factored, `iters` of its x-updates are
    timed; the full solve is estimated as N times the factor time plus
    N x iterations x the x-update time (the iteration count of the all-core run)."""
    import numpy as np
    from oracle import Weighted, default_rho
    from oracle.parallel import ScenarioPool
    W = Weighted(prob.subset_scenarios([0]))
    pool = ScenarioPool(W, default_rho(Weighted(prob)), workers=1, blas_threads=1)
    try:
        z = np.zeros(prob.n)
        y = np.zeros((1, prob.n))
        t0 = time.perf_counter()
        for _ in range(iters):
            pool.xupdate(z, y)
        per = (time.perf_counter() - t0) / iters
    finally:
        pool.close()
    return {"factor_s_per_scenario": pool.factor_s, "xupdate_s_per_scenario": per, "cores": 1, "blas_threads": 1}


def cg_extrapolated(prob, budget_s=20.0):
    """Labelled extra: the oracle's ADMM-BB with CG subproblems (the GPU's
    method, same parameters), first iterations timed in one process and scaled
    by the oracle's own scenario-pass count to tolerance (golden file)."""
    from oracle import Weighted, admm_bb, default_rho
    gold_path = os.path.join(ROOT, "tests", "golden", "realistic_seed0_oracle.json")
    W = Weighted(prob)
    rho = default_rho(W)
    t1 = time.perf_counter()
    k = 0
    res = None
    while time.perf_counter() - t1 < budget_s and k < 50:
        k += 1
        res = admm_bb(W, rho=rho, eps_abs=1e-4, eps_rel=1e-4, max_iter=k, subproblem="cg",
                      cg_theta=0.15, cg_eta0=1e-2, cg_floor_rel=1e-6, cg_max=50, cg_precond="jacobi")
        if time.perf_counter() - t1 > budget_s / 2:
            break
    passes_sample = res["cg_iterations"] + k * prob.N
    if not os.path.exists(gold_path):
        return None
    cg = json.load(open(gold_path))["admm_cg"]
    passes_total = cg["cg_iterations"] + cg["iterations"] * prob.N
    return {"value": res["seconds"] / passes_sample * passes_total, "unit": "s", "kind": "oracle, extrapolated",
            "sample": f"first {k} CG ADMM-BB iterations ({res['seconds']:.1f} s, {passes_sample} scenario "
                      f"passes) scaled to the oracle's {passes_total} passes to tolerance"}


def run_batch(args, rpt, dev, stream, peak):
    """Batched form: plans of uneven size solved one by one, then together as
    one batched plan (rpt_plans_create_batched: one persistent row pass over
    the scenarios of every plan still iterating, each plan with its own
    penalty, BB step and stop; ring configuration picked by the autotuner), and
    for reference as one block-diagonal problem (one shared penalty, BB step
    and stop).  'large': four plans over 49 scenarios; 'small': eight plans over
    13 scenarios, each too small to fill the GPU alone."""
    import numpy as np
    import torch
    from synthetic import config_batch, block_diagonal, BATCH_SIZES_SMALL, scenario_set_13
    t0 = time.perf_counter()
    if args.batch == "small":
        probs = config_batch(args.seed, workers=args.workers, nnz_per_col=1500.0,
                             scenarios=scenario_set_13(), sizes=BATCH_SIZES_SMALL)
        label = ("8 plans (voxels, spots) = 12k/250 ... 54k/950 in steps of 6k/100; 13 scenarios each; "
                 "~1500 nnz/spot")
    else:
        probs = config_batch(args.seed, workers=args.workers)
        label = "4 plans (voxels, spots) = 100k/2k, 170k/3k, 230k/4k, 300k/5k; 49 scenarios each; ~1700 nnz/spot"
    gen_s = time.perf_counter() - t0
    params = rpt.admm_params()

    def timed(fn):
        fn()                                                 # warm-up (graph capture)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1) / 1e3

    seq = []
    for p in probs:
        P = rpt.Plan.from_problem(p, device=dev, stream=stream.cuda_stream)
        (z, info), t = timed(lambda: P.admm_bb_solve(params))
        ms, by = P.profile_row_pass(0, reps=10)
        seq.append({"m": p.m, "n": p.n, "nnz": int(P.stats()["nnz"]), "solve_s": t, "iterations": info["iterations"],
                    "f": info["f"], "pass_ms": ms, "pass_gbs": by / ms / 1e6})
        P.close()
    t1 = time.perf_counter()
    P = rpt.Plan.batched(probs, device=dev, stream=stream.cuda_stream, autotune=1)
    create_s = time.perf_counter() - t1
    st = P.stats()
    (xs, info, per), t = timed(lambda: P.admm_bb_solve_batched(params))
    ms, by = P.profile_row_pass(0, reps=10)
    P.close()
    batched = {"nnz": int(st["nnz"]), "create_s": create_s, "solve_s": t, "status": info["status"],
               "iterations": info["iterations"], "iterations_per_plan": [q["iterations"] for q in per],
               "status_per_plan": [q["status"] for q in per], "rho_per_plan": [q["rho"] for q in per],
               "row_passes": info["row_passes"], "f": info["f"], "f_per_plan": [q["f"] for q in per],
               "f_rel_vs_alone": [(q["f"] - a["f"]) / a["f"] for q, a in zip(per, seq)],
               "pass_ms_all_plans": ms, "pass_gbs": by / ms / 1e6, "frac_of_peak": by / ms / 1e6 / peak,
               "ring": {"chunk_entries": st["chunk_entries"], "chunk_rows": st["chunk_rows"],
                        "stages": st["stages"], "configs_timed": st["autotuned"]}}
    big = block_diagonal(probs)
    del probs
    P = rpt.Plan.from_problem(big, device=dev, stream=stream.cuda_stream, autotune=1)
    del big
    (z, infob), tb = timed(lambda: P.admm_bb_solve(params))
    P.close()
    one = sum(q["solve_s"] for q in seq)
    return {"workload": label, "generate_s": round(gen_s, 1),
            "one_by_one": seq, "one_by_one_solve_s": one,
            "batched": batched, "speedup_batched_over_one_by_one": one / t,
            "block_diagonal_shared_step": {"solve_s": tb, "iterations": infob["iterations"],
                                           "status": infob["status"], "f": infob["f"]}}


def run_learned(args, rpt, dev, stream, n_train=2000, n_test=200):
    """Learned warm start against the cold start at the learned form's scale:
    an MLP 9 -> 512 -> 512 -> 512 -> 200 with bfloat16 weights on the tensor
    cores (FP32 accumulation), trained on the GPU by the library's kernels on
    n_train solutions that the solver generates over a sweep of structure
    weights (log-uniform in [0.1, 100]) and prescriptions ([60, 75] Gy) of the
    20^3 tiny geometry (one plan, reweighted in place; each training target
    solved to eps 1e-6 with the cached-factor x-update).  n_test held-out
    settings are then solved to eps = 1e-4 with the benchmark's method (CG
    x-updates) from a cold start and from the network's z0, each timed with
    CUDA events (the learned time includes the network's inference and, if the
    warm start fails, the cold-start fallback)."""
    import numpy as np
    import torch
    from synthetic import config_tiny_plain, reweighted, sample_weights, N_WEIGHT_SLOTS

    def features(sw, d):
        f = np.zeros(N_WEIGHT_SLOTS + 1, dtype=np.float32)
        nz = sw > 0
        f[:N_WEIGHT_SLOTS][nz] = np.log10(sw[nz]) / 2.0
        f[-1] = (d - 67.5) / 7.5
        return f

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1) / 1e3

    base = config_tiny_plain(args.seed)
    rng = np.random.default_rng(7)
    settings = [sample_weights(rng, base.labels) for _ in range(n_train + n_test)]
    feats, targets = [], []
    t0 = time.perf_counter()
    statuses = []
    with rpt.Plan.from_problem(base, device=dev, stream=stream.cuda_stream) as P:
        for sw, d in settings[:n_train]:
            prob = reweighted(base, sw, d)
            P.set_weights(prob.voxel_w, prob.presc)
            z, info = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, subproblem=rpt.SUB_CHOL)
            statuses.append(info["status"])
            feats.append(features(sw, d))
            targets.append((z / base.ub).astype(np.float32))
        gen_s = time.perf_counter() - t0
        X, Y = np.stack(feats), np.stack(targets)
        rows = []
        with rpt.Mlp(X.shape[1], 512, 3, base.n, seed=2, device=dev) as net:
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            final_loss = net.train(X, Y, epochs=150, batch=128, lr=1e-3)
            torch.cuda.synchronize(dev)
            train_s = time.perf_counter() - t1
            warm_graph = False
            for sw, d in settings[n_train:]:
                prob = reweighted(base, sw, d)
                P.set_weights(prob.voxel_w, prob.presc)
                f = features(sw, d)
                if not warm_graph:
                    P.admm_bb_solve()                                # warm-up (graph capture)
                    warm_graph = True
                (_, ic), tc = timed(lambda: P.admm_bb_solve())
                (_, iw, used), tw = timed(lambda: rpt.admm_bb_solve_learned(P, net, f, base.ub))
                rows.append((tc, ic["iterations"], tw, iw["iterations"], bool(used), ic["f"], iw["f"],
                             ic["status"], iw["status"]))
    return {"workload": (f"tiny geometry (20^3 grid, 200 spots, 13 scenarios); {n_train} training and {n_test} "
                         "held-out weight settings (structure weights log-uniform in [0.1, 100], prescription "
                         "in [60, 75] Gy)"),
            "network": "9 -> 512 -> 512 -> 512 -> 200, ReLU, bfloat16 tensor-core GEMMs (FP32 accumulate), "
                       "Adam, 150 epochs of batch 128",
            "training_targets": {"solves": n_train, "eps": 1e-6, "subproblem": "cached factor",
                                 "converged": int(sum(s == 0 for s in statuses)), "seconds": round(gen_s, 2)},
            "train_s": train_s, "final_train_loss": final_loss,
            "cold_s": statistics.mean(r[0] for r in rows), "cold_iterations": statistics.mean(r[1] for r in rows),
            "learned_s": statistics.mean(r[2] for r in rows),
            "learned_iterations": statistics.mean(r[3] for r in rows),
            "speedup_learned_over_cold": statistics.mean(r[0] for r in rows) / statistics.mean(r[2] for r in rows),
            "warm_start_used": sum(r[4] for r in rows), "held_out": len(rows),
            "all_converged": all(r[7] == 0 and r[8] == 0 for r in rows),
            "max_rel_f_diff": max(abs(r[6] - r[5]) / r[5] for r in rows)}


def run_scenario_sweep(args, rpt, dev, stream, prob):
    """Time to tolerance against the number of scenarios (the paper's scenario
    scaling study, Sec. 3.1): the realistic plan restricted to its first N
    scenarios (nominal first), ADMM-BB to eps = 1e-4 and PGD to the objective
    ADMM-BB reached, both timed with CUDA events after a warm-up solve."""
    import torch

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return out, e0.elapsed_time(e1) / 1e3

    rows = []
    for N in (1, 3, 7, 13):
        if N > prob.N:
            break
        sub = prob.subset_scenarios(range(N))
        with rpt.Plan.from_problem(sub, device=dev, stream=stream.cuda_stream, autotune=1) as P:
            P.admm_bb_solve()                                        # warm-up (graph capture)
            (_, ia), ta = timed(lambda: P.admm_bb_solve())
            (_, ip), tp = timed(lambda: P.pgd_solve(f_target=ia["f"] * (1 + 1e-6), tol_rel_df=0.0,
                                                    max_iter=20000))
            rows.append({"N": N, "admm_s": ta, "admm_iterations": ia["iterations"], "admm_status": ia["status"],
                         "pgd_s": tp, "pgd_iterations": ip["iterations"], "pgd_status": ip["status"],
                         "speedup_admm_over_pgd": tp / ta})
    return rows


STRUCTURE_NAMES = {0: "body", 1: "target", 2: "oar1", 3: "oar2", 4: "oar3"}


def dvh_report(doses, labels, levels=None, names=STRUCTURE_NAMES):
    """DVH bands and dose metrics over the scenarios (the report of Sec. 3.2,
    on synthetic structures).  doses: [N, m] physical dose per scenario (Gy),
    scenario 0 nominal; labels: [m] structure of each voxel (negative: none).
    Per structure: the cumulative DVH V_s(d) = fraction of its voxels with dose
    >= d at each level d, its band (minimum and maximum over s) and the nominal
    curve; and, per scenario, the mean dose, the maximum dose, D98 and D2 (the
    doses that 98 % and 2 % of the volume receive at least: the 0.02 and 0.98
    quantiles, linearly interpolated), reported as (min, median, max) over s."""
    import numpy as np
    doses = np.asarray(doses, dtype=np.float64)
    labels = np.asarray(labels)
    if levels is None:
        levels = np.arange(0.0, 80.0 + 1e-9, 2.5)
    levels = np.asarray(levels, dtype=np.float64)
    out = {}
    for k in sorted(int(v) for v in np.unique(labels) if v >= 0):
        vol = doses[:, labels == k]
        V = (vol[:, :, None] >= levels[None, None, :]).mean(axis=1)          # [N, levels]
        mets = {"mean": vol.mean(axis=1), "max": vol.max(axis=1),
                "d98": np.quantile(vol, 0.02, axis=1), "d2": np.quantile(vol, 0.98, axis=1)}
        out[names.get(k, f"structure{k}")] = {
            "voxels": int(vol.shape[1]),
            "levels_gy": levels.tolist(),
            "dvh_nominal": V[0].tolist(), "dvh_band_min": V.min(axis=0).tolist(),
            "dvh_band_max": V.max(axis=0).tolist(),
            "metrics_gy": {key: [float(v.min()), float(np.median(v)), float(v.max())] for key, v in mets.items()}}
    return out


def run_reference(args):
    """The reference arm: the paper's CPU method (cached-Cholesky ADMM-BB with the
    scenario subproblems on worker processes) on the host cores, timed over one
    complete solve of the benchmark workload; steps = 1 whatever --steps asks
    (each solve takes about half a minute), plus labelled extras: a one-core
    sample and the CG oracle extrapolated from its first iterations."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    prob = _workload(args.seed, args.workers)
    cb = cpu_baseline(prob)
    v = cb["value"]
    extras = {}
    try:
        one = cpu_one_core_sample(prob)
        one["estimate_s"] = prob.N * (one["factor_s_per_scenario"] + cb["iterations"] * one["xupdate_s_per_scenario"])
        extras["one_core"] = one
    except Exception as e:                                   # extras never fail the arm
        extras["one_core"] = {"error": str(e)}
    try:
        extras["cg_extrapolated"] = cg_extrapolated(prob, budget_s=args.ref_budget)
    except Exception as e:
        extras["cg_extrapolated"] = {"error": str(e)}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": 1, "warmup": 0,
           "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "eps": 1e-4, "seed": args.seed,
                      "note": "one complete solve (steps 1, warmup 0) whatever --steps/--warmup ask"},
           "cpu_baseline": cb, "extras": extras,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-pgd", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the reduced-precision storage forms")
    ap.add_argument("--no-chol", action="store_true", help="skip the cached-factor subproblem solver")
    ap.add_argument("--no-variants", action="store_true", help="skip the per-scenario BB step variant")
    ap.add_argument("--ring", default=None,
                    help="entries,rows,stages of the row-pass ring (default: the autotuner's choice)")
    ap.add_argument("--ring-threads", type=int, default=0,
                    help="threads of a bundled row-pass CTA: 1024, 768 or 640 (default: the autotuner's choice)")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-sum (bitwise reproducible) variant")
    ap.add_argument("--no-tto", action="store_true", help="skip the times to the objective target (1 + 1e-4) f*")
    ap.add_argument("--dvh", action="store_true",
                    help="also report DVH bands and dose metrics over the scenarios for the solved plan")
    ap.add_argument("--scenario-sweep", action="store_true",
                    help="also time ADMM-BB and PGD on the first 1, 3, 7 and 13 scenarios of the workload")
    ap.add_argument("--learned", action="store_true",
                    help="also run the learned warm start against the cold start (tiny geometry, weight sweep)")
    ap.add_argument("--batch", nargs="?", const="large", default=None, choices=["large", "small"],
                    help="also run the batched form, one stacked plan vs one by one: 'large' = 4 plans x 49 "
                         "scenarios (~9 GB), 'small' = 8 small plans x 13 scenarios")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--max-iter", type=int, default=0,
                    help="cap ADMM iterations (short profiling runs; not a benchmark setting)")
    ap.add_argument("--row-path", type=int, default=0, help="0 default, 1 register, 2 bulk-copy ring")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven loop instead of one CUDA graph (profilers then see every launch)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = local

    from paper_2304_14568_gb300 import build as build_mod
    from paper_2304_14568_gb300 import rpt
    build_mod.build()

    t_gen = time.perf_counter()
    prob = _workload(args.seed, args.workers)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream(device=dev)
    ring_kw = dict(autotune=1)
    if args.ring:
        e_, r_, s_ = (int(v) for v in args.ring.split(","))
        ring_kw = dict(chunk_entries=e_, chunk_rows=r_, stages=s_)
    plan = rpt.Plan.from_problem(prob, device=dev, stream=stream.cuda_stream, row_path=args.row_path,
                                 ring_threads=args.ring_threads, **ring_kw)
    st = plan.stats()
    params = rpt.admm_params()          # eps_abs = eps_rel = 1e-4, defaults of the library
    if args.max_iter > 0:
        params.max_iter = args.max_iter
    if args.no_graph:
        params.use_graph = 0

    def barrier():
        if world > 1:
            dist.barrier()

    info = None
    for _ in range(args.warmup):
        _, info = plan.admm_bb_solve(params)
    sampler = ClockSampler(dev)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        x, info = plan.admm_bb_solve(params)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    ms_step = ms_total / args.steps
    ms_step = max_over_ranks(ms_step, world, f"cuda:{dev}")
    iters = statistics.mean(i["iterations"] for i in infos)
    kernels = int(sum(i["kernels"] for i in infos))

    # dominant kernel: the CG operator row pass, timed alone on the plan's stream
    rng = np.random.default_rng(1)
    plan.apply_normal(rng.uniform(0.0, 5.0, size=(prob.N, prob.n)), 0.0)
    ms_pass, bytes_pass = plan.profile_row_pass(0, reps=30)
    ms_resid, bytes_resid = plan.profile_row_pass(1, reps=10)
    peak, peak_src = _peaks()
    achieved = bytes_pass / (ms_pass * 1e-3) / 1e9
    passes_per_solve = statistics.mean(i["row_passes"] for i in infos)
    # DRAM bytes of one launch from a stored ncu capture of this kernel on this
    # workload (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the kernel
    # variant; null when no capture of the variant in use is stored
    variant = ("bundled-" + ("exact" if st["exact_sums"] else "float") +
               ("" if st["ring_threads"] in (0, 1024) else f"-{st['ring_threads']}t") if st["row_path"] == 4
               else {1: "register", 2: "ring", 3: "stream"}[st["row_path"]])
    traffic, traffic_src = None, None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            rec = json.load(open(tr_path)).get(f"kNormal f32 int32 {variant}")
            if rec:
                traffic, traffic_src = rec["bytes_per_launch"], rec["source"]
        except Exception:
            traffic = None

    out = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": prob.m, "m_active": st["m_active"], "n": prob.n,
                   "N": prob.N, "nnz": st["nnz"], "matrix_bytes": st["matrix_bytes"],
                   "eps_abs": params.eps_abs, "eps_rel": params.eps_rel,
                   "rho": infos[-1]["rho"], "l2": "inputs 1.02 GB > 129 MB L2, no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU", "seed": args.seed,
                   "ring": {"chunk_entries": st["chunk_entries"], "chunk_rows": st["chunk_rows"],
                            "stages": st["stages"], "threads": st["ring_threads"],
                            "configs_timed": st["autotuned"]}},
        "admm": {"f_rel_gap_vs_exact": (None if _golden_fstar() is None or args.seed != 0
                                        else (infos[-1]["f"] - _golden_fstar()) / _golden_fstar()),
                 "iterations": iters, "cg_iterations": statistics.mean(i["inner"] for i in infos),
                 "row_passes": passes_per_solve, "f": infos[-1]["f"], "status": infos[-1]["status"],
                 "iterations_per_s": iters / (ms_step / 1e3),
                 "solve_seconds_info": statistics.mean(i["seconds"] for i in infos)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": traffic_src or "no stored capture of this kernel variant",
                     "kernel": ("k_rowpass_tma" if st["row_path"] in (2, 4) else "k_rowpass") +
                               f"<kNormal,f32,int32,{variant}> (CG operator pass, all scenarios)",
                     "ms_per_launch": ms_pass, "bytes_per_launch": bytes_pass,
                     "bytes_note": ("bundled layout: stored block columns (4 values + 1 index, 20 B) and 64-byte "
                                    "bundle records, plus the spot vectors in and out"
                                    if st["row_path"] == 4 else "CSR: values + indices, row records, vectors"),
                     "csr_equivalent_gbs": (st["nnz"] * 8 + 4.0 * prob.N * st["m_active"] + 8.0 * prob.N * prob.n)
                                           / (ms_pass * 1e-3) / 1e9,
                     "peak_source": f"{peak_src} hbm_gbs (burst; kernel timed alone)",
                     "resid_pass_gbs": bytes_resid / (ms_resid * 1e-3) / 1e9},
        "clocks": clocks,
        "gpu_launches": kernels,
        "workload_gen_s": round(t_gen, 1),
    }

    if not args.no_exact:
        # the bundled pass with exact fixed-point sums (bitwise reproducible solves)
        with rpt.Plan.from_problem(prob, device=dev, stream=stream.cuda_stream, autotune=1, accumulate=1) as px:
            px.apply_normal(rng.uniform(0.0, 5.0, size=(prob.N, prob.n)), 0.0)
            ms_x, by_x = px.profile_row_pass(0, reps=20)
            px.admm_bb_solve(params)
            xe0 = torch.cuda.Event(enable_timing=True)
            xe1 = torch.cuda.Event(enable_timing=True)
            xe0.record(stream)
            zx, ix = px.admm_bb_solve(params)
            xe1.record(stream)
            torch.cuda.synchronize(dev)
            zx2, ix2 = px.admm_bb_solve(params)
            out["exact_sums"] = {"ms_per_pass": ms_x, "gbs": by_x / ms_x / 1e6, "frac_of_peak": by_x / ms_x / 1e6 / peak,
                                 "solve_s": xe0.elapsed_time(xe1) / 1e3, "iterations": ix["iterations"],
                                 "f": ix["f"], "repeat_solve_bitwise_equal": bool(np.array_equal(zx, zx2))}

    if not args.no_pgd:
        # PGD baseline (Sec. 2.1) to the objective ADMM-BB reached
        fa = infos[-1]["f"]
        pe0 = torch.cuda.Event(enable_timing=True)
        pe1 = torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        _, pinfo = plan.pgd_solve(f_target=fa * (1 + 1e-6), tol_rel_df=0.0, max_iter=20000)
        pe1.record(stream)
        torch.cuda.synchronize(dev)
        out["pgd"] = {"seconds": pe0.elapsed_time(pe1) / 1e3, "iterations": pinfo["iterations"],
                      "trials": pinfo["inner"], "row_passes": pinfo["row_passes"], "f": pinfo["f"],
                      "target_f": fa * (1 + 1e-6), "status": pinfo["status"],
                      "speedup_admm_over_pgd": (pe0.elapsed_time(pe1) / 1e3) / (ms_step / 1e3)}

    if not args.no_forms:
        # reduced-precision storage forms on the same workload: row-pass bandwidth
        # and time to the same tolerance; objective of their optimum on the float32 plan
        forms = {}
        for name, vf, iw in (("f32+u16", rpt.F32, 16), ("bf16+u16", rpt.BF16, 16), ("fp8+u16", rpt.FP8E4M3, 16),
                             ("bf16+int32", rpt.BF16, 32)):
            pf = rpt.Plan.from_problem(prob, device=dev, stream=stream.cuda_stream, value_format=vf,
                                       index_width=iw, row_path=args.row_path, autotune=1)
            pf.apply_normal(rng.uniform(0.0, 5.0, size=(prob.N, prob.n)), 0.0)
            ms_f, by_f = pf.profile_row_pass(0, reps=20)
            pf.admm_bb_solve(params)                     # warm-up solve
            fe0 = torch.cuda.Event(enable_timing=True)
            fe1 = torch.cuda.Event(enable_timing=True)
            fe0.record(stream)
            zf, fi = pf.admm_bb_solve(params)
            fe1.record(stream)
            torch.cuda.synchronize(dev)
            f_on_f32 = plan.objective(zf)
            sf = pf.stats()
            forms[name] = {"ring": [sf["chunk_entries"], sf["stages"], sf["ring_threads"]],
                           "ms_per_pass": ms_f, "bytes_per_pass": by_f, "gbs": by_f / ms_f / 1e6,
                           "frac_of_peak": by_f / ms_f / 1e6 / peak,
                           "solve_s": fe0.elapsed_time(fe1) / 1e3, "iterations": fi["iterations"],
                           "row_passes": fi["row_passes"],
                           "f_rel_vs_f32_optimum": (f_on_f32 - infos[-1]["f"]) / infos[-1]["f"]}
            pf.close()
        out["forms"] = forms

    if not args.no_chol:
        # the paper's subproblem solver (App. A): cached factor of B_s, x_s = B_s^{-1} c_s
        prm_c = rpt.admm_params(subproblem=rpt.SUB_CHOL)
        if args.max_iter > 0:
            prm_c.max_iter = args.max_iter
        if args.no_graph:
            prm_c.use_graph = 0
        zc, ic0 = plan.admm_bb_solve(prm_c)          # forms and inverts B_s (timed by the library)
        ce0 = torch.cuda.Event(enable_timing=True)
        ce1 = torch.cuda.Event(enable_timing=True)
        runs = []
        for _ in range(max(1, args.steps)):
            ce0.record(stream)
            zc, ic = plan.admm_bb_solve(prm_c)
            ce1.record(stream)
            torch.cuda.synchronize(dev)
            runs.append((ce0.elapsed_time(ce1) / 1e3, ic))
        fstar = _golden_fstar()
        out["cached_factor"] = {
            "setup_s": ic0["setup_seconds"], "solve_s": statistics.mean(r[0] for r in runs),
            "iterations": statistics.mean(r[1]["iterations"] for r in runs),
            "time_to_tolerance_incl_setup_s": ic0["setup_seconds"] + statistics.mean(r[0] for r in runs),
            "f": runs[-1][1]["f"], "f_rel_gap_vs_exact": None if fstar is None else (runs[-1][1]["f"] - fstar) / fstar,
            "bytes_per_iteration": 4.0 * prob.n * prob.n * prob.N,
            "note": "B_s = A~'A~ + rho/2 I formed, factored and inverted once (FP32); each iteration one dense "
                    "matrix-vector product per scenario and no sparse pass"}

    fstar = _golden_fstar() if args.seed == 0 else None
    if fstar is not None and not args.no_tto:
        # the second time-to-tolerance: until f(z) <= (1 + 1e-4) f*, with f* the exact
        # optimum (golden file); the objective is checked every iteration (one pass)
        tt = {}
        for name, prm_kw in (("admm_cg", {}), ("admm_cached_factor", {"subproblem": rpt.SUB_CHOL})):
            prm_t = rpt.admm_params(f_target=fstar * (1 + 1e-4), max_iter=20000, **prm_kw)
            plan.admm_bb_solve(prm_t)                                   # warm-up (graph, factor)
            te0 = torch.cuda.Event(enable_timing=True)
            te1 = torch.cuda.Event(enable_timing=True)
            te0.record(stream)
            _, ti = plan.admm_bb_solve(prm_t)
            te1.record(stream)
            torch.cuda.synchronize(dev)
            tt[name] = {"seconds": te0.elapsed_time(te1) / 1e3, "iterations": ti["iterations"],
                        "status": ti["status"], "f": ti["f"]}
        te0 = torch.cuda.Event(enable_timing=True)
        te1 = torch.cuda.Event(enable_timing=True)
        te0.record(stream)
        _, ti = plan.pgd_solve(f_target=fstar * (1 + 1e-4), tol_rel_df=0.0, max_iter=20000)
        te1.record(stream)
        torch.cuda.synchronize(dev)
        tt["pgd"] = {"seconds": te0.elapsed_time(te1) / 1e3, "iterations": ti["iterations"],
                     "status": ti["status"], "f": ti["f"]}
        out["time_to_objective"] = {"target": "f(z) <= (1 + 1e-4) f*", "f_star": fstar, **tt}

    if not args.no_variants:
        # per-scenario BB steps (Eq. 8 applied to each scenario's blocks) on the same plan
        prm_v = rpt.admm_params(bb_per_scenario=1)
        if args.max_iter > 0:
            prm_v.max_iter = args.max_iter
        if args.no_graph:
            prm_v.use_graph = 0
        plan.admm_bb_solve(prm_v)                          # warm-up
        runs = []
        for _ in range(max(1, min(3, args.steps))):
            ve0 = torch.cuda.Event(enable_timing=True)
            ve1 = torch.cuda.Event(enable_timing=True)
            ve0.record(stream)
            zv, iv = plan.admm_bb_solve(prm_v)
            ve1.record(stream)
            torch.cuda.synchronize(dev)
            runs.append((ve0.elapsed_time(ve1) / 1e3, iv))
        fstar = _golden_fstar()
        out["variants"] = {"bb_per_scenario": {
            "solve_s": statistics.mean(r[0] for r in runs),
            "iterations": statistics.mean(r[1]["iterations"] for r in runs),
            "row_passes": statistics.mean(r[1]["row_passes"] for r in runs),
            "status": runs[-1][1]["status"], "f": runs[-1][1]["f"],
            "f_rel_gap_vs_exact": None if fstar is None else (runs[-1][1]["f"] - fstar) / fstar}}

    if args.batch:
        out["batch"] = run_batch(args, rpt, dev, stream, peak)

    if args.learned:
        out["learned"] = run_learned(args, rpt, dev, stream)

    if args.dvh:
        _, doses = plan.objective(x, dose=True)
        out["dvh"] = dvh_report(doses, prob.labels)

    if args.scenario_sweep:
        out["scenario_sweep"] = run_scenario_sweep(args, rpt, dev, stream, prob)

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: upload + solve + result read-back
        h2d = st["matrix_bytes"] + prob.m * 16 + prob.n * 16
        e2e, e2e_it, phases = [], [], []
        for _ in range(max(2, args.steps)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            p2 = rpt.Plan.from_problem(prob, device=dev, stream=stream.cuda_stream, row_path=args.row_path,
                                       autotune=1)
            x2, i2 = p2.admm_bb_solve(params)
            torch.cuda.synchronize(dev)
            e2e.append(time.perf_counter() - t0)
            e2e_it.append(i2["iterations"])
            s2 = p2.stats()
            phases.append((s2["layout_seconds"], s2["device_seconds"], s2["autotune_seconds"], i2["seconds"]))
            p2.close()
        out["e2e"] = {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(prob.n * 8), "runs": len(e2e),
                      "iterations": e2e_it,
                      "phases_s": {k: statistics.mean(p[i] for p in phases) for i, k in
                                   enumerate(("create_host_layout", "create_device", "create_autotune", "solve"))},
                      "note": "plan_create from host CSR (validate, bundle, upload, autotune the ring) + solve + "
                              "x read-back; mean over runs (the iteration count of a solve varies by a few "
                              "percent with the order of floating-point atomics)"}

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(prob, budget_s=args.cpu_budget)
    plan.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
