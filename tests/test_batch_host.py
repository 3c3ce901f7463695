"""Stacking of several problems into one batched plan (paper_2304_14568_gb300/
csrc/batch.h, built here with the host compiler alone) against the seeded
generator's block-diagonal stacking, and the batched entry points' argument
checks, which run before any device work."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2304_14568_gb300 import rpt
from synthetic import random_problem, block_diagonal

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2304_14568_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    out = str(tmp_path_factory.mktemp("batch") / "libbatch_shim.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "batch_shim.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    L.shim_error.restype = C.c_char_p
    return L


def _structs(problems):
    built = [rpt._problem_struct(*rpt._problem_fields(p)) for p in problems]
    arr = (C.POINTER(rpt._Problem) * len(built))(*[C.pointer(pr) for pr, _ in built])
    return built, arr


def _stacked(shim):
    m, n, N, k, sw = (C.c_int32() for _ in range(5))
    shim.shim_sizes(C.byref(m), C.byref(n), C.byref(N), C.byref(k), C.byref(sw))
    out = dict(m=m.value, n=n.value, N=N.value)
    out["rp"], out["ci"], out["va"] = [], [], []
    for s in range(N.value):
        nnz = shim.shim_nnz(s)
        rp = np.empty(m.value + 1, np.int32)
        ci = np.empty(nnz, np.int32)
        va = np.empty(nnz, np.float32)
        shim.shim_scenario(s, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                           va.ctypes.data_as(C.c_void_p))
        out["rp"].append(rp)
        out["ci"].append(ci)
        out["va"].append(va)
    for i, name, ln in [(0, "w", m.value), (1, "p", m.value), (2, "lb", n.value), (3, "ub", n.value)]:
        v = np.empty(ln)
        shim.shim_vector(i, v.ctypes.data_as(C.c_void_p))
        out[name] = v
    if sw.value:
        v = np.empty(N.value)
        shim.shim_vector(4, v.ctypes.data_as(C.c_void_p))
        out["sw"] = v
    off = np.empty(k.value, np.int32)
    shim.shim_offsets(off.ctypes.data_as(C.c_void_p))
    out["off"] = off
    return out


@pytest.mark.parametrize("seed,with_sw", [(0, False), (1, True), (2, False)])
def test_stacking_matches_the_block_diagonal_definition(shim, seed, with_sw):
    rng = np.random.default_rng(seed)
    probs = [random_problem(seed * 10 + k, m=int(rng.integers(20, 90)), n=int(rng.integers(3, 30)), N=3,
                            mean_row=4.0, empty_frac=0.2, ub=float(k + 2)) for k in range(4)]
    if with_sw:
        for p in probs:
            p.scen_weight = np.array([0.2, 0.5, 0.3])
    built, arr = _structs(probs)
    assert shim.shim_stack(len(probs), arr) == rpt.OK, shim.shim_error()
    got = _stacked(shim)
    ref = block_diagonal(probs)
    assert (got["m"], got["n"], got["N"]) == (ref.m, ref.n, ref.N)
    for s in range(ref.N):
        np.testing.assert_array_equal(got["rp"][s], ref.row_ptr[s])
        np.testing.assert_array_equal(got["ci"][s], ref.col_idx[s])
        np.testing.assert_array_equal(got["va"][s], ref.val[s])
    np.testing.assert_array_equal(got["w"], ref.voxel_w)
    np.testing.assert_array_equal(got["p"], ref.presc)
    np.testing.assert_array_equal(got["lb"], ref.lb)
    np.testing.assert_array_equal(got["ub"], ref.ub)
    np.testing.assert_array_equal(got["off"], [0] + list(np.cumsum([p.n for p in probs])))
    assert ("sw" in got) == with_sw
    if with_sw:
        np.testing.assert_array_equal(got["sw"], probs[0].scen_weight)


def test_missing_bounds_take_their_defaults(shim):
    probs = [random_problem(k, m=30, n=5, N=2) for k in range(2)]
    probs[0].lb = None
    probs[1].ub = None
    built, arr = _structs(probs)
    assert shim.shim_stack(2, arr) == rpt.OK
    got = _stacked(shim)
    np.testing.assert_array_equal(got["lb"][:5], 0.0)
    assert np.all(np.isinf(got["ub"][5:]))


@pytest.mark.parametrize("change", ["N", "format", "sw_some", "sw_differ"])
def test_stacking_refuses_problems_that_do_not_stack(shim, change):
    probs = [random_problem(k, m=30, n=5, N=2) for k in range(3)]
    if change == "N":
        probs[2] = random_problem(9, m=30, n=5, N=3)
    if change in ("sw_some", "sw_differ"):
        probs[0].scen_weight = np.array([0.5, 0.5])
        if change == "sw_differ":
            probs[1].scen_weight = np.array([0.5, 0.5])
            probs[2].scen_weight = np.array([0.5, 0.25])
    fmt = [rpt.F32, rpt.F32, rpt.BF16 if change == "format" else rpt.F32]
    built = [rpt._problem_struct(*rpt._problem_fields(p), value_format=f) for p, f in zip(probs, fmt)]
    arr = (C.POINTER(rpt._Problem) * 3)(*[C.pointer(pr) for pr, _ in built])
    assert shim.shim_stack(3, arr) == rpt.EINVAL
    assert shim.shim_error()


# ---- the library's batched entry points: argument checks before any device work ----

def test_batched_create_rejects_invalid_problems_without_touching_the_device():
    probs = [random_problem(k, m=30, n=5, N=2) for k in range(2)]
    # a column of problem 1 out of its own range but inside the stacked range
    probs[1].col_idx[0] = probs[1].col_idx[0].copy()
    probs[1].col_idx[0][0] = 7
    with pytest.raises(rpt.RptError) as e:
        rpt.Plan.batched(probs)
    assert e.value.status == rpt.EINVAL
    assert b"problem 1" in rpt.lib().rpt_last_error()
    probs = [random_problem(k, m=30, n=5, N=2) for k in range(2)] + [random_problem(5, m=30, n=5, N=3)]
    with pytest.raises(rpt.RptError) as e:
        rpt.Plan.batched(probs)
    assert e.value.status == rpt.EINVAL


def test_batched_null_arguments():
    L = rpt.lib()
    h = C.c_void_p()
    assert L.rpt_plans_create_batched(0, None, None, C.byref(h)) == rpt.EINVAL
    assert L.rpt_plans_create_batched(1, None, None, C.byref(h)) == rpt.EINVAL
    k = C.c_int32()
    assert L.rpt_plan_batch_query(None, C.byref(k), None) == rpt.EINVAL
    assert L.rpt_admm_bb_solve_batched(None, None, None, None) == rpt.EINVAL
