"""The units of a batched plan (paper_2304_14568_gb300/csrc/batch.h, built here
with the host compiler alone) against their definition written out below, and
the batched entry points' argument checks, which run before any device work.

Definition.  Problems k = 0 .. G-1 with the same scenario count Ns; voxel rows
numbered one problem after another (problem k from row_off[k]); unit
u = k * Ns + s holds problem k's scenario-s rows at their shifted row numbers,
no entry in another problem's rows, the problem's own spot indices, and
n = max_k n_k spots per unit; per problem a box of n spots whose extra spots
(j >= n_k) are held at lb = ub = 0; scenario weights per unit from the
problem's own (1 when it has none)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2304_14568_gb300 import rpt
from synthetic import random_problem

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


def _units(shim):
    m, n, U, G, Ns = (C.c_int32() for _ in range(5))
    shim.shim_sizes(C.byref(m), C.byref(n), C.byref(U), C.byref(G), C.byref(Ns))
    out = dict(m=m.value, n=n.value, U=U.value, G=G.value, Ns=Ns.value, rp=[], ci=[], va=[])
    for u in range(U.value):
        nnz = shim.shim_nnz(u)
        rp = np.empty(m.value + 1, np.int32)
        ci = np.empty(max(nnz, 1), np.int32)
        va = np.empty(max(nnz, 1), np.float32)
        shim.shim_unit(u, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                       va.ctypes.data_as(C.c_void_p))
        out["rp"].append(rp)
        out["ci"].append(ci[:nnz])
        out["va"].append(va[:nnz])
    lens = [m.value, m.value, G.value * n.value, G.value * n.value, U.value]
    for i, name in enumerate(["w", "p", "lb", "ub", "sw"]):
        v = np.empty(lens[i])
        shim.shim_vector(i, v.ctypes.data_as(C.c_void_p))
        out[name] = v
    for i, name, ln in [(0, "row_off", G.value + 1), (1, "col_off", G.value + 1), (2, "n_g", G.value)]:
        v = np.empty(ln, np.int32)
        shim.shim_offsets(i, v.ctypes.data_as(C.c_void_p))
        out[name] = v
    return out


def _expected(probs):
    """The definition in the module docstring, written out with numpy."""
    G, Ns = len(probs), probs[0].N
    M = sum(p.m for p in probs)
    n = max(p.n for p in probs)
    row_off = np.concatenate([[0], np.cumsum([p.m for p in probs])])
    rp, ci, va = [], [], []
    for k, p in enumerate(probs):
        for s in range(Ns):
            r = np.zeros(M + 1, np.int64)
            q = np.asarray(p.row_ptr[s], np.int64)
            r[row_off[k]:row_off[k] + p.m + 1] = q
            r[row_off[k] + p.m + 1:] = q[-1]
            rp.append(r)
            ci.append(np.asarray(p.col_idx[s]))
            va.append(np.asarray(p.val[s], np.float32))
    lb = np.zeros((G, n))
    ub = np.zeros((G, n))
    sw = np.ones(G * Ns)
    for k, p in enumerate(probs):
        lb[k, :p.n] = 0.0 if p.lb is None else p.lb
        ub[k, :p.n] = np.inf if p.ub is None else p.ub
        if p.scen_weight is not None:
            sw[k * Ns:(k + 1) * Ns] = p.scen_weight
    return dict(m=M, n=n, U=G * Ns, G=G, Ns=Ns, rp=rp, ci=ci, va=va,
                w=np.concatenate([p.voxel_w for p in probs]), p=np.concatenate([p.presc for p in probs]),
                lb=lb.ravel(), ub=ub.ravel(), sw=sw, row_off=row_off,
                col_off=np.concatenate([[0], np.cumsum([p.n for p in probs])]), n_g=[p.n for p in probs])


@pytest.mark.parametrize("seed,with_sw", [(0, False), (1, True), (2, False)])
def test_units_match_their_definition(shim, seed, with_sw):
    rng = np.random.default_rng(seed)
    probs = [random_problem(seed * 10 + k, m=int(rng.integers(20, 90)), n=int(rng.integers(3, 30)), N=3,
                            mean_row=4.0, empty_frac=0.2, ub=float(k + 2)) for k in range(4)]
    if with_sw:
        for k, p in enumerate(probs):
            p.scen_weight = np.array([0.2, 0.5, 0.3]) if k % 2 == 0 else None
    built, arr = _structs(probs)
    assert shim.shim_stack(len(probs), arr) == rpt.OK, shim.shim_error()
    got, ref = _units(shim), _expected(probs)
    for key in ("m", "n", "U", "G", "Ns"):
        assert got[key] == ref[key], key
    for u in range(ref["U"]):
        np.testing.assert_array_equal(got["rp"][u], ref["rp"][u])
        np.testing.assert_array_equal(got["ci"][u], ref["ci"][u])
        np.testing.assert_array_equal(got["va"][u], ref["va"][u])
    for key in ("w", "p", "lb", "ub", "sw", "row_off", "col_off", "n_g"):
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)


def test_missing_bounds_take_their_defaults(shim):
    probs = [random_problem(k, m=30, n=5 + k, N=2) for k in range(2)]
    probs[0].lb = None
    probs[1].ub = None
    built, arr = _structs(probs)
    assert shim.shim_stack(2, arr) == rpt.OK
    got = _units(shim)
    assert got["n"] == 6
    lb, ub = got["lb"].reshape(2, 6), got["ub"].reshape(2, 6)
    np.testing.assert_array_equal(lb[0, :5], 0.0)
    assert np.all(np.isinf(ub[1, :6]))
    assert lb[0, 5] == ub[0, 5] == 0.0   # problem 0 has 5 spots: the sixth is held at 0


@pytest.mark.parametrize("change", ["N", "format", "too_many"])
def test_stacking_refuses_problems_that_do_not_stack(shim, change):
    count = 65 if change == "too_many" else 3
    probs = [random_problem(k % 3, m=30, n=5, N=2) for k in range(count)]
    if change == "N":
        probs[2] = random_problem(9, m=30, n=5, N=3)
    fmt = [rpt.F32] * count
    if change == "format":
        fmt[2] = rpt.BF16
    built = [rpt._problem_struct(*rpt._problem_fields(p), value_format=f) for p, f in zip(probs, fmt)]
    arr = (C.POINTER(rpt._Problem) * count)(*[C.pointer(pr) for pr, _ in built])
    assert shim.shim_stack(count, arr) == (rpt.EUNSUPPORTED if change == "too_many" else rpt.EINVAL)
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
    assert L.rpt_admm_bb_solve_batched(None, None, None, None, None) == rpt.EINVAL
