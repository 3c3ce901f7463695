"""The C ABI without a GPU: the library builds and loads, exports every symbol
include/rpt.h declares, the binding's struct layouts match the C compiler's, and
argument validation rejects bad problems before any device call."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2304_14568_gb300 import build as build_mod
from paper_2304_14568_gb300 import rpt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rpt.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return rpt.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpt_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", rpt.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rpt_[a-z0-9_]+)", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    assert set(rpt.EXPORTED) == set(declared)
    for f in declared:
        getattr(lib, f)


def test_struct_layouts_match_c_compiler(lib):
    structs = {
        "rpt_problem": rpt._Problem, "rpt_device_opts": rpt._DeviceOpts,
        "rpt_admm_params": rpt.AdmmParams, "rpt_pgd_params": rpt.PgdParams,
        "rpt_solve_info": rpt._Info, "rpt_plan_stats": rpt._Stats,
        "rpt_mlp_train_params": rpt.MlpTrainParams, "rpt_dose_constraint": rpt._DoseConstraint,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rpt.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_defaults_and_status_strings(lib):
    p = rpt.admm_params()
    assert p.eps_abs == 1e-4 and p.eps_rel == 1e-4 and p.bb_mode == rpt.BB_PAPER
    assert p.z_mode == rpt.Z_STD and p.max_iter > 0 and p.use_graph == 1
    assert np.isinf(p.tol_obj)
    q = rpt.pgd_params()
    assert 0 < q.beta < 1 and 0 < q.gamma < 1 and q.max_trials >= 1
    for s in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.rpt_status_string(s)
    assert b"sm_103a" in lib.rpt_version()


def _tiny():
    rp = [np.array([0, 2, 3], np.int32)]
    ci = [np.array([0, 1, 1], np.int32)]
    va = [np.array([1.0, 0.5, 2.0], np.float32)]
    return dict(m=2, n=2, N=1, row_ptr=rp, col_idx=ci, val=va,
                voxel_w=np.array([1.0, 2.0]), presc=np.array([1.0, 0.0]))


@pytest.mark.parametrize("mutate,code", [
    (lambda d: d["col_idx"][0].__setitem__(1, 5), rpt.EINVAL),            # column out of range
    (lambda d: d["col_idx"][0].__setitem__(1, 0), rpt.EINVAL),            # not strictly increasing
    (lambda d: d["val"][0].__setitem__(0, np.nan), rpt.EINVAL),           # NaN value
    (lambda d: d["val"][0].__setitem__(0, -1.0), rpt.EINVAL),             # negative dose influence
    (lambda d: d["row_ptr"][0].__setitem__(1, 4), rpt.EINVAL),            # decreasing row_ptr
    (lambda d: d["voxel_w"].__setitem__(0, np.inf), rpt.EINVAL),          # non-finite weight
    (lambda d: d["presc"].__setitem__(1, -2.0), rpt.EINVAL),              # negative prescription
    (lambda d: d.update(lb=np.array([1.0, 0.0]), ub=np.array([0.5, 1.0])), rpt.EINVAL),   # lb > ub
    (lambda d: d.update(n=rpt.MAX_SPOTS + 1), rpt.EUNSUPPORTED),
    (lambda d: d.update(value_format=7), rpt.EUNSUPPORTED),
])
def test_plan_create_rejects_bad_input_without_touching_the_device(lib, mutate, code):
    d = _tiny()
    mutate(d)
    with pytest.raises(rpt.RptError) as ei:
        rpt.Plan(**d)
    assert ei.value.status == code
    assert lib.rpt_last_error()


@pytest.mark.parametrize("opt", [dict(row_path=5), dict(accumulate=3), dict(ring_threads=512)])
def test_plan_create_rejects_bad_options_without_touching_the_device(lib, opt):
    with pytest.raises(rpt.RptError) as ei:
        rpt.Plan(**_tiny(), **opt)
    assert ei.value.status == rpt.EINVAL
    assert b"ring_threads" in lib.rpt_last_error()


def test_null_arguments_are_errors(lib):
    assert lib.rpt_plan_create(None, None, None) == rpt.EINVAL
    assert lib.rpt_admm_bb_solve(None, None, None, None, None, None) == rpt.EINVAL
    assert lib.rpt_pgd_solve(None, None, None, None, None) == rpt.EINVAL
    assert lib.rpt_objective(None, None, None, None) == rpt.EINVAL
    assert lib.rpt_mlp_infer(None, None, None) == rpt.EINVAL
    lib.rpt_plan_destroy(None)   # accepted


@pytest.mark.parametrize("mutate", [
    lambda d: d["row_ptr"].__setitem__(0, np.array([0, 2], np.int32)),         # m + 1 entries needed
    lambda d: d["col_idx"].__setitem__(0, np.array([0, 1], np.int32)),         # fewer than row_ptr[m]
    lambda d: d["val"].__setitem__(0, np.array([1.0], np.float32)),
    lambda d: d.update(voxel_w=np.array([1.0])),                               # m weights needed
    lambda d: d.update(presc=np.array([1.0, 0.0, 3.0])),
    lambda d: d.update(scen_weight=np.array([1.0, 1.0])),                      # N weights needed
    lambda d: d.update(lb=np.zeros(3)),                                        # n bounds needed
    lambda d: d.update(N=2),                                                   # one array per scenario
])
def test_binding_checks_array_lengths_before_the_call(lib, mutate):
    """The C ABI reads exactly the documented counts through plain pointers, so
    the binding refuses arrays of the wrong length before calling it."""
    d = _tiny()
    mutate(d)
    with pytest.raises(ValueError):
        rpt.Plan(**d)


def test_vector_helper_shapes():
    v = rpt._vec([[1, 2], [3, 4]], np.float64, 4, "x")
    assert v.shape == (4,) and v.dtype == np.float64 and v.flags.c_contiguous
    with pytest.raises(ValueError):
        rpt._vec(np.zeros(3), np.float64, 4, "x")
    assert rpt._vec(np.zeros(5), np.float32, 4, "x", at_least=True).size == 5
    with pytest.raises(ValueError):
        rpt._vec(np.zeros(3), np.float32, 4, "x", at_least=True)
    assert rpt._rows(np.zeros(9), np.float32, 9, "X").shape == (1, 9)
    with pytest.raises(ValueError):
        rpt._rows(np.zeros((4, 8)), np.float32, 9, "X")
