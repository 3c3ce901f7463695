"""Thin ctypes binding of librpt (include/rpt.h).  Argument marshalling only:
every step of the solvers runs in the library's CUDA kernels.  Importing this
module fails loudly if the library has not been built; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpt.so")

OK, NOT_CONVERGED, EINVAL, ENOMEM, ECUDA, TIMEOUT, DIVERGED, EUNSUPPORTED = 0, 1, -1, -2, -3, -4, -5, -6
F32, BF16, FP8E4M3 = 0, 1, 2
SUB_CG, SUB_CHOL = 0, 1
DOSE_MAX, DOSE_MIN, DOSE_MEAN = 0, 1, 2
BB_PAPER, BB_GUARDED, BB_OFF = 0, 1, 2
Z_STD, Z_LIT = 0, 1
MAX_SPOTS = 24576

EXPORTED = [
    "rpt_admm_params_default", "rpt_pgd_params_default", "rpt_plan_create", "rpt_plan_destroy",
    "rpt_plan_query", "rpt_admm_bb_solve", "rpt_pgd_solve", "rpt_objective", "rpt_gradient",
    "rpt_apply_normal", "rpt_profile_row_pass", "rpt_normal_apply_noalloc", "rpt_state_get", "rpt_state_set", "rpt_status_string", "rpt_last_error",
    "rpt_version", "rpt_mlp_train_params_default", "rpt_mlp_create", "rpt_mlp_destroy", "rpt_mlp_param_count",
    "rpt_mlp_get_params", "rpt_mlp_set_params", "rpt_mlp_loss_grad", "rpt_mlp_train", "rpt_mlp_predict",
    "rpt_admm_bb_solve_learned", "rpt_trace_get", "rpt_plans_create_batched", "rpt_plan_batch_query",
    "rpt_admm_bb_solve_batched", "rpt_mlp_infer", "rpt_mlp_set_compute", "rpt_plan_set_weights",
    "rpt_admm_bb_solve_constrained",
]


class MlpTrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("weight_decay", C.c_double), ("seed", C.c_uint64)]


class _DoseConstraint(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_voxels", C.c_int32), ("voxels", C.POINTER(C.c_int32)),
                ("limit", C.c_double)]


class RptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Problem(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("N", C.c_int32),
                ("row_ptr", C.POINTER(C.POINTER(C.c_int32))),
                ("col_idx", C.POINTER(C.POINTER(C.c_int32))),
                ("val", C.POINTER(C.POINTER(C.c_float))),
                ("voxel_w", C.POINTER(C.c_double)), ("presc", C.POINTER(C.c_double)),
                ("scen_weight", C.POINTER(C.c_double)),
                ("lb", C.POINTER(C.c_double)), ("ub", C.POINTER(C.c_double)),
                ("value_format", C.c_int32), ("index_width", C.c_int32)]


class _DeviceOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", C.c_void_p), ("ctas_per_sm", C.c_int32),
                ("row_path", C.c_int32), ("autotune", C.c_int32), ("chunk_entries", C.c_int32),
                ("chunk_rows", C.c_int32), ("stages", C.c_int32), ("min_lanes", C.c_int32),
                ("inject_timeout", C.c_int32), ("device_mem_cap", C.c_int64), ("accumulate", C.c_int32),
                ("ring_threads", C.c_int32)]


def _device_opts(device=0, stream=None, ctas_per_sm=0, row_path=0, autotune=0, chunk_entries=0, chunk_rows=0,
                 stages=0, min_lanes=0, inject_timeout=0, device_mem_cap=0, accumulate=0, ring_threads=0):
    return _DeviceOpts(device, stream, ctas_per_sm, row_path, autotune, chunk_entries, chunk_rows, stages,
                       min_lanes, inject_timeout, device_mem_cap, accumulate, ring_threads)


class AdmmParams(C.Structure):
    _fields_ = [("rho", C.c_double), ("rho_scale", C.c_double), ("eps_abs", C.c_double),
                ("eps_rel", C.c_double), ("tol_obj", C.c_double), ("max_iter", C.c_int32),
                ("bb_mode", C.c_int32), ("bb_kappa", C.c_double), ("z_mode", C.c_int32),
                ("cg_max", C.c_int32), ("cg_theta", C.c_double), ("cg_eta0", C.c_double),
                ("cg_floor_rel", C.c_double), ("use_graph", C.c_int32), ("check_every", C.c_int32),
                ("resume", C.c_int32), ("cg_precond", C.c_int32), ("subproblem", C.c_int32),
                ("trace", C.c_int32), ("bb_per_scenario", C.c_int32), ("f_target", C.c_double)]


class PgdParams(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("tol_rel_df", C.c_double), ("f_target", C.c_double), ("max_iter", C.c_int32),
                ("max_trials", C.c_int32), ("use_graph", C.c_int32), ("reserved", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("inner", C.c_int64),
                ("row_passes", C.c_int64), ("kernels", C.c_int64), ("seconds", C.c_double), ("f", C.c_double),
                ("r_prim", C.c_double), ("r_dual", C.c_double), ("eps_prim", C.c_double),
                ("eps_dual", C.c_double), ("step", C.c_double), ("rho", C.c_double),
                ("setup_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Stats(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("N", C.c_int32), ("m_active", C.c_int32),
                ("nnz", C.c_int64), ("matrix_bytes", C.c_int64), ("value_format", C.c_int32),
                ("index_width", C.c_int32), ("row_blocks", C.c_int32), ("sm_count", C.c_int32),
                ("default_rho", C.c_double), ("const_term", C.c_double),
                ("row_path", C.c_int32), ("min_lanes", C.c_int32), ("chunk_entries", C.c_int32),
                ("chunk_rows", C.c_int32), ("stages", C.c_int32), ("autotuned", C.c_int32),
                ("autotune_ms", C.c_double), ("bundles", C.c_int64), ("block_cols", C.c_int64),
                ("bundle_fill", C.c_double), ("exact_sums", C.c_int32), ("ring_threads", C.c_int32),
                ("layout_seconds", C.c_double), ("device_seconds", C.c_double), ("autotune_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load librpt.so (in-tree build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librpt.so not built ({LIB_PATH}); run paper_2304_14568_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    dp = C.POINTER(C.c_double)
    L.rpt_admm_params_default.argtypes = [C.POINTER(AdmmParams)]
    L.rpt_admm_params_default.restype = None
    L.rpt_pgd_params_default.argtypes = [C.POINTER(PgdParams)]
    L.rpt_pgd_params_default.restype = None
    L.rpt_plan_create.argtypes = [C.POINTER(_Problem), C.POINTER(_DeviceOpts), C.POINTER(C.c_void_p)]
    L.rpt_plan_create.restype = C.c_int
    L.rpt_plan_destroy.argtypes = [C.c_void_p]
    L.rpt_plan_destroy.restype = None
    L.rpt_plan_query.argtypes = [C.c_void_p, C.POINTER(_Stats)]
    L.rpt_plan_query.restype = C.c_int
    L.rpt_admm_bb_solve.argtypes = [C.c_void_p, C.POINTER(AdmmParams), dp, dp, dp, C.POINTER(_Info)]
    L.rpt_admm_bb_solve.restype = C.c_int
    L.rpt_pgd_solve.argtypes = [C.c_void_p, C.POINTER(PgdParams), dp, dp, C.POINTER(_Info)]
    L.rpt_pgd_solve.restype = C.c_int
    L.rpt_objective.argtypes = [C.c_void_p, dp, dp, dp]
    L.rpt_objective.restype = C.c_int
    L.rpt_gradient.argtypes = [C.c_void_p, dp, dp, dp]
    L.rpt_gradient.restype = C.c_int
    L.rpt_apply_normal.argtypes = [C.c_void_p, dp, C.c_double, dp]
    L.rpt_apply_normal.restype = C.c_int
    L.rpt_profile_row_pass.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, dp]
    L.rpt_profile_row_pass.restype = C.c_int
    L.rpt_normal_apply_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    L.rpt_normal_apply_noalloc.restype = C.c_int
    L.rpt_state_get.argtypes = [C.c_void_p, dp, dp, dp]
    L.rpt_state_get.restype = C.c_int
    L.rpt_state_set.argtypes = [C.c_void_p, dp, dp, dp]
    L.rpt_state_set.restype = C.c_int
    L.rpt_status_string.argtypes = [C.c_int]
    L.rpt_status_string.restype = C.c_char_p
    L.rpt_last_error.argtypes = []
    L.rpt_last_error.restype = C.c_char_p
    L.rpt_version.argtypes = []
    L.rpt_version.restype = C.c_char_p
    fp = C.POINTER(C.c_float)
    L.rpt_mlp_train_params_default.argtypes = [C.POINTER(MlpTrainParams)]
    L.rpt_mlp_train_params_default.restype = C.c_int
    L.rpt_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32,
                                 C.POINTER(C.c_void_p)]
    L.rpt_mlp_create.restype = C.c_int
    L.rpt_mlp_destroy.argtypes = [C.c_void_p]
    L.rpt_mlp_destroy.restype = C.c_int
    L.rpt_mlp_param_count.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    L.rpt_mlp_param_count.restype = C.c_int
    L.rpt_mlp_get_params.argtypes = [C.c_void_p, fp]
    L.rpt_mlp_get_params.restype = C.c_int
    L.rpt_mlp_set_params.argtypes = [C.c_void_p, fp]
    L.rpt_mlp_set_params.restype = C.c_int
    L.rpt_mlp_loss_grad.argtypes = [C.c_void_p, fp, fp, C.c_int32, dp, fp]
    L.rpt_mlp_loss_grad.restype = C.c_int
    L.rpt_mlp_train.argtypes = [C.c_void_p, fp, fp, C.c_int32, C.POINTER(MlpTrainParams), dp]
    L.rpt_mlp_train.restype = C.c_int
    L.rpt_mlp_predict.argtypes = [C.c_void_p, fp, C.c_int32, fp]
    L.rpt_mlp_predict.restype = C.c_int
    L.rpt_mlp_infer.argtypes = [C.c_void_p, fp, fp]
    L.rpt_mlp_infer.restype = C.c_int
    L.rpt_mlp_set_compute.argtypes = [C.c_void_p, C.c_int32]
    L.rpt_mlp_set_compute.restype = C.c_int
    L.rpt_plan_set_weights.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.rpt_plan_set_weights.restype = C.c_int
    L.rpt_admm_bb_solve_constrained.argtypes = [C.c_void_p, C.POINTER(AdmmParams), C.c_int32,
                                                C.POINTER(_DoseConstraint), C.c_double, dp, dp,
                                                C.POINTER(_Info)]
    L.rpt_admm_bb_solve_constrained.restype = C.c_int
    L.rpt_admm_bb_solve_learned.argtypes = [C.c_void_p, C.c_void_p, fp, dp, C.POINTER(AdmmParams), dp,
                                            C.POINTER(_Info), C.POINTER(C.c_int32)]
    L.rpt_admm_bb_solve_learned.restype = C.c_int
    L.rpt_trace_get.argtypes = [C.c_void_p, dp, C.c_int32, C.POINTER(C.c_int32)]
    L.rpt_trace_get.restype = C.c_int
    L.rpt_plans_create_batched.argtypes = [C.c_int32, C.POINTER(C.POINTER(_Problem)), C.POINTER(_DeviceOpts),
                                           C.POINTER(C.c_void_p)]
    L.rpt_plans_create_batched.restype = C.c_int
    L.rpt_plan_batch_query.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.rpt_plan_batch_query.restype = C.c_int
    L.rpt_admm_bb_solve_batched.argtypes = [C.c_void_p, C.POINTER(AdmmParams), C.POINTER(C.POINTER(C.c_double)),
                                            C.POINTER(_Info), C.POINTER(_Info)]
    L.rpt_admm_bb_solve_batched.restype = C.c_int
    _lib = L
    return L


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(a, dtype, size, name, at_least=False):
    """a as a contiguous flat array of `dtype`, or ValueError if it does not
    hold `size` elements (at least `size` with at_least).  The C ABI takes
    plain pointers and reads exactly the documented counts, so every length is
    checked here, before the call."""
    v = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
    if (v.size < size) if at_least else (v.size != size):
        raise ValueError(f"{name}: {v.size} elements, need {'at least ' if at_least else ''}{size}")
    return v


def _rows(a, dtype, cols, name):
    """a as a contiguous [k, cols] array of `dtype` (one row allowed as 1-D)."""
    v = np.ascontiguousarray(np.atleast_2d(a), dtype=dtype)
    if v.ndim != 2 or v.shape[1] != cols:
        raise ValueError(f"{name}: shape {v.shape}, need [k, {cols}]")
    return v


def _check(rc, allow=(OK,)):
    if rc not in allow:
        raise RptError(rc, lib().rpt_last_error().decode() or lib().rpt_status_string(rc).decode())
    return rc


def admm_params(**kw) -> AdmmParams:
    p = AdmmParams()
    lib().rpt_admm_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def pgd_params(**kw) -> PgdParams:
    p = PgdParams()
    lib().rpt_pgd_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _problem_struct(m, n, N, row_ptr, col_idx, val, voxel_w, presc, scen_weight=None, lb=None, ub=None,
                    value_format=F32, index_width=32):
    """An rpt_problem over contiguous copies of the arrays, after checking every
    length; returns (struct, arrays to keep alive while the struct is used)."""
    m, n, N = int(m), int(n), int(N)
    if m < 1 or n < 1 or N < 1:
        raise ValueError("m, n and N must be >= 1")
    if not (len(row_ptr) == len(col_idx) == len(val) == N):
        raise ValueError("row_ptr, col_idx and val need one array per scenario")
    rp = [_vec(a, np.int32, m + 1, f"row_ptr[{s}]") for s, a in enumerate(row_ptr)]
    nnz = [max(int(a[-1]), 0) for a in rp]
    ci = [_vec(a, np.int32, k, f"col_idx[{s}]", at_least=True) for s, (a, k) in enumerate(zip(col_idx, nnz))]
    va = [_vec(a, np.float32, k, f"val[{s}]", at_least=True) for s, (a, k) in enumerate(zip(val, nnz))]
    w = _vec(voxel_w, np.float64, m, "voxel_w")
    p = _vec(presc, np.float64, m, "presc")
    sw = None if scen_weight is None else _vec(scen_weight, np.float64, N, "scen_weight")
    lbv = None if lb is None else _vec(lb, np.float64, n, "lb")
    ubv = None if ub is None else _vec(ub, np.float64, n, "ub")
    RP = (C.POINTER(C.c_int32) * N)(*[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in rp])
    CI = (C.POINTER(C.c_int32) * N)(*[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in ci])
    VA = (C.POINTER(C.c_float) * N)(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in va])
    pr = _Problem(m, n, N, RP, CI, VA, _dptr(w), _dptr(p), _dptr(sw), _dptr(lbv), _dptr(ubv),
                  value_format, index_width)
    return pr, (rp, ci, va, w, p, sw, lbv, ubv, RP, CI, VA)


def _problem_fields(prob):
    return (prob.m, prob.n, prob.N, prob.row_ptr, prob.col_idx, prob.val, prob.voxel_w, prob.presc,
            prob.scen_weight, prob.lb, prob.ub)


class Plan:
    """A device-resident plan (rpt_plan_create / rpt_plan_destroy)."""

    def __init__(self, m, n, N, row_ptr, col_idx, val, voxel_w, presc, scen_weight=None,
                 lb=None, ub=None, value_format=F32, index_width=32, **device_opts):
        """device_opts: the fields of rpt_device_opts (device, stream, ctas_per_sm,
        row_path, autotune, chunk_entries, chunk_rows, stages, min_lanes,
        inject_timeout, device_mem_cap, accumulate)."""
        L = lib()
        m, n, N = int(m), int(n), int(N)
        pr, _keep = _problem_struct(m, n, N, row_ptr, col_idx, val, voxel_w, presc, scen_weight, lb, ub,
                                    value_format, index_width)
        opts = _device_opts(**device_opts)
        h = C.c_void_p()
        _check(L.rpt_plan_create(C.byref(pr), C.byref(opts), C.byref(h)))
        self._h = h
        self.m, self.n, self.N = m, n, N

    @classmethod
    def from_problem(cls, prob, **kw):
        """Build from any object with the fields of the C struct rpt_problem."""
        return cls(*_problem_fields(prob), **kw)

    @classmethod
    def batched(cls, problems, value_format=F32, index_width=32, **device_opts):
        """One plan holding several problems, solved side by side (rpt_plans_create_batched)."""
        L = lib()
        built = [_problem_struct(*_problem_fields(p), value_format=value_format, index_width=index_width)
                 for p in problems]
        arr = (C.POINTER(_Problem) * len(built))(*[C.pointer(pr) for pr, _ in built])
        opts = _device_opts(**device_opts)
        h = C.c_void_p()
        _check(L.rpt_plans_create_batched(len(built), arr, C.byref(opts), C.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        st = self.stats()
        self.m, self.n, self.N = st["m"], st["n"], st["N"]
        return self

    def set_weights(self, voxel_w, presc):
        """New voxel weights and prescription for the same matrices (rpt_plan_set_weights)."""
        w = _vec(voxel_w, np.float64, self.m, "voxel_w")
        p = _vec(presc, np.float64, self.m, "presc")
        _check(lib().rpt_plan_set_weights(self._h, _dptr(w), _dptr(p)))

    def batch_offsets(self):
        """Spot ranges of the plan's problems: offsets [n_plans + 1] (rpt_plan_batch_query)."""
        k = C.c_int32()
        _check(lib().rpt_plan_batch_query(self._h, C.byref(k), None))
        off = np.empty(k.value + 1, dtype=np.int32)
        _check(lib().rpt_plan_batch_query(self._h, C.byref(k), off.ctypes.data_as(C.POINTER(C.c_int32))))
        return off

    def admm_bb_solve_batched(self, params: AdmmParams | None = None, **kw):
        """ADMM-BB on every problem of the plan, each with its own penalty, BB
        step and stop; returns ([x_k per problem], info of the whole solve,
        [info per problem])."""
        prm = params if params is not None else admm_params(**kw)
        off = self.batch_offsets()
        xs = [np.empty(int(off[k + 1] - off[k])) for k in range(len(off) - 1)]
        ptrs = (C.POINTER(C.c_double) * len(xs))(*[_dptr(x) for x in xs])
        info = _Info()
        per = (_Info * len(xs))()
        rc = lib().rpt_admm_bb_solve_batched(self._h, C.byref(prm), ptrs, C.byref(info), per)
        _check(rc, allow=(OK, NOT_CONVERGED, DIVERGED))
        return xs, info.as_dict(), [p.as_dict() for p in per]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rpt_plan_destroy(self._h)
            self._h = None

    plan_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        s = _Stats()
        _check(lib().rpt_plan_query(self._h, C.byref(s)))
        return s.as_dict()

    def admm_bb_solve(self, params: AdmmParams | None = None, z0=None, y0=None, **kw):
        prm = params if params is not None else admm_params(**kw)
        x = np.empty(self.n)
        z0a = None if z0 is None else _vec(z0, np.float64, self.n, "z0")
        y0a = None if y0 is None else _vec(y0, np.float64, self.N * self.n, "y0")
        info = _Info()
        rc = lib().rpt_admm_bb_solve(self._h, C.byref(prm), _dptr(z0a), _dptr(y0a), _dptr(x), C.byref(info))
        _check(rc, allow=(OK, NOT_CONVERGED))
        return x, info.as_dict()

    def admm_bb_solve_constrained(self, constraints, sigma=0.0, params: AdmmParams | None = None, **kw):
        """ADMM-BB with dose constraints (rpt_admm_bb_solve_constrained).  constraints:
        a list of (kind, voxels, limit) with kind DOSE_MAX / DOSE_MIN / DOSE_MEAN.
        Returns (x, mu [N][K], info)."""
        prm = params if params is not None else admm_params(**kw)
        keep, arr = [], (_DoseConstraint * max(1, len(constraints)))()
        K = 0
        for i, (kind, voxels, limit) in enumerate(constraints):
            v = np.ascontiguousarray(np.asarray(voxels, dtype=np.int32))
            keep.append(v)
            arr[i] = _DoseConstraint(int(kind), int(v.size), v.ctypes.data_as(C.POINTER(C.c_int32)), float(limit))
            K += 1 if int(kind) == DOSE_MEAN else int(v.size)
        x = np.empty(self.n)
        mu = np.empty(max(1, self.N * K))
        info = _Info()
        rc = lib().rpt_admm_bb_solve_constrained(self._h, C.byref(prm), len(constraints), arr, float(sigma),
                                                 _dptr(x), _dptr(mu), C.byref(info))
        _check(rc, allow=(OK, NOT_CONVERGED))
        return x, mu[:self.N * K].reshape(self.N, K), info.as_dict()

    def pgd_solve(self, params: PgdParams | None = None, x0=None, **kw):
        prm = params if params is not None else pgd_params(**kw)
        x = np.empty(self.n)
        x0a = None if x0 is None else _vec(x0, np.float64, self.n, "x0")
        info = _Info()
        rc = lib().rpt_pgd_solve(self._h, C.byref(prm), _dptr(x0a), _dptr(x), C.byref(info))
        _check(rc, allow=(OK, NOT_CONVERGED))
        return x, info.as_dict()

    def objective(self, x, dose=False):
        xa = _vec(x, np.float64, self.n, "x")
        f = C.c_double()
        d = np.empty(self.N * self.m) if dose else None
        _check(lib().rpt_objective(self._h, _dptr(xa), C.byref(f), _dptr(d)))
        return (f.value, d.reshape(self.N, self.m)) if dose else f.value

    def gradient(self, x):
        xa = _vec(x, np.float64, self.n, "x")
        g = np.empty(self.n)
        f = C.c_double()
        _check(lib().rpt_gradient(self._h, _dptr(xa), _dptr(g), C.byref(f)))
        return g, f.value

    def apply_normal(self, v, rho=0.0):
        va = _vec(v, np.float64, self.N * self.n, "v")
        u = np.empty(self.N * self.n)
        _check(lib().rpt_apply_normal(self._h, _dptr(va), float(rho), _dptr(u)))
        return u.reshape(self.N, self.n)

    def profile_row_pass(self, mode=0, reps=20):
        """(milliseconds per launch, algorithmic bytes per launch) of the row pass."""
        ms = C.c_double()
        by = C.c_double()
        _check(lib().rpt_profile_row_pass(self._h, int(mode), int(reps), C.byref(ms), C.byref(by)))
        return ms.value, by.value

    TRACE_FIELDS = ("iteration", "seconds", "r_prim", "r_dual", "eps_prim", "eps_dual", "step", "cg_steps")

    def trace(self):
        """Per-iteration record of the last solve run with trace=1, as an array
        [iterations][8] with columns TRACE_FIELDS."""
        cnt = C.c_int32()
        _check(lib().rpt_trace_get(self._h, None, 0, C.byref(cnt)))
        out = np.empty((cnt.value, 8))
        if cnt.value:
            _check(lib().rpt_trace_get(self._h, _dptr(out), cnt.value, C.byref(cnt)))
        return out

    def state_get(self):
        z = np.empty(self.n)
        x = np.empty(self.N * self.n)
        y = np.empty(self.N * self.n)
        _check(lib().rpt_state_get(self._h, _dptr(z), _dptr(x), _dptr(y)))
        return z, x.reshape(self.N, self.n), y.reshape(self.N, self.n)

    def state_set(self, z, x, y):
        za = _vec(z, np.float64, self.n, "z")
        xa = _vec(x, np.float64, self.N * self.n, "x")
        ya = _vec(y, np.float64, self.N * self.n, "y")
        _check(lib().rpt_state_set(self._h, _dptr(za), _dptr(xa), _dptr(ya)))


def plan_create(prob, **kw) -> Plan:
    return Plan.from_problem(prob, **kw)


def normal_apply_noalloc(m, n, row_ptr_dev, col_idx_dev, val_dev, row_w_dev, v_dev, rho, u_dev, stream=None):
    """u = A^T diag(w) A v + (rho/2) v from device arrays (integer device
    addresses), with no device allocation.  Asynchronous on `stream`."""
    _check(lib().rpt_normal_apply_noalloc(int(m), int(n), row_ptr_dev, col_idx_dev, val_dev, row_w_dev, v_dev,
                                          float(rho), u_dev, stream))


def _fptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def mlp_train_params(**kw) -> MlpTrainParams:
    tp = MlpTrainParams()
    _check(lib().rpt_mlp_train_params_default(C.byref(tp)))
    for k, v in kw.items():
        setattr(tp, k, v)
    return tp


class Mlp:
    """Learned warm-start network (rpt_mlp_*)."""

    def __init__(self, n_in, n_hidden, n_hidden_layers, n_out, seed=0, device=0, compute=None):
        """compute: BF16 (tensor cores, the library default) or F32 (CUDA cores)."""
        h = C.c_void_p()
        _check(lib().rpt_mlp_create(int(n_in), int(n_hidden), int(n_hidden_layers), int(n_out), int(seed),
                                    int(device), C.byref(h)))
        self._h = h
        if compute is not None:
            _check(lib().rpt_mlp_set_compute(h, int(compute)))
        self.n_in, self.n_out = int(n_in), int(n_out)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rpt_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def param_count(self) -> int:
        c = C.c_int64()
        _check(lib().rpt_mlp_param_count(self._h, C.byref(c)))
        return c.value

    def get_params(self):
        p = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().rpt_mlp_get_params(self._h, _fptr(p)))
        return p

    def set_params(self, p):
        pa = _vec(p, np.float32, self.param_count(), "params")
        _check(lib().rpt_mlp_set_params(self._h, _fptr(pa)))

    def loss_grad(self, X, Y):
        Xa = _rows(X, np.float32, self.n_in, "X")
        Ya = _rows(Y, np.float32, self.n_out, "Y")
        if Ya.shape[0] != Xa.shape[0]:
            raise ValueError("X and Y need the same number of rows")
        loss = C.c_double()
        g = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().rpt_mlp_loss_grad(self._h, _fptr(Xa), _fptr(Ya), int(Xa.shape[0]), C.byref(loss), _fptr(g)))
        return loss.value, g

    def train(self, X, Y, params: MlpTrainParams | None = None, **kw):
        tp = params if params is not None else mlp_train_params(**kw)
        Xa = _rows(X, np.float32, self.n_in, "X")
        Ya = _rows(Y, np.float32, self.n_out, "Y")
        if Ya.shape[0] != Xa.shape[0]:
            raise ValueError("X and Y need the same number of rows")
        loss = C.c_double()
        _check(lib().rpt_mlp_train(self._h, _fptr(Xa), _fptr(Ya), int(Xa.shape[0]), C.byref(tp), C.byref(loss)))
        return loss.value

    def predict(self, X):
        Xa = _rows(X, np.float32, self.n_in, "X")
        Y = np.empty((Xa.shape[0], self.n_out), dtype=np.float32)
        _check(lib().rpt_mlp_predict(self._h, _fptr(Xa), int(Xa.shape[0]), _fptr(Y)))
        return Y


def mlp_infer(mlp, features):
    """The network's output for one feature vector (rpt_mlp_infer)."""
    f = _vec(features, np.float32, mlp.n_in, "features")
    out = np.empty(mlp.n_out, dtype=np.float32)
    _check(lib().rpt_mlp_infer(mlp._h, _fptr(f), _fptr(out)))
    return out


def admm_bb_solve_learned(plan, mlp, features, zscale, params: AdmmParams | None = None, **kw):
    """ADMM-BB warm-started by the network (cold-start fallback); returns
    (x, info, used_warm_start)."""
    prm = params if params is not None else admm_params(**kw)
    f = _vec(features, np.float32, mlp.n_in, "features")
    zs = _vec(zscale, np.float64, plan.n, "zscale")
    x = np.empty(plan.n)
    info = _Info()
    used = C.c_int32()
    rc = lib().rpt_admm_bb_solve_learned(plan._h, mlp._h, _fptr(f), _dptr(zs), C.byref(prm), _dptr(x),
                                         C.byref(info), C.byref(used))
    _check(rc, allow=(OK, NOT_CONVERGED))
    return x, info.as_dict(), bool(used.value)


def version() -> str:
    return lib().rpt_version().decode()


def inf():
    return math.inf
