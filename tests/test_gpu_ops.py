"""Row-pass operators through the C ABI against the float64 oracle, element by
element (App. A operator B_s, Eq. 4 gradient, Eq. 1-2 objective, doses).

Tolerance: each result is a float32 dot of <= L terms followed by a float32
scatter of <= K terms, so |gpu - exact| <= (L + K + 8) eps32 * (same sum with
absolute values), evaluated per element by the oracle on |A|, |v|, |p|."""
import numpy as np
import pytest
import scipy.sparse as sp

from synthetic import random_problem, config_tiny_plain
from oracle import Weighted
from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound

pytestmark = pytest.mark.gpu

CASES = {
    "ragged": dict(seed=1, m=500, n=70, N=3, mean_row=12.0, scen_weight=True),
    "long_rows": dict(seed=2, m=300, n=300, N=2, mean_row=40.0, long_rows=5),
    "one_spot": dict(seed=3, m=200, n=1, N=2, mean_row=1.0),
    "n33_N1": dict(seed=4, m=257, n=33, N=1, mean_row=9.0, empty_frac=0.4),
    "many_empty": dict(seed=5, m=2000, n=130, N=4, mean_row=6.0, empty_frac=0.9, zero_w_frac=0.2),
    "dense_1200": dict(seed=6, m=150, n=1200, N=2, mean_row=25.0, long_rows=3),   # rows past 512 entries
}


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


# row-pass implementations: register-direct loads, the bulk-copy ring, the ring
# with tiny stages (many chunks per segment, stage wrap-around, segment
# switches), the streaming path, and the streaming path with tiny chunks (many
# chunk hand-overs, class changes inside a warp's run, one-row chunks)
PATHS = {
    "reg": (1, {}),
    "tma": (2, {}),
    "tma_small": (2, {"RPT_TMA_CMAX": "1280", "RPT_TMA_RMAX": "8", "RPT_TMA_STAGES": "2"}),
    "stream": (3, {}),
    "stream_small": (3, {"RPT_STR_CMAX": "64", "RPT_STR_RMAX": "3"}),
}


@pytest.fixture(params=sorted(PATHS))
def path(request, monkeypatch):
    row_path, env = PATHS[request.param]
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    return row_path


def _abs_W(W):
    class A:
        pass
    a = A()
    a.At = [abs(M) for M in W.At]
    a.pt = [np.abs(p) for p in W.pt]
    return a


@pytest.mark.parametrize("case", sorted(CASES))
def test_apply_normal(rpt, case, path):
    prob = random_problem(**CASES[case])
    W = Weighted(prob)
    rng = np.random.default_rng(11)
    V = rng.normal(size=(prob.N, prob.n)) * rng.uniform(0.1, 5.0, size=(prob.N, prob.n))
    rho = 3.7
    with plan_of(rpt, prob, row_path=path) as P:
        U = P.apply_normal(V, rho)
    Wa = _abs_W(W)
    k = fp32_op_bound(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], rho)
        mag = Wa.At[s].T @ (Wa.At[s] @ np.abs(V[s])) + 0.5 * rho * np.abs(V[s])
        err = np.abs(U[s] - ref)
        assert np.all(err <= k * mag + 1e-300), (case, s, float((err / np.maximum(mag, 1e-300)).max()))


@pytest.mark.parametrize("case", sorted(CASES))
def test_gradient_and_objective(rpt, case, path):
    prob = random_problem(**CASES[case])
    W = Weighted(prob)
    rng = np.random.default_rng(12)
    x = rng.uniform(0.0, 4.0, size=prob.n)
    with plan_of(rpt, prob, row_path=path) as P:
        g, f = P.gradient(x)
        f2 = P.objective(x)
    Wa = _abs_W(W)
    k = fp32_op_bound(prob)
    mag = np.zeros(prob.n)
    for s in range(prob.N):
        mag += 2.0 * (Wa.At[s].T @ (Wa.At[s] @ np.abs(x) + Wa.pt[s]))
    ref = W.grad(x)
    assert np.all(np.abs(g - ref) <= k * mag + 1e-300), float((np.abs(g - ref) / mag).max())
    fref = W.f(x)
    # f = sum of squares of float32 residuals: relative error <= 2 (L + 8) eps32 * sum(w (|a||x| + p)^2) / f
    fmag = sum(float(np.sum((Wa.At[s] @ np.abs(x) + Wa.pt[s]) ** 2)) for s in range(prob.N))
    assert abs(f - fref) <= 2 * k * fmag
    assert abs(f2 - fref) <= 2 * k * fmag


@pytest.mark.parametrize("case", ["ragged", "many_empty"])
def test_doses(rpt, case, path):
    prob = random_problem(**CASES[case])
    W = Weighted(prob)
    x = np.random.default_rng(13).uniform(0.0, 4.0, size=prob.n)
    with plan_of(rpt, prob, row_path=path) as P:
        f, D = P.objective(x, dose=True)
    k = fp32_op_bound(prob)
    for s in range(prob.N):
        ref = W.dose(s, x)
        mag = abs(W.A[s]) @ np.abs(x)
        assert np.all(np.abs(D[s] - ref) <= k * mag + 1e-300)


def test_tiny_plain_operators(rpt):
    prob = config_tiny_plain(0)
    W = Weighted(prob)
    rng = np.random.default_rng(5)
    V = rng.uniform(0, 5, size=(prob.N, prob.n))
    with plan_of(rpt, prob) as P:
        st = P.stats()
        U = P.apply_normal(V, 0.0)
        g, f = P.gradient(V[0])
    assert st["nnz"] == sum(prob.nnz()) and st["m_active"] <= prob.m
    assert st["row_blocks"] >= prob.N
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s])
        np.testing.assert_allclose(U[s], ref, rtol=2e-5, atol=1e-6 * np.abs(ref).max())
    np.testing.assert_allclose(g, W.grad(V[0]), rtol=1e-4, atol=1e-5 * np.abs(W.grad(V[0])).max())
    assert f == pytest.approx(W.f(V[0]), rel=1e-6)


def test_default_rho_matches_oracle_rule(rpt):
    from oracle import default_rho
    prob = random_problem(**CASES["ragged"])
    with plan_of(rpt, prob) as P:
        st = P.stats()
    assert st["default_rho"] == pytest.approx(default_rho(Weighted(prob)), rel=1e-12)
    # a row that is empty in scenario s contributes the constant c_s w_i p_i^2 to f
    # (Eq. 1); rows empty in every scenario are not stored at all
    c = np.ones(prob.N) if prob.scen_weight is None else prob.scen_weight
    const = 0.0
    empty_all = np.ones(prob.m, bool)
    for s, rp in enumerate(prob.row_ptr):
        e = np.diff(rp) == 0
        empty_all &= e
        const += float(c[s] * np.sum(prob.voxel_w[e] * prob.presc[e] ** 2))
    assert st["const_term"] == pytest.approx(const, rel=1e-12, abs=1e-9)
    assert st["m_active"] == int((~empty_all).sum())


def test_row_path_selection(rpt, monkeypatch):
    monkeypatch.delenv("RPT_ROW_PATH", raising=False)
    prob = random_problem(**CASES["long_rows"])          # rows of 300 entries
    with plan_of(rpt, prob) as P:
        assert P.stats()["row_blocks"] >= 1
    monkeypatch.setenv("RPT_TMA_CMAX", "128")           # a row no longer fits one stage
    with pytest.raises(rpt.RptError) as e:
        plan_of(rpt, prob, row_path=2)
    assert e.value.status == rpt.EUNSUPPORTED
    with plan_of(rpt, prob) as P:                        # the default falls back to the register path
        U = P.apply_normal(np.ones((prob.N, prob.n)), 1.0)
    W = Weighted(prob)
    np.testing.assert_allclose(U[0], W.normal_apply(0, np.ones(prob.n), 1.0), rtol=1e-4)


def test_stream_path_takes_rows_longer_than_a_chunk(rpt, monkeypatch):
    monkeypatch.setenv("RPT_STR_CMAX", "128")           # rows of 300 entries: one-row chunks
    prob = random_problem(**CASES["long_rows"])
    with plan_of(rpt, prob, row_path=3) as P:
        assert P.stats()["row_path"] == 3
        V = np.random.default_rng(3).uniform(-1, 1, size=(prob.N, prob.n))
        U = P.apply_normal(V, 0.5)
    W = Weighted(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], 0.5)
        np.testing.assert_allclose(U[s], ref, rtol=2e-4, atol=2e-4 * np.abs(ref).max())


def test_profile_row_pass(rpt):
    prob = random_problem(**CASES["ragged"])
    with plan_of(rpt, prob) as P:
        P.apply_normal(np.ones((prob.N, prob.n)), 0.0)
        ms, by = P.profile_row_pass(0, reps=3)
        ms1, by1 = P.profile_row_pass(1, reps=3)
        st = P.stats()
    assert ms > 0 and ms1 > 0
    assert by == st["matrix_bytes"] + 4.0 * prob.N * st["m_active"] + 8.0 * prob.N * prob.n
    assert by1 == by + 4.0 * prob.N * st["m_active"]
