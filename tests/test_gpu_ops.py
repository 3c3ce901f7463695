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
from tests.gpu_util import gpu_lib, plan_of, fp32_op_bound, fixed_point_slack

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
# switches), the streaming path, the streaming path with tiny chunks (many
# chunk hand-overs, class changes inside a warp's run, one-row chunks), the
# bundled ring and the bundled ring with tiny stages, each with float atomics
# and with exact fixed-point sums, and the bundled ring's smaller CTAs (768 and
# 640 threads, 8 and 10 block columns per lane in registers)
PATHS = {
    "reg": dict(row_path=1),
    "tma": dict(row_path=2),
    "tma_small": dict(row_path=2, chunk_entries=1280, chunk_rows=8, stages=2),
    "stream": dict(row_path=3),
    "stream_small": dict(row_path=3, chunk_entries=64, chunk_rows=3),
    "bun": dict(row_path=4),
    "bun_small": dict(row_path=4, chunk_entries=1280, chunk_rows=3, stages=2),
    "bun_exact": dict(row_path=4, accumulate=1),
    "bun_exact_small": dict(row_path=4, accumulate=1, chunk_entries=1280, chunk_rows=3, stages=2),
    "bun_768": dict(row_path=4, ring_threads=768),
    "bun_640_small": dict(row_path=4, ring_threads=640, chunk_entries=1280, chunk_rows=3, stages=2),
    "bun_640_exact": dict(row_path=4, ring_threads=640, accumulate=1),
}


@pytest.fixture(params=sorted(PATHS))
def path(request):
    return PATHS[request.param]


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
    with plan_of(rpt, prob, **path) as P:
        U = P.apply_normal(V, rho)
    Wa = _abs_W(W)
    k = fp32_op_bound(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], rho)
        mag = Wa.At[s].T @ (Wa.At[s] @ np.abs(V[s])) + 0.5 * rho * np.abs(V[s])
        err = np.abs(U[s] - ref)
        slack = fixed_point_slack(prob, s, V[s])
        assert np.all(err <= k * mag + slack + 1e-300), (case, s, float((err / np.maximum(mag, 1e-300)).max()))


@pytest.mark.parametrize("case", sorted(CASES))
def test_gradient_and_objective(rpt, case, path):
    prob = random_problem(**CASES[case])
    W = Weighted(prob)
    rng = np.random.default_rng(12)
    x = rng.uniform(0.0, 4.0, size=prob.n)
    with plan_of(rpt, prob, **path) as P:
        g, f = P.gradient(x)
        f2 = P.objective(x)
    Wa = _abs_W(W)
    k = fp32_op_bound(prob)
    mag = np.zeros(prob.n)
    for s in range(prob.N):
        mag += 2.0 * (Wa.At[s].T @ (Wa.At[s] @ np.abs(x) + Wa.pt[s]))
    ref = W.grad(x)
    slack = sum(2.0 * fixed_point_slack(prob, s, x, resid=True) for s in range(prob.N))
    assert np.all(np.abs(g - ref) <= k * mag + slack + 1e-300), float((np.abs(g - ref) / mag).max())
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
    with plan_of(rpt, prob, **path) as P:
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


def test_row_path_selection(rpt):
    prob = random_problem(**CASES["long_rows"])          # rows of 300 entries
    with plan_of(rpt, prob) as P:                        # default: the bundled ring where it fits
        assert P.stats()["row_path"] == 4 and P.stats()["row_blocks"] >= 1
    for path in (2, 4):                                  # a row (bundle) no longer fits one stage
        with pytest.raises(rpt.RptError) as e:
            plan_of(rpt, prob, row_path=path, chunk_entries=128)
        assert e.value.status == rpt.EUNSUPPORTED
    with plan_of(rpt, prob, chunk_entries=128) as P:     # the default falls back to the register path
        assert P.stats()["row_path"] == 1
        U = P.apply_normal(np.ones((prob.N, prob.n)), 1.0)
    W = Weighted(prob)
    np.testing.assert_allclose(U[0], W.normal_apply(0, np.ones(prob.n), 1.0), rtol=1e-4)
    with pytest.raises(rpt.RptError) as e:                # CTA sizes of the bundled ring: 640, 768, 1024
        plan_of(rpt, prob, ring_threads=512)
    assert e.value.status == rpt.EINVAL


def test_stream_path_takes_rows_longer_than_a_chunk(rpt):
    prob = random_problem(**CASES["long_rows"])          # rows of 300 entries: one-row chunks of 128
    with plan_of(rpt, prob, row_path=3, chunk_entries=128) as P:
        assert P.stats()["row_path"] == 3
        V = np.random.default_rng(3).uniform(-1, 1, size=(prob.N, prob.n))
        U = P.apply_normal(V, 0.5)
    W = Weighted(prob)
    for s in range(prob.N):
        ref = W.normal_apply(s, V[s], 0.5)
        np.testing.assert_allclose(U[s], ref, rtol=2e-4, atol=2e-4 * np.abs(ref).max())


def test_bundled_pass_is_bitwise_reproducible(rpt):
    """The bundled ring with exact sums (accumulate = 1) adds 64-bit fixed-point
    contributions, which is exact: repeated passes give identical bits whatever
    order the atomics and the chunk queues take, on every value format, and the
    same bits on every CTA size (a lane's dot product runs in the same order)."""
    prob = random_problem(**CASES["ragged"])
    V = np.random.default_rng(21).normal(size=(prob.N, prob.n))
    x = np.random.default_rng(22).uniform(0.0, 3.0, size=prob.n)
    by_thr = {}
    for vf, thr in ((rpt.F32, 0), (rpt.BF16, 0), (rpt.FP8E4M3, 0), (rpt.F32, 768), (rpt.F32, 640)):
        with plan_of(rpt, prob, row_path=4, value_format=vf, accumulate=1, ring_threads=thr) as P:
            assert P.stats()["exact_sums"] == 1
            assert P.stats()["ring_threads"] == (thr or 1024)
            U = [P.apply_normal(V, 1.3) for _ in range(4)]
            G = [P.gradient(x)[0] for _ in range(4)]
        for k in range(1, 4):
            assert np.array_equal(U[0], U[k]) and np.array_equal(G[0], G[k])
        if vf == rpt.F32:
            by_thr[thr] = (U[0], G[0])
    for thr in (768, 640):
        assert np.array_equal(by_thr[thr][0], by_thr[0][0]) and np.array_equal(by_thr[thr][1], by_thr[0][1])


def test_profile_row_pass(rpt):
    prob = random_problem(**CASES["ragged"])
    with plan_of(rpt, prob) as P:
        P.apply_normal(np.ones((prob.N, prob.n)), 0.0)
        ms, by = P.profile_row_pass(0, reps=3)
        ms1, by1 = P.profile_row_pass(1, reps=3)
        st = P.stats()
    assert ms > 0 and ms1 > 0
    assert st["row_path"] == 4 and 0.0 < st["bundle_fill"] <= 1.0
    # bundled: block columns (4 values + index) and 64-byte bundle records, plus the vectors
    assert by == st["block_cols"] * 20.0 + 64.0 * (st["bundles"] + prob.N) + 8.0 * prob.N * prob.n
    assert by1 == by
    assert st["matrix_bytes"] == st["block_cols"] * 20 + 4 * (st["bundles"] + prob.N)
    with plan_of(rpt, prob, row_path=2) as P:
        P.apply_normal(np.ones((prob.N, prob.n)), 0.0)
        ms, by = P.profile_row_pass(0, reps=3)
        ms1, by1 = P.profile_row_pass(1, reps=3)
        st = P.stats()
    assert by == st["matrix_bytes"] + 4.0 * prob.N * st["m_active"] + 8.0 * prob.N * prob.n
    assert by1 == by + 4.0 * prob.N * st["m_active"]


@pytest.mark.parametrize("path", [2, 4])
def test_set_weights_matches_a_fresh_plan(rpt, path):
    """rpt_plan_set_weights: new voxel weights and prescriptions on an existing
    plan give the operators of a plan created with them (bitwise on the bundled
    path 4 with exact sums, within the float32 bound on path 2), the
    default rho and the constant of Eq. 2 of the oracle's rule, and a solve that
    reaches the new problem's optimum."""
    from oracle import default_rho, lsq_box
    prob = random_problem(**CASES["ragged"])
    rng = np.random.default_rng(31)
    w2 = prob.voxel_w * rng.uniform(0.1, 10.0, size=prob.m)
    p2 = prob.presc + rng.uniform(0.0, 2.0, size=prob.m) * (rng.random(prob.m) < 0.3)
    import copy
    prob2 = copy.copy(prob)
    prob2.voxel_w, prob2.presc = w2, p2
    W2 = Weighted(prob2)
    V = rng.normal(size=(prob.N, prob.n))
    x = rng.uniform(0.0, 3.0, size=prob.n)
    acc = 1 if path == 4 else 0
    with plan_of(rpt, prob, row_path=path, accumulate=acc) as P, \
            plan_of(rpt, prob2, row_path=path, accumulate=acc) as Q:
        P.set_weights(w2, p2)
        sp, sq = P.stats(), Q.stats()
        Up, Uq = P.apply_normal(V, 0.7), Q.apply_normal(V, 0.7)
        (gp, fp), (gq, fq) = P.gradient(x), Q.gradient(x)
        zp, ip = P.admm_bb_solve(eps_abs=1e-7, eps_rel=1e-7, max_iter=20000)
    assert sp["const_term"] == sq["const_term"]
    assert sp["default_rho"] == pytest.approx(default_rho(W2), rel=1e-9)
    if path == 4:
        assert np.array_equal(Up, Uq) and np.array_equal(gp, gq) and fp == fq
    else:
        k = fp32_op_bound(prob)
        Wa = _abs_W(W2)
        for s in range(prob.N):
            mag = Wa.At[s].T @ (Wa.At[s] @ np.abs(V[s])) + 0.35 * np.abs(V[s])
            assert np.all(np.abs(Up[s] - Uq[s]) <= 2 * k * mag + 1e-300)
    xs = lsq_box(W2)
    assert (W2.f(zp) - W2.f(xs)) / W2.f(xs) <= 1e-6
