"""Learned warm start (rpt_mlp_*): the network's forward pass and gradient on
the GPU against the float64 oracle (oracle/mlp.py), training, and what the
trained network gains over cold-start ADMM-BB on held-out objective weights,
with the oracle's objective and optimality certificate deciding."""
import numpy as np
import pytest

from oracle import Weighted, certificates
from oracle.mlp import forward, loss_grad
from synthetic import config_tiny_plain, reweighted, sample_weights, N_WEIGHT_SLOTS

from tests.gpu_util import gpu_lib, plan_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpt():
    return gpu_lib()


def test_gradient_and_forward_match_oracle(rpt):
    """FP32 compute form (CUDA cores) against the float64 oracle."""
    dims = [9, 70, 70, 45]                     # sizes that leave ragged GEMM tiles
    rng = np.random.default_rng(3)
    X = rng.normal(size=(37, 9)).astype(np.float32)
    Y = rng.normal(size=(37, 45)).astype(np.float32)
    with rpt.Mlp(9, 70, 2, 45, seed=5, compute=rpt.F32) as net:
        p = net.get_params().astype(np.float64)
        loss, g = net.loss_grad(X, Y)
        out = net.predict(X)
        one = rpt.mlp_infer(net, X[5])
    ref_out = forward(p, dims, X)[-1]
    np.testing.assert_allclose(out, ref_out, rtol=1e-4, atol=1e-5 * np.abs(ref_out).max())
    # rpt_mlp_infer: the same network on one input
    np.testing.assert_allclose(one, out[5], rtol=1e-5, atol=1e-6 * np.abs(out[5]).max())
    ref_loss, ref_g = loss_grad(p, dims, X, Y)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    np.testing.assert_allclose(g, ref_g, rtol=1e-3, atol=1e-4 * np.abs(ref_g).max())


@pytest.mark.parametrize("dims,rows", [([9, 70, 70, 45], 37), ([9, 512, 512, 512, 200], 128)])
def test_bf16_tensor_core_gradient_matches_oracle(rpt, dims, rows):
    """BF16 compute form (tensor cores, FP32 accumulation) against the float64
    oracle of the same form (oracle.mlp with bf16_operand: every operand of the
    layer products rounded to bfloat16, sums, biases and ReLUs exact).  What
    remains is float32 accumulation and the rare activation whose float32 value
    rounds to the other bfloat16 neighbour: 1e-3 relative per tensor (in norm).
    The form's own deviation from the exact float64 network is reported.
    Ragged tiles (70, 45, 37 rows) and the learned form's own shape
    (9 -> 512 x 3 -> 200, batch 128)."""
    from oracle.mlp import unpack, bf16_operand
    rng = np.random.default_rng(4)
    X = rng.normal(size=(rows, dims[0])).astype(np.float32)
    Y = rng.normal(size=(rows, dims[-1])).astype(np.float32)
    with rpt.Mlp(dims[0], dims[1], len(dims) - 2, dims[-1], seed=6) as net:
        p = net.get_params().astype(np.float64)
        loss, g = net.loss_grad(X, Y)
        out = net.predict(X)
    ref_out = forward(p, dims, X, bf16_operand)[-1]
    assert np.linalg.norm(out - ref_out) <= 1e-3 * np.linalg.norm(ref_out)
    ref_loss, ref_g = loss_grad(p, dims, X, Y, bf16_operand)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    worst = 0.0
    for (W, b), (Wr, br) in zip(unpack(g, dims), unpack(ref_g, dims)):
        assert np.linalg.norm(W - Wr) <= 1e-3 * np.linalg.norm(Wr)
        assert np.linalg.norm(b - br) <= 1e-3 * np.linalg.norm(br)
    _, exact_g = loss_grad(p, dims, X, Y)
    for (W, _), (We, _) in zip(unpack(g, dims), unpack(exact_g, dims)):
        worst = max(worst, float(np.linalg.norm(W - We) / np.linalg.norm(We)))
    print(f"bfloat16 form vs exact float64 network, worst weight-gradient tensor: {worst:.2e}")


def test_set_params_round_trip_and_training_reduces_loss(rpt):
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(512, 4)).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], X[:, 2] ** 2 - X[:, 3]], axis=1).astype(np.float32)
    with rpt.Mlp(4, 64, 2, 2, seed=1) as net:
        p0 = net.get_params()
        net.set_params(p0)
        np.testing.assert_array_equal(net.get_params(), p0)
        l0, _ = net.loss_grad(X, Y)
        net.train(X, Y, epochs=200, batch=64, lr=3e-3)
        l1, _ = net.loss_grad(X, Y)
    assert l1 < 0.1 * l0, (l0, l1)


def _features(sw, d):
    f = np.zeros(N_WEIGHT_SLOTS + 1, dtype=np.float32)
    nz = sw > 0
    f[:N_WEIGHT_SLOTS][nz] = np.log10(sw[nz]) / 2.0
    f[-1] = (d - 67.5) / 7.5
    return f


def test_learned_warm_start_gains_over_cold_start(rpt):
    """The learned form's network (9 -> 512 x 3 -> n, bfloat16 tensor cores) trained
    on solutions of one plan reweighted in place (rpt_plan_set_weights) over a
    weight sweep; on held-out settings the warm start needs fewer iterations
    than the cold start, and the oracle judges both results."""
    base = config_tiny_plain(0)
    rng = np.random.default_rng(7)
    n_train, n_test = 96, 8
    settings = [sample_weights(rng, base.labels) for _ in range(n_train + n_test)]
    feats, targets = [], []
    cold_it, warm_it = [], []
    with plan_of(rpt, base) as P:
        for sw, d in settings[:n_train]:
            prob = reweighted(base, sw, d)
            P.set_weights(prob.voxel_w, prob.presc)
            z, info = P.admm_bb_solve(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, subproblem=rpt.SUB_CHOL)
            assert info["status"] == 0
            feats.append(_features(sw, d))
            targets.append((z / prob.ub).astype(np.float32))
        X, Y = np.stack(feats), np.stack(targets)
        with rpt.Mlp(X.shape[1], 512, 3, base.n, seed=2) as net:
            net.train(X, Y, epochs=300, batch=32, lr=1e-3)
            for sw, d in settings[n_train:]:
                prob = reweighted(base, sw, d)
                W = Weighted(prob)
                P.set_weights(prob.voxel_w, prob.presc)
                xc, ic = P.admm_bb_solve()
                xw, iw, used = rpt.admm_bb_solve_learned(P, net, _features(sw, d), prob.ub)
                assert ic["status"] == 0 and iw["status"] == 0
                # the oracle checks both results: same objective to the tolerance, near-optimal
                fc, fw = W.f(xc), W.f(xw)
                assert abs(fw - fc) / fc <= 1e-3, (fw, fc)
                assert certificates(W, xw)["pg"] < 1e-2
                cold_it.append(ic["iterations"])
                warm_it.append(iw["iterations"])
    print(f"held-out iterations to 1e-4: cold {np.mean(cold_it):.1f}, learned warm start {np.mean(warm_it):.1f}")
    assert np.mean(warm_it) < 0.9 * np.mean(cold_it), (cold_it, warm_it)
