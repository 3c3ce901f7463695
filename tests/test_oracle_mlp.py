"""Pin of the oracle's MLP gradient (oracle/mlp.py) by central finite
differences, and its forward pass by a literal per-neuron loop."""
import numpy as np

from oracle.mlp import forward, loss_grad, unpack


def _setup(seed=0, dims=(5, 7, 6, 4), B=9):
    rng = np.random.default_rng(seed)
    n = sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))
    p = rng.normal(size=n) * 0.5
    X = rng.normal(size=(B, dims[0]))
    Y = rng.normal(size=(B, dims[-1]))
    return p, list(dims), X, Y


def test_gradient_matches_central_differences():
    p, dims, X, Y = _setup()
    L, g = loss_grad(p, dims, X, Y)
    h = 1e-6
    num = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        num[k] = (loss_grad(p + e, dims, X, Y)[0] - loss_grad(p - e, dims, X, Y)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-8)


def test_forward_matches_neuron_loop():
    p, dims, X, Y = _setup(1)
    layers = unpack(p, dims)
    out = forward(p, dims, X)[-1]
    for i in range(X.shape[0]):
        a = list(X[i])
        for l, (W, b) in enumerate(layers):
            nxt = []
            for r in range(W.shape[0]):
                z = b[r] + sum(W[r, c] * a[c] for c in range(W.shape[1]))
                nxt.append(max(z, 0.0) if l + 1 < len(layers) else z)
            a = nxt
        np.testing.assert_allclose(out[i], a, rtol=1e-12, atol=1e-12)


def test_bf16_form_rounds_only_the_product_operands():
    """The bfloat16 compute form of the oracle network: with one linear layer
    whose weights and inputs are already bfloat16 values, rounding the operands
    changes nothing, so it equals the exact function (biases and sums exact);
    with hidden layers it stays within a few bfloat16 units of the exact one;
    and its rounding is the library-pinned bfloat16 rounding of a float32 value."""
    from oracle.mlp import bf16_operand, forward, loss_grad
    from oracle.quantize import bf16_round
    rng = np.random.default_rng(9)
    dims = [6, 5]
    p = bf16_round(rng.normal(size=6 * 5 + 5).astype(np.float32)).astype(np.float64)
    p[30:] = rng.normal(size=5)                  # biases need not be bfloat16 values
    X = bf16_round(rng.normal(size=(7, 6)).astype(np.float32)).astype(np.float64)
    Y = rng.normal(size=(7, 5))
    np.testing.assert_array_equal(forward(p, dims, X, bf16_operand)[-1], forward(p, dims, X)[-1])
    l0, g0 = loss_grad(p, dims, X, Y)
    l1, g1 = loss_grad(p, dims, X, Y, bf16_operand)
    assert l0 == l1
    # dW = r(d)^T X: only the output gradient is rounded here
    np.testing.assert_allclose(g1, g0, rtol=2 ** -7, atol=2 ** -7 * np.abs(g0).max())
    dims = [9, 40, 40, 12]
    q = rng.normal(size=sum(a * b + a for a, b in zip(dims[1:], dims[:-1]))) * 0.3
    X = rng.normal(size=(20, 9))
    out0 = forward(q, dims, X)[-1]
    out1 = forward(q, dims, X, bf16_operand)[-1]
    assert np.linalg.norm(out1 - out0) <= 3 * 2 ** -8 * np.linalg.norm(out0)
    x = np.float64(1.0 + 2 ** -8 + 2 ** -12)     # past half a bfloat16 unit (2^-7 at 1): rounds up
    assert bf16_operand(np.array([x]))[0] == 1.0 + 2 ** -7
    assert bf16_operand(np.array([1.0 + 2 ** -9]))[0] == 1.0
