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
