"""Multilayer perceptron of the learned warm start, in float64
(TEST INFRASTRUCTURE ONLY, like the rest of this package).

Network: x -> h_1 = relu(W_0 x + b_0) -> ... -> out = W_L h_L + b_L (the last
layer linear).  Loss of a batch of B rows and n_out outputs:
    L = (1 / (B n_out)) sum_{i,j} (out_ij - y_ij)^2.
Parameters as one array: for each layer W ([out][in], row-major) then b ([out]).
The gradient is written out by the chain rule, layer by layer, and pinned to
central finite differences in the tests.
"""
import numpy as np


def layer_shapes(dims):
    return [(dims[l + 1], dims[l]) for l in range(len(dims) - 1)]


def unpack(params, dims):
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for (r, c) in layer_shapes(dims):
        W = p[o:o + r * c].reshape(r, c)
        o += r * c
        b = p[o:o + r]
        o += r
        out.append((W, b))
    assert o == p.size
    return out


def bf16_operand(x):
    """The bfloat16 compute form's rounding of a GEMM operand: the value as the
    GPU holds it (float32), rounded to the nearest bfloat16 (ties to even)."""
    from .quantize import bf16_round
    return bf16_round(np.asarray(x, dtype=np.float64).astype(np.float32)).astype(np.float64)


def forward(params, dims, X, rnd=None):
    """All layer outputs: acts[0] = X, acts[l+1] = output of layer l.
    rnd: None for exact arithmetic, or a rounding applied to both operands of
    every layer product (bf16_operand: the bfloat16 compute form, whose weights
    and layer inputs are bfloat16 and whose sums, biases and ReLUs are exact)."""
    acts = [np.asarray(X, dtype=np.float64)]
    layers = unpack(params, dims)
    r = (lambda a: a) if rnd is None else rnd
    for l, (W, b) in enumerate(layers):
        z = r(acts[-1]) @ r(W).T + b
        acts.append(np.maximum(z, 0.0) if l + 1 < len(layers) else z)
    return acts


def loss_grad(params, dims, X, Y, rnd=None):
    """(loss, gradient as one array in the parameter layout).  rnd as in
    forward; in the backward products it rounds the layer-output gradient (after
    the ReLU mask), the layer input and the weights; the bias gradient sums the
    unrounded layer-output gradient."""
    layers = unpack(params, dims)
    acts = forward(params, dims, X, rnd)
    r = (lambda a: a) if rnd is None else rnd
    Y = np.asarray(Y, dtype=np.float64)
    B, n_out = Y.shape
    err = acts[-1] - Y
    loss = float(np.sum(err * err) / (B * n_out))
    d = 2.0 * err / (B * n_out)                  # dL/d out
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        if l + 1 < len(layers):
            d = d * (acts[l + 1] > 0.0)           # through the ReLU of layer l
        W, _ = layers[l]
        grads[l] = (r(d).T @ r(acts[l]), d.sum(axis=0))
        d = r(d) @ r(W)                           # dL/d acts[l]
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
