"""Pins of the oracle's reduced-precision storage definition (oracle/quantize.py).

The rounding is checked against an independent library routine (PyTorch's
float32 -> bfloat16 / float8_e4m3fn casts), against landmarks of the published
formats, and the dequantised matrices against the rounding error bound.
"""
import numpy as np
import pytest

from oracle.quantize import bf16_round, e4m3_round, e4m3_values, quantise_values, quantised_problem
from synthetic import random_problem

torch = pytest.importorskip("torch")


def test_bf16_matches_library_cast_including_ties():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100_000) * 10.0 ** rng.uniform(-6, 6, 100_000)).astype(np.float32)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 3 * 2 ** -130], dtype=np.float32)
    x = np.concatenate([x, ties])
    ref = torch.tensor(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(bf16_round(x), ref)
    assert bf16_round(np.float32([1 + 2 ** -8]))[0] == 1.0            # tie to even
    assert bf16_round(np.float32([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6  # tie to even (upward)


def test_e4m3_table_landmarks():
    v = e4m3_values()
    assert len(v) == 127 and np.all(np.diff(v) > 0)
    assert v[-1] == 448.0                 # S.1111.110
    assert v[1] == 2.0 ** -9              # smallest subnormal
    assert v[8] == 2.0 ** -6              # smallest normal
    assert v[0x38] == 1.0


def test_e4m3_matches_library_cast_in_range_and_saturates():
    rng = np.random.default_rng(1)
    x = (rng.uniform(-448, 448, 100_000) * 10.0 ** rng.uniform(-5, 0, 100_000)).astype(np.float32)
    mids = (e4m3_values()[:-1] + e4m3_values()[1:]) / 2            # exact ties
    x = np.concatenate([x, mids.astype(np.float32), -mids.astype(np.float32)])
    ref = torch.tensor(x).to(torch.float8_e4m3fn).float().numpy()
    np.testing.assert_array_equal(e4m3_round(x), ref)
    np.testing.assert_array_equal(e4m3_round(np.float32([500.0, -1e6])), [448.0, -448.0])


@pytest.mark.parametrize("fmt,rel", [("bf16", 2.0 ** -8), ("fp8", 2.0 ** -4)])   # half an ulp, relative
def test_dequantised_entries_within_rounding_bound(fmt, rel):
    prob = random_problem(7, m=400, n=50, N=2, mean_row=10.0)
    for s in range(prob.N):
        a = np.asarray(prob.val[s], dtype=np.float64)
        deq, q, sc = quantise_values(a, prob.col_idx[s], prob.n, fmt)
        col = prob.col_idx[s]
        # relative rounding error in the normal range; absolute near zero (subnormal step of the code times the scale)
        tiny = (2.0 ** -133 if fmt == "bf16" else 2.0 ** -10) * sc[col]
        assert np.all(np.abs(deq - a) <= rel * np.abs(a) * (1 + 1e-5) + tiny + 1e-12 * np.abs(a))
        # the largest entry of every column keeps its magnitude up to one rounding
        for j in np.unique(col):
            k = np.argmax(np.where(col == j, np.abs(a), -1))
            assert abs(deq[k] - a[k]) <= rel * abs(a[k]) * (1 + 1e-5)
    qp = quantised_problem(prob, fmt)
    assert qp.N == prob.N and qp.row_ptr is prob.row_ptr and qp.col_idx is prob.col_idx
