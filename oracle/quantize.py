"""Reduced-precision storage of the dose matrices, as a plain definition
(TEST INFRASTRUCTURE ONLY, like the rest of this package).

The paper keeps A_s in double precision.  The library also offers a storage
form with fewer bytes per entry.  For every scenario s and spot column j:
  * an FP32 scale  s_j = max_i |a_ij| / F  (s_j = 1 for an empty column), where
    F = 1 for bfloat16 and F = 448, the largest finite FP8-e4m3 value, for FP8;
  * a code  q_ij = round(a_ij / s_j)  in the target format: round to nearest,
    ties to even; e4m3 saturates at +-448;
  * the dequantised entry  q_ij * s_j, which is what the stored matrix means.
The divisions and the maximum are float32 operations, as the definition states.
The formats follow their published definitions: bfloat16 is the upper half of
an IEEE binary32; OCP FP8 E4M3 has 1 sign bit, 4 exponent bits (bias 7) and
3 mantissa bits, subnormals, no infinities, and S.1111.111 as NaN.
"""
import numpy as np

F_MAX = {"bf16": 1.0, "fp8": 448.0}


def bf16_round(x):
    """float32 array -> float32 array holding the nearest bfloat16 values
    (ties to even).  Finite inputs only."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32)


def e4m3_values():
    """The 127 non-negative finite E4M3 values, increasing; index = code."""
    v = []
    for code in range(127):            # 0x7F is NaN
        e, m = code >> 3, code & 7
        v.append(m * 2.0 ** -9 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(v)


_E4M3 = e4m3_values()


def e4m3_round(x):
    """float32 array -> float32 array holding the nearest E4M3 values (ties to
    the even code, i.e. even mantissa; magnitudes above 448 saturate)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.minimum(np.abs(x), _E4M3[-1])
    hi = np.clip(np.searchsorted(_E4M3, ax, side="left"), 0, len(_E4M3) - 1)
    lo = np.maximum(hi - 1, 0)
    dlo = ax - _E4M3[lo]
    dhi = _E4M3[hi] - ax
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo)
    return (np.sign(x) * _E4M3[code]).astype(np.float32)


def column_scales(val, col, n, fmt):
    """FP32 per-column scales of one scenario's entries."""
    mx = np.zeros(n, dtype=np.float32)
    np.maximum.at(mx, col, np.abs(val.astype(np.float32)))
    s = np.ones(n, dtype=np.float32)
    nz = mx > 0
    s[nz] = mx[nz] / np.float32(F_MAX[fmt])
    return s


def quantise_values(val, col, n, fmt):
    """(dequantised float64 entries, codes as float32, scales) of one scenario."""
    s = column_scales(val, col, n, fmt)
    r = val.astype(np.float32) / s[col]                 # float32 division
    q = bf16_round(r) if fmt == "bf16" else e4m3_round(r)
    return q.astype(np.float64) * s[col].astype(np.float64), q, s


def quantised_problem(prob, fmt):
    """The same problem with every A_s replaced by its dequantised storage."""
    from copy import copy
    out = copy(prob)
    out.val = []
    for s in range(prob.N):
        deq, _, _ = quantise_values(np.asarray(prob.val[s]), np.asarray(prob.col_idx[s]), prob.n, fmt)
        out.val.append(deq)
    return out
