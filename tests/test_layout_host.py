"""Host layout logic of plan creation on the CPU (paper_2304_14568_gb300/csrc/
layout.h, built here with the host compiler alone): lanes per row, the
bank-balanced entry order, the lane-interleaved order of the streaming path and
the cutting of row lists into row-pass chunks.  Each is checked against its
stated contract: permutations stay permutations, groups spread over banks,
chunks cover every row once within their size limits."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2304_14568_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("layout") / "liblayout_shim.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(HERE, "layout_shim.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    i32p, f32p, i64p = (np.ctypeslib.ndpointer(t, flags="C") for t in (np.int32, np.float32, np.int64))
    L.shim_bank_balance.argtypes = [i32p, f32p, C.c_int, C.c_int]
    L.shim_interleave_row.argtypes = [i32p, f32p, C.c_int, C.c_int, i32p, f32p]
    L.shim_build_chunks.argtypes = [C.c_int, i32p, i32p, i64p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    i64p, i32p, i32p, i32p, i32p, i32p, i32p, i32p]
    L.shim_build_bundles.argtypes = [C.c_int, i32p, i32p, f32p, i32p, f32p, f32p, C.c_int64, C.c_int,
                                     i32p, f32p, i32p, i32p, C.POINTER(C.c_int)]
    L.shim_build_bundles.restype = C.c_int64
    L.shim_bundles_all_equal.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int]
    return L


def test_lanes_per_row(shim):
    for mn in (1, 2, 4, 8, 16, 32):
        for ln in range(0, 400):
            g = shim.shim_lanes_for(ln, mn)
            assert g >= mn and g <= max(32, mn) and (g & (g - 1)) == 0
            assert g == 32 or g * 8 >= ln                              # 8 entries per lane suffice
            assert g == mn or (g // 2) * 8 < ln                         # and it is the smallest such
    # streaming classes: lanes 8/16/32/32/32 for padded rows up to 32/64/128/256/any entries
    for ln, cls in [(4, 0), (32, 0), (36, 1), (64, 1), (68, 2), (128, 2), (132, 3), (256, 3), (260, 4), (5000, 4)]:
        assert shim.shim_stream_class(ln) == cls
    assert [shim.shim_stream_lanes(x) for x in (32, 64, 128, 256, 999)] == [8, 16, 32, 32, 32]


@pytest.mark.parametrize("seed", range(6))
def test_bank_balance_is_a_permutation_that_spreads_banks(shim, seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        ln = int(rng.integers(1, 300))
        G = int(rng.choice([8, 16, 32]))
        # sorted distinct columns, clustered (a row of the dose periphery) or spread
        span = int(rng.choice([ln + 5, 4 * ln, 5000]))
        col = np.sort(rng.choice(span, size=ln, replace=False)).astype(np.int32)
        val = (rng.random(ln) + 0.1).astype(np.float32)
        c2, v2 = col.copy(), val.copy()
        shim.shim_bank_balance(c2, v2, ln, G)
        pairs = sorted(zip(col.tolist(), val.tolist()))
        assert sorted(zip(c2.tolist(), v2.tolist())) == pairs              # same entries, same pairing
        # every aligned group of G takes distinct banks while the row has enough banks left
        for g0 in range(0, ln, G):
            grp = c2[g0:g0 + G] & 31
            left = np.unique(c2[g0:] & 31).size                         # banks with entries not yet placed
            assert np.unique(grp).size >= min(grp.size, left)


def _bank_order_rule(col, G):
    """The bank order's rule written out: entries grouped by bank (spot column
    mod 32) in their original order; every group of G output slots takes one
    entry from each non-empty bank, banks with the most entries left first (ties:
    the lower bank), then, if there are fewer such banks than slots, further
    entries from those banks again in the same order."""
    left = {b: [i for i in range(len(col)) if col[i] % 32 == b] for b in range(32)}
    order = []
    while len(order) < len(col):
        banks = sorted((b for b in range(32) if left[b]), key=lambda b: (-len(left[b]), b))
        want = min(G, len(col) - len(order))
        taken = 0
        for b in banks[:want]:
            order.append(left[b].pop(0))
            taken += 1
        k = 0
        while taken < want:
            b = banks[k % len(banks)]
            if left[b]:
                order.append(left[b].pop(0))
                taken += 1
            k += 1
    return order


@pytest.mark.parametrize("seed", range(3))
def test_bank_balance_order_follows_its_rule(shim, seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(60):
        ln = int(rng.integers(1, 200))
        G = int(rng.choice([1, 2, 8, 16, 32]))
        kind = int(rng.integers(0, 3))
        if kind == 0:     # clustered: a few banks only, so groups are filled from them again
            col = np.sort(rng.choice(np.arange(0, 32 * ln, 32), size=ln, replace=False) + rng.integers(0, 3))
        else:
            span = ln + 5 if kind == 1 else 5000
            col = np.sort(rng.choice(span, size=ln, replace=False))
        col = col.astype(np.int32)
        val = np.arange(ln, dtype=np.float32)
        c2, v2 = col.copy(), val.copy()
        shim.shim_bank_balance(c2, v2, ln, G)
        order = _bank_order_rule(col.tolist(), G)
        assert c2.tolist() == col[order].tolist() and v2.tolist() == val[order].tolist()


@pytest.mark.parametrize("plen,G", [(4, 8), (32, 8), (36, 8), (64, 16), (96, 32), (128, 32), (132, 32), (260, 32)])
def test_interleave_row_formula(shim, plen, G):
    col = np.arange(plen, dtype=np.int32) * 3
    val = np.arange(plen, dtype=np.float32) + 0.5
    oc = np.empty(plen, np.int32)
    ov = np.empty(plen, np.float32)
    shim.shim_interleave_row(col, val, plen, G, oc, ov)
    assert sorted(oc.tolist()) == sorted(col.tolist())                  # a permutation
    np.testing.assert_array_equal(ov, oc.astype(np.float32) / 3 + 0.5)   # pairs kept
    nq = plen // 4
    for b in range((nq + G - 1) // G):
        gb = min(G, nq - b * G)
        for lane in range(gb):
            for k in range(4):
                assert oc[4 * (b * G + lane) + k] == col[4 * b * G + k * gb + lane]


def _chunks(shim, nrows, plen, base, cmax, rmax, stream, min_lanes=8):
    N = len(nrows)
    cap = int(sum(nrows)) + 8
    arr = {k: np.zeros(cap, np.int32) for k in ("rb", "nr", "ne", "gr", "s", "pad")}
    g_al = np.zeros(cap, np.int64)
    sc = np.zeros(N + 1, np.int32)
    n = shim.shim_build_chunks(N, np.asarray(nrows, np.int32), np.asarray(plen, np.int32),
                               np.asarray(base, np.int64), cmax, rmax, int(stream), min_lanes, cap, g_al,
                               arr["rb"], arr["nr"], arr["ne"], arr["gr"], arr["s"], arr["pad"], sc)
    return n, g_al, arr, sc


@pytest.mark.parametrize("stream", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_chunks_cover_every_row_once_within_limits(shim, stream, seed):
    rng = np.random.default_rng(seed)
    N = 3
    nrows = [int(rng.integers(1, 400)) for _ in range(N)]
    plen, base = [], []
    off = 0
    for s in range(N):
        lens = np.sort(rng.integers(1, 600, size=nrows[s]))[::-1]          # decreasing, as at plan creation
        p = ((lens + 3) // 4 * 4).astype(np.int32)
        plen.extend(p.tolist())
        base.append(off)
        off += int(p.sum())
    cmax, rmax = (1536, 128) if stream else (2048, 64)
    n, g_al, a, sc = _chunks(shim, nrows, plen, base, cmax, rmax, stream)
    assert n > 0 and sc[0] == 0 and sc[N] == n
    k0 = 0
    for s in range(N):
        p = np.asarray(plen[k0:k0 + nrows[s]])
        start = np.concatenate([[0], np.cumsum(p)])
        k0 += nrows[s]
        nxt = 0
        for c in range(sc[s], sc[s + 1]):
            assert a["s"][c] == s and a["rb"][c] == nxt and a["nr"][c] >= 1   # consecutive, no gaps
            rows = range(a["rb"][c], a["rb"][c] + a["nr"][c])
            nxt += a["nr"][c]
            assert a["nr"][c] <= rmax
            lo = base[s] + start[a["rb"][c]]
            hi = base[s] + start[a["rb"][c] + a["nr"][c]]
            assert g_al[c] % 16 == 0 and g_al[c] <= lo and g_al[c] > lo - 16
            assert a["ne"][c] % 16 == 0 and g_al[c] + a["ne"][c] >= hi          # the copy spans the rows
            if not (stream and a["nr"][c] == 1):
                assert a["ne"][c] <= cmax or a["ne"][c] == 16
            cls = [shim.shim_stream_class(int(p[r])) if stream else shim.shim_lanes_for(int(p[r]), 8)
                   for r in rows]
            assert len(set(cls)) == 1                                   # one class per chunk
            assert a["gr"][c] == (shim.shim_stream_lanes(int(p[rows[0]])) if stream else cls[0])
        assert nxt == nrows[s]                                          # every row exactly once


def test_ring_refuses_a_row_longer_than_a_stage(shim):
    n, *_ = _chunks(shim, [2], [4096, 8], [0], 2048, 64, False)
    assert n == -1
    n, *_ = _chunks(shim, [2], [4096, 8], [0], 2048, 64, True)          # the streaming path takes it alone
    assert n == 2


def _bundles(shim, rp, ci, va, kept, wc, pr):
    nr = rp.size - 1
    cap_bc, cap_b = int(rp[-1]) + 8, nr // 4 + 2
    col = np.zeros(cap_bc, np.int32)
    val = np.zeros(cap_bc * 4, np.float32)
    rec = np.zeros((cap_b + 1) * 16, np.int32)
    pos = np.zeros(cap_b, np.int32)
    nb = C.c_int()
    nbc = shim.shim_build_bundles(nr, rp, ci, va, kept, wc, pr, cap_bc, cap_b, col, val, rec, pos, C.byref(nb))
    assert nbc >= 0
    return col[:nbc], val[:4 * nbc].reshape(-1, 4), rec[:(nb.value + 1) * 16].reshape(-1, 4, 4), pos[:nb.value]


@pytest.mark.parametrize("seed", range(5))
def test_bundles_store_every_entry_once(shim, seed):
    """Row bundles (the bundled ring's layout): 4 consecutive rows per bundle;
    every entry of the input appears exactly once, at its row slot and spot
    column; absent entries are stored as 0; every bundle's columns are distinct;
    bundles are sorted by decreasing width; pos_of is a permutation; records hold
    the offsets, weights, prescriptions and kept indices (-1 for missing rows)."""
    rng = np.random.default_rng(seed)
    nr = int(rng.integers(1, 60))
    n = int(rng.choice([5, 40, 300]))
    lens = rng.integers(1, min(n, 50) + 1, size=nr)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    va = (rng.random(rp[-1]) + 0.01).astype(np.float32)
    kept = np.sort(rng.choice(10 * nr, size=nr, replace=False)).astype(np.int32)
    wc = rng.random(nr).astype(np.float32)
    pr = rng.random(nr).astype(np.float32)
    col, val, rec, pos = _bundles(shim, rp, ci, va, kept, wc, pr)
    nb = (nr + 3) // 4
    assert pos.size == nb and sorted(pos.tolist()) == list(range(nb))
    widths = [rec[b + 1, 0, 0] - rec[b, 0, 0] for b in range(nb)]
    assert all(w1 >= w2 for w1, w2 in zip(widths, widths[1:]))
    assert rec[nb, 0, 0] == col.size
    seen = np.zeros(rp[-1], bool)
    for q in range(nb):
        b = pos[q]
        lo, hi = rec[b, 0, 0], rec[b + 1, 0, 0]
        cols = col[lo:hi]
        assert np.unique(cols).size == cols.size
        assert shim.shim_bundle_lanes(int(hi - lo)) in (8, 16, 32)
        for r in range(4):
            i = 4 * q + r
            if i >= nr:
                assert rec[b, 3, r] == -1 and rec[b, 1, r] == 0 and np.all(val[lo:hi, r] == 0)
                continue
            assert rec[b, 3, r] == kept[i]
            assert rec[b, 1, r] == wc[i:i + 1].view(np.int32)[0] and rec[b, 2, r] == pr[i:i + 1].view(np.int32)[0]
            row = dict(zip(ci[rp[i]:rp[i + 1]].tolist(), range(rp[i], rp[i + 1])))
            for k in range(lo, hi):
                e = row.get(int(col[k]))
                if e is None:
                    assert val[k, r] == 0.0
                else:
                    assert val[k, r] == va[e] and not seen[e]
                    seen[e] = True
            # the union covers the row
            assert set(row) <= set(cols.tolist())
    assert seen.all()


@pytest.mark.parametrize("seed", range(3))
def test_bundles_of_all_scenarios_on_threads_equal_one_by_one(shim, seed):
    """Plan creation bundles every scenario with the work cut into ranges that
    several threads take (build_bundles_all): the arrays equal those of
    build_bundles run scenario by scenario, for empty, small and multi-range
    scenarios and any thread count."""
    rng = np.random.default_rng(200 + seed)
    N = int(rng.integers(1, 6))
    keep = []
    for _ in range(N):
        nr = int(rng.choice([0, 1, 5, 300, 9000]))      # 9000 rows: two ranges of 2048 bundles
        n = int(rng.choice([7, 100, 3000]))
        lens = rng.integers(1, min(n, 120) + 1, size=nr)
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        ci = np.concatenate([np.sort(rng.choice(n, size=int(k), replace=False)) for k in lens] +
                            [np.zeros(0)]).astype(np.int32)
        va = rng.random(int(rp[-1])).astype(np.float32)
        keep.append((rp, ci, va))
    nrows = (C.c_int * N)(*[r.size - 1 for r, _, _ in keep])
    ptrs = [(C.c_void_p * N)(*[a[k].ctypes.data for a in keep]) for k in range(3)]
    for nt in (1, 3, 8):
        assert shim.shim_bundles_all_equal(N, nrows, *ptrs, nt) == 1, nt
