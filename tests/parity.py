"""Shared helpers for the parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them element by element.

The bar (per semiring):
  * integer, bool and min/select semirings and the heterogeneous
    maxw_label (compared as raw record bits): bit-exact row pointers,
    columns and values;
  * (+,x) fp64: identical pattern and |c - c_ref| <= 1e-12 * sum|a_ik b_kj|
    per entry (sum of |products| accumulated by the oracle).  For an entry
    with m products any two summation orders differ by at most about
    2(m-1)u*sum|ab| with u = 2^-53, so 1e-12 holds up to m ~ 4500 products
    per entry, above every entry of the test workloads.
"""
from __future__ import annotations

import numpy as np

FP64_TOL = 1e-12


def compare_rows(sr, got, want, rows=None, tol=FP64_TOL):
    """got = (row_ptr, col, val) over all rows (host arrays); want = oracle output
    over `rows` (all rows when None).  Raises AssertionError on the first mismatch."""
    g_rp, g_col, g_val = got
    w_rp, w_col, w_val, w_abs = want
    if rows is None:
        assert np.array_equal(g_rp, w_rp), _first_diff("row_ptr", g_rp, w_rp)
        assert np.array_equal(g_col, w_col), _first_diff("col", g_col, w_col)
        gv, wv, ab = g_val, w_val, w_abs
    else:
        rows = np.asarray(rows, dtype=np.int64)
        lens = g_rp[rows + 1] - g_rp[rows]
        assert np.array_equal(lens, np.diff(w_rp)), "row sizes differ on sampled rows"
        idx = np.concatenate([np.arange(g_rp[r], g_rp[r + 1]) for r in rows]) if len(rows) else \
            np.zeros(0, np.int64)
        assert np.array_equal(g_col[idx], w_col), _first_diff("col", g_col[idx], w_col)
        gv, wv, ab = g_val[idx], w_val, w_abs
    if sr == "maxw_label":  # (weight, label) records, compared as raw bits (NaN weights too)
        gv = np.ascontiguousarray(gv).view(np.uint64)
        wv = np.ascontiguousarray(wv).view(np.uint64)
    if sr == "plus_times_f64":
        err = np.abs(gv - wv)
        bad = err > tol * ab
        assert not bad.any(), f"fp64 tolerance exceeded at {np.nonzero(bad)[0][:5]}: " \
                              f"{gv[bad][:5]} vs {wv[bad][:5]}"
        return float(np.max(err / np.where(ab > 0, ab, 1.0))) if err.size else 0.0
    assert np.array_equal(gv, wv), _first_diff("val", gv, wv)
    return 0.0


def _first_diff(name, a, b):
    if a.shape != b.shape:
        return f"{name}: shape {a.shape} vs {b.shape}"
    i = np.nonzero(a != b)[0]
    return f"{name}: first difference at {i[:5]}: {a[i[:5]]} vs {b[i[:5]]}"


def check_structure(rp, col, ncols):
    """Properties that hold at any size: monotone row pointers, columns in
    range and strictly increasing inside each row."""
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0)
    assert col.size == rp[-1]
    if col.size:
        assert col.min() >= 0 and col.max() < ncols
        d = np.diff(col.astype(np.int64))
        starts = rp[1:-1]
        boundary = np.zeros(col.size - 1, dtype=bool) if col.size > 1 else np.zeros(0, bool)
        inner = starts[(starts > 0) & (starts < col.size)] - 1
        boundary[inner] = True
        assert np.all((d > 0) | boundary), "columns not strictly increasing inside a row"


def sample_rows(m, flops, frac=0.01, top=100, seed=0):
    """A seeded fraction of the rows plus the `top` rows with most products."""
    rng = np.random.default_rng(seed)
    k = max(1, int(m * frac))
    pick = rng.choice(m, size=min(k, m), replace=False)
    heavy = np.argsort(-np.asarray(flops), kind="stable")[:top]
    return np.unique(np.concatenate([pick, heavy])).astype(np.int64)


# ---------------------------------------------------------------------------
# per-product digests (the definition cb.h states for cb_opts.digests),
# computed here from host arrays, e.g. the oracle's output
# ---------------------------------------------------------------------------

_U = np.uint64


def _sm64(x):
    """splitmix64 output function on uint64 arrays (wrapping arithmetic)."""
    x = x + _U(0x9E3779B97F4A7C15)
    x = (x ^ (x >> _U(30))) * _U(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> _U(27))) * _U(0x94D049BB133111EB)
    return x ^ (x >> _U(31))


def digest(sr, rp, col, val):
    """(D0, V): the pattern/value digest word, and for (+,x) fp64 the weighted
    checksum V = sum v * w(r, c) (the exactly rounded sum of the rounded
    terms; None for the other semirings)."""
    import math
    rp = np.asarray(rp, dtype=np.int64)
    n = rp.size - 1
    lens = np.diff(rp)
    with np.errstate(over="ignore"):
        r = np.arange(n, dtype=np.uint64)
        d = np.sum(_sm64(_sm64(_U(2) * r) + lens.astype(np.uint64)), dtype=np.uint64)
        row_of = np.repeat(r, lens)
        j = (np.arange(col.size, dtype=np.int64) - np.repeat(rp[:-1], lens)).astype(np.uint64)
        hr = _sm64(_U(2) * row_of + _U(1))
        c = np.asarray(col, dtype=np.int64).astype(np.uint64)
        f64 = sr == "plus_times_f64"
        if f64:
            bits = _U(0)
        else:
            v = np.ascontiguousarray(val)
            bits = v.view({1: np.uint8, 4: np.uint32, 8: np.uint64}[v.dtype.itemsize]).astype(np.uint64)
        d = d + np.sum(_sm64(_sm64(_sm64(hr + j) + c) + bits), dtype=np.uint64)
        V = None
        if f64:
            w = 1.0 + (_sm64(hr ^ c) >> _U(11)).astype(np.float64) * 2.0 ** -53
            V = exact_sum(np.asarray(val, dtype=np.float64) * w)
    return int(d), V


def exact_sum(x):
    """The sum of a float64 array, rounded once (up to a few ulps of |sum| in
    total): a pairwise tree whose every addition's rounding error is kept
    (TwoSum, Knuth) and summed separately, the level sums then combined by
    math.fsum."""
    import math
    x = np.asarray(x, dtype=np.float64)
    parts = []
    while x.size > 1:
        if x.size % 2:
            x = np.append(x, 0.0)
        a, b = x[0::2], x[1::2]
        s = a + b
        bb = s - a
        parts.append(float(np.sum((a - (s - bb)) + (b - bb))))
        x = s
    return math.fsum(([float(x[0])] if x.size else []) + parts)


def digest_words(dig, i):
    """Product i's two words from the digests copied to the host (int64 numpy
    array of 2 * count entries), as (unsigned D0, float V)."""
    w = np.ascontiguousarray(dig[2 * i:2 * i + 2], dtype=np.int64)
    return int(w[:1].view(np.uint64)[0]), float(w[1:].view(np.float64)[0])


# |V_gpu - V_ref| <= (2 * 1e-12 + 40 u) * sum of the oracle's |a b| sums: each
# entry is within 1e-12 sum|ab| (R4) and weighted by w < 2 (so |v w| <= 2
# sum|ab|), plus the rounding of the weighted terms (u each side), of the
# device's compensated sum (<= 16 u sum|v w|) and of exact_sum (a few u |V|).
CHECKSUM_TOL = 2 * FP64_TOL + 40 * 2.0 ** -53
