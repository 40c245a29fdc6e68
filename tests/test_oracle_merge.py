"""Pins of the merge oracle (the semiring sum of k partial results), CPU only.

- brute force: a dictionary over coordinates with exact Python arithmetic;
- distributivity: splitting the inner dimension of A.B into k blocks and
  merging the k partial products gives A.B (SpGEMM oracle, independent code);
- the semiring laws: an idempotent (+) merges a matrix with itself into
  itself, (+,x) int64 doubles it; merging is associative and commutative;
- k = 1 of a sorted, duplicate-free matrix is that matrix.
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

SR = gen.SEMIRINGS
MASK64 = (1 << 64) - 1


def _wrap64(x):
    x &= MASK64
    return x - (1 << 64) if x >= 1 << 63 else x


def brute(sr, parts):
    acc = {}
    for P in parts:
        for i in range(P.nrows):
            for q in range(P.row_ptr[i], P.row_ptr[i + 1]):
                key = (i, int(P.col[q]))
                v = P.val[q]
                v = float(v) if sr == "plus_times_f64" else int(v)
                if key not in acc:
                    acc[key] = (1 if v else 0) if sr == "or_and_bool" else v
                elif sr == "plus_times_i64":
                    acc[key] = _wrap64(acc[key] + v)
                elif sr == "plus_times_f64":
                    acc[key] += v
                elif sr == "or_and_bool":
                    acc[key] = 1 if (acc[key] or v) else 0
                else:
                    acc[key] = min(acc[key], v)
    return acc


def as_dict(res):
    rp, col, val = res[:3]
    out = {}
    for i in range(rp.size - 1):
        for q in range(rp[i], rp[i + 1]):
            out[(i, int(col[q]))] = val[q]
    return out


@pytest.mark.parametrize("sr", SR)
def test_matches_brute_force(sr):
    parts = [gen.random_csr(9, 11, 0.3, seed=100 + k, semiring=sr, duplicates=True, shuffle=True,
                            empty_rows=0.2) for k in range(3)]
    got = oracle.merge(sr, parts)
    rp, col = got[0], got[1]
    for i in range(9):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    want = brute(sr, parts)
    g = as_dict(got)
    assert set(g) == set(want)
    for k, v in want.items():
        if sr == "plus_times_f64":
            assert abs(g[k] - v) <= 1e-12 * max(1.0, abs(v))
        else:
            assert int(g[k]) == v, (k, g[k], v)


def _column_block(A, lo, hi):
    """A restricted to columns [lo, hi) (same shape)."""
    keep = (A.col >= lo) & (A.col < hi)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))[keep]
    rp = np.zeros(A.nrows + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return gen.CSR(A.nrows, A.ncols, np.cumsum(rp), A.col[keep], A.val[keep])


def _row_block(B, lo, hi):
    """B restricted to rows [lo, hi) (same shape)."""
    lens = np.diff(B.row_ptr).copy()
    lens[:lo] = 0
    lens[hi:] = 0
    rp = np.zeros(B.nrows + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    s, e = B.row_ptr[lo], B.row_ptr[hi]
    return gen.CSR(B.nrows, B.ncols, rp, B.col[s:e], B.val[s:e])


@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("k", [1, 3, 8])
def test_partial_products_merge_to_the_product(sr, k):
    A = gen.random_csr(60, 48, 0.15, seed=7, semiring=sr, empty_rows=0.1)
    B = gen.random_csr(48, 70, 0.15, seed=8, semiring=sr, empty_rows=0.1)
    cuts = np.linspace(0, 48, k + 1).astype(int)
    parts = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        rp, col, val, _ = oracle.spgemm(sr, _column_block(A, lo, hi), _row_block(B, lo, hi))
        parts.append(gen.CSR(A.nrows, B.ncols, rp, col, val))
    got = oracle.merge(sr, parts)
    compare_rows(sr, got[:3], oracle.spgemm(sr, A, B))


@pytest.mark.parametrize("sr", SR)
def test_semiring_laws(sr):
    P = gen.random_csr(30, 25, 0.2, seed=20, semiring=sr)
    Q = gen.random_csr(30, 25, 0.2, seed=21, semiring=sr)
    R = gen.random_csr(30, 25, 0.2, seed=22, semiring=sr)
    one = oracle.merge(sr, [P])
    assert np.array_equal(one[0], P.row_ptr) and np.array_equal(one[1], P.col)
    assert np.array_equal(one[2], P.val)
    twice = oracle.merge(sr, [P, P])
    assert np.array_equal(twice[1], P.col)
    if sr == "plus_times_i64":
        assert np.array_equal(twice[2], P.val * 2)
    elif sr != "plus_times_f64":
        assert np.array_equal(twice[2], P.val)
    if sr != "plus_times_f64":
        pqr = oracle.merge(sr, [P, Q, R])
        left = oracle.merge(sr, [gen.CSR(30, 25, *oracle.merge(sr, [P, Q])[:3]), R])
        qp = oracle.merge(sr, [Q, P, R])
        for x, y, z in zip(pqr[:3], left[:3], qp[:3]):
            assert np.array_equal(x, y) and np.array_equal(x, z)
