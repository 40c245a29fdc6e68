"""Pins of the SpMSpV oracle (y^T = x^T A), CPU only.

- the SpGEMM oracle (independent C++ code) on x as a one-row matrix;
- brute force with exact Python arithmetic on tiny inputs;
- textbook reductions: one BFS level expansion on (or,and) is the union of
  the frontier's neighbour sets; on (min,+) one Bellman-Ford relaxation from
  a distance vector, written as a separate edge loop.
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

SR = gen.SEMIRINGS


def as_row(n, idx, val):
    return gen.CSR(1, n, np.array([0, idx.size], np.int64), idx.astype(np.int32), val)


@pytest.mark.parametrize("sr", SR)
def test_matches_spgemm_oracle_on_a_one_row_matrix(sr):
    A = gen.random_csr(80, 120, 0.08, seed=4, semiring=sr, duplicates=True, shuffle=True, empty_rows=0.2)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 80, 30)                      # unsorted, with duplicates
    val = gen.random_values(sr, 30, 6)
    y = oracle.spmspv(sr, A, idx, val)
    rp, col, v, ab = oracle.spgemm(sr, as_row(80, idx, val), A)
    compare_rows(sr, (np.array([0, y[0].size]), y[0], y[1]), (rp, col, v, ab))


@pytest.mark.parametrize("sr", SR)
def test_brute_force(sr):
    A = gen.random_csr(9, 7, 0.4, seed=7, semiring=sr, duplicates=True)
    idx = np.array([3, 0, 3, 8, 5])
    val = gen.random_values(sr, 5, 8)
    acc = {}
    for p in range(idx.size):
        i = idx[p]
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            c = int(A.col[q])
            a, b = val[p], A.val[q]
            if sr == "plus_times_i64":
                prod = (int(a) * int(b)) & ((1 << 64) - 1)
            elif sr == "plus_times_f64":
                prod = float(a) * float(b)
            elif sr == "min_plus_u32":
                prod = min(int(a) + int(b), 0xFFFFFFFF)
            elif sr == "or_and_bool":
                prod = int(bool(a) and bool(b))
            else:
                prod = int(b)
            if c not in acc:
                acc[c] = prod
            elif sr == "plus_times_i64":
                acc[c] = (acc[c] + prod) & ((1 << 64) - 1)
            elif sr == "plus_times_f64":
                acc[c] += prod
            elif sr == "or_and_bool":
                acc[c] = acc[c] | prod
            else:
                acc[c] = min(acc[c], prod)
    yi, yv, _ = oracle.spmspv(sr, A, idx, val)
    assert list(yi) == sorted(acc)
    for c, v in zip(yi, yv):
        w = acc[int(c)]
        if sr == "plus_times_i64":
            assert int(np.int64(v)) & ((1 << 64) - 1) == w
        elif sr == "plus_times_f64":
            assert abs(v - w) <= 1e-12 * max(1.0, abs(w))
        else:
            assert int(v) == w


def test_bfs_level_and_bellman_ford_step():
    P = gen.rmat(9, 8, *gen.RMAT_ABCD, seed=9)
    edges = [(i, int(P.col[q])) for i in range(P.nrows) for q in range(P.row_ptr[i], P.row_ptr[i + 1])]
    frontier = np.array([1, 7, 30, 200, 511])
    # BFS: the neighbours of the frontier
    yi, yv, _ = oracle.spmspv("or_and_bool", P.with_values(np.ones(P.nnz, np.uint8)), frontier,
                              np.ones(frontier.size, np.uint8))
    want = sorted({j for i, j in edges if i in set(frontier.tolist())})
    assert list(yi) == want and np.all(yv == 1)
    # Bellman-Ford: one relaxation from distances d on the frontier
    w = gen.random_values("min_plus_u32", P.nnz, 10)
    d = np.array([0, 5, 17, 2, 9], np.uint32)
    yi, yv, _ = oracle.spmspv("min_plus_u32", P.with_values(w), frontier, d)
    best = {}
    pos = 0
    for i in range(P.nrows):
        for q in range(P.row_ptr[i], P.row_ptr[i + 1]):
            if i in frontier:
                dist = int(d[list(frontier).index(i)]) + int(w[q])
                j = int(P.col[q])
                best[j] = min(best.get(j, 1 << 40), dist)
    assert list(yi) == sorted(best)
    assert [int(v) for v in yv] == [best[int(j)] for j in yi]
