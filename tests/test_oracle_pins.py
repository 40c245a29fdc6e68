"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of oracle.cpp's own formulation (ordered map per
row, Gustavson order): dense brute force over Python integers, enumeration
of stored entry pairs, closed forms (identity, permutation, one-entry rows),
algebraic laws (associativity, distributivity, transposition), a textbook
reduction ((min,+) squaring is one Bellman-Ford relaxation), a library
cross-check (scipy), and a hand-derived worked example under tests/golden/.
A plausible slip in the oracle (a dropped product, a wrong index, a
transposed operand, a non-saturating add, an order-dependent reduction)
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen

SR = oracle.SEMIRINGS
EXACT = ("plus_times_i64", "min_plus_u32", "or_and_bool", "sel2nd_min_i32")
U32MAX = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# independent restatements (Python integers / floats, entry-pair enumeration)
# ----------------------------------------------------------------------------

def _mul(sr, a, b):
    if sr == "plus_times_i64":
        return int(a) * int(b)                 # exact; wrapped at the end
    if sr == "plus_times_f64":
        return float(a) * float(b)
    if sr == "min_plus_u32":
        return min(int(a) + int(b), U32MAX)
    if sr == "or_and_bool":
        return bool(a) and bool(b)
    return int(b)                              # select2nd


def _add(sr, x, y):
    if sr in ("plus_times_i64", "plus_times_f64"):
        return x + y
    if sr == "or_and_bool":
        return x or y
    return min(x, y)


def _finish(sr, x):
    if sr == "plus_times_i64":
        x &= (1 << 64) - 1
        return x - (1 << 64) if x >= (1 << 63) else x
    if sr == "or_and_bool":
        return 1 if x else 0
    return x


def pairs_product(sr, A, B):
    """Dict (i,j) -> (value, sum|products|) by enumerating every stored pair (a in A, b in B)."""
    out = {}
    arows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    brows = np.repeat(np.arange(B.nrows), np.diff(B.row_ptr))
    by_k = {}
    for q in range(B.nnz):
        by_k.setdefault(int(brows[q]), []).append(q)
    for p in range(A.nnz):
        i, k = int(arows[p]), int(A.col[p])
        for q in by_k.get(k, []):
            j = int(B.col[q])
            v = _mul(sr, A.val[p], B.val[q])
            if (i, j) in out:
                x, s = out[(i, j)]
                out[(i, j)] = (_add(sr, x, v), s + abs(float(v)))
            else:
                out[(i, j)] = (v, abs(float(v)))
    return {key: (_finish(sr, v), s) for key, (v, s) in out.items()}


def dense_product(sr, A, B):
    """Dense triple loop over a stored-mask; requires no duplicate coordinates."""
    m, n, k = A.nrows, A.ncols, B.ncols
    Am = np.zeros((m, n), bool)
    Bm = np.zeros((n, k), bool)
    Av = np.zeros((m, n), object)
    Bv = np.zeros((n, k), object)
    for i in range(m):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            Am[i, A.col[p]] = True
            Av[i, A.col[p]] = A.val[p]
    for r in range(n):
        for q in range(B.row_ptr[r], B.row_ptr[r + 1]):
            Bm[r, B.col[q]] = True
            Bv[r, B.col[q]] = B.val[q]
    out = {}
    for i in range(m):
        for j in range(k):
            acc, s, hit = None, 0.0, False
            for t in range(n):
                if Am[i, t] and Bm[t, j]:
                    v = _mul(sr, Av[i, t], Bv[t, j])
                    acc = v if not hit else _add(sr, acc, v)
                    s += abs(float(v))
                    hit = True
            if hit:
                out[(i, j)] = (_finish(sr, acc), s)
    return out


def to_dict(rp, col, val, absum, rows=None):
    out = {}
    rows = np.arange(len(rp) - 1) if rows is None else rows
    for r, i in enumerate(rows):
        for p in range(rp[r], rp[r + 1]):
            out[(int(i), int(col[p]))] = (val[p].item(), float(absum[p]))
    return out


def assert_same(sr, got, want, tol=1e-12):
    assert set(got) == set(want), f"pattern differs: {len(set(got) ^ set(want))} entries"
    for key, (v, _) in got.items():
        w, s = want[key]
        if sr == "plus_times_f64":
            assert abs(v - w) <= tol * s + 1e-300, (key, v, w, s)
        else:
            assert int(v) == int(w), (key, v, w)


def check_sorted_unique(rp, col):
    for r in range(len(rp) - 1):
        c = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c.astype(np.int64)) > 0)


def tiny_cases():
    cases = []
    for seed, (m, n, k, dens) in enumerate([(1, 1, 1, 1.0), (5, 7, 3, 0.4), (17, 13, 19, 0.2),
                                            (24, 24, 24, 0.15), (9, 30, 2, 0.5), (12, 1, 12, 0.7)]):
        cases.append((seed, m, n, k, dens))
    return cases


# ----------------------------------------------------------------------------
# brute force
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("case", tiny_cases())
def test_dense_brute_force(sr, case):
    seed, m, n, k, dens = case
    A = gen.random_csr(m, n, dens, seed=100 + seed, semiring=sr, empty_rows=0.2, full_rows=0.1)
    B = gen.random_csr(n, k, dens, seed=200 + seed, semiring=sr, empty_rows=0.2, full_rows=0.1)
    rp, col, val, ab = oracle.spgemm(sr, A, B)
    check_sorted_unique(rp, col)
    assert_same(sr, to_dict(rp, col, val, ab), dense_product(sr, A, B))


@pytest.mark.parametrize("sr", SR)
def test_explicit_zeros_are_structural(sr):
    # Values drawn from {0,1} (bool) / include zeros: entries stay even when their value is 0.
    lo, hi = {"plus_times_i64": (-2, 2), "plus_times_f64": (-1.0, 1.0), "min_plus_u32": (0, 3),
              "or_and_bool": (0, 1), "sel2nd_min_i32": (-3, 3)}[sr]
    A = gen.random_csr(15, 11, 0.3, seed=7, semiring=sr, lo=lo, hi=hi)
    B = gen.random_csr(11, 13, 0.3, seed=8, semiring=sr, lo=lo, hi=hi)
    if sr == "plus_times_i64":
        A.val[::3] = 0
    rp, col, val, ab = oracle.spgemm(sr, A, B)
    assert_same(sr, to_dict(rp, col, val, ab), dense_product(sr, A, B))


@pytest.mark.parametrize("sr", SR)
def test_duplicates_and_unsorted_inputs(sr):
    A = gen.random_csr(20, 16, 0.25, seed=11, semiring=sr, duplicates=True, shuffle=True)
    B = gen.random_csr(16, 18, 0.25, seed=12, semiring=sr, duplicates=True, shuffle=True)
    rp, col, val, ab = oracle.spgemm(sr, A, B)
    check_sorted_unique(rp, col)
    assert_same(sr, to_dict(rp, col, val, ab), pairs_product(sr, A, B))


def test_int64_wraps_and_u32_saturates():
    A = gen.random_csr(6, 5, 0.8, seed=21, semiring="plus_times_i64", lo=(1 << 61), hi=(1 << 62))
    B = gen.random_csr(5, 6, 0.8, seed=22, semiring="plus_times_i64", lo=-(1 << 62), hi=(1 << 62))
    rp, col, val, ab = oracle.spgemm("plus_times_i64", A, B)
    assert_same("plus_times_i64", to_dict(rp, col, val, ab), dense_product("plus_times_i64", A, B))
    A = gen.random_csr(6, 5, 0.8, seed=23, semiring="min_plus_u32", lo=U32MAX - 10, hi=U32MAX)
    B = gen.random_csr(5, 6, 0.8, seed=24, semiring="min_plus_u32", lo=0, hi=20)
    rp, col, val, ab = oracle.spgemm("min_plus_u32", A, B)
    d = dense_product("min_plus_u32", A, B)
    assert_same("min_plus_u32", to_dict(rp, col, val, ab), d)
    assert any(v == U32MAX for v, _ in d.values())        # the case really saturates


def test_row_stats_against_pair_count():
    A = gen.random_csr(30, 25, 0.2, seed=31, duplicates=True)
    B = gen.random_csr(25, 40, 0.2, seed=32, duplicates=True)
    flops, maxb = oracle.row_stats(A, B)
    blen = np.diff(B.row_ptr)
    for i in range(A.nrows):
        ks = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert flops[i] == sum(int(blen[k]) for k in ks)
        assert maxb[i] == (max(int(blen[k]) for k in ks) if len(ks) else 0)


# ----------------------------------------------------------------------------
# closed forms and special cases
# ----------------------------------------------------------------------------

ONE = {"plus_times_i64": 1, "plus_times_f64": 1.0, "min_plus_u32": 0, "or_and_bool": 1,
       "sel2nd_min_i32": 0}


def identity(n, sr):
    return gen.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32),
                   np.full(n, ONE[sr], dtype=gen.VALUE_DTYPE[sr]))


@pytest.mark.parametrize("sr", SR)
def test_identity(sr):
    A = gen.random_csr(23, 19, 0.3, seed=41, semiring=sr, empty_rows=0.2)
    rp, col, val, _ = oracle.spgemm(sr, identity(23, sr), A)           # I.A = A
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)
    rp, col, val, _ = oracle.spgemm(sr, A, identity(19, sr))           # A.I = A (select2nd: I's value)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    want = A.val if sr != "sel2nd_min_i32" else np.zeros_like(A.val)
    assert np.array_equal(val, want)


@pytest.mark.parametrize("sr", SR)
def test_permutation_gathers_rows(sr):
    B = gen.random_csr(31, 27, 0.25, seed=42, semiring=sr, empty_rows=0.1)
    perm = gen.rng_for(43).permutation(31)
    P = gen.CSR(31, 31, np.arange(32, dtype=np.int64), perm.astype(np.int32),
                np.full(31, ONE[sr], dtype=gen.VALUE_DTYPE[sr]))
    rp, col, val, _ = oracle.spgemm(sr, P, B)
    for i in range(31):
        s, e = B.row_ptr[perm[i]], B.row_ptr[perm[i] + 1]
        assert np.array_equal(col[rp[i]:rp[i + 1]], B.col[s:e])
        assert np.array_equal(val[rp[i]:rp[i + 1]], B.val[s:e])


@pytest.mark.parametrize("sr", SR)
def test_one_entry_rows_give_scaled_gather(sr):
    A = gen.er_exact(40, 35, 1, seed=44)
    A = A.with_values(gen.random_values(sr, A.nnz, 45))
    B = gen.random_csr(35, 50, 0.2, seed=46, semiring=sr)
    rp, col, val, _ = oracle.spgemm(sr, A, B)
    flops, _ = oracle.row_stats(A, B)
    assert np.array_equal(np.diff(rp), flops)                          # nnz(C_i) = flops_i
    for i in range(40):
        k = A.col[i]
        s, e = B.row_ptr[k], B.row_ptr[k + 1]
        assert np.array_equal(col[rp[i]:rp[i + 1]], B.col[s:e])
        want = [_finish(sr, _mul(sr, A.val[i], b)) for b in B.val[s:e]]
        assert [v.item() for v in val[rp[i]:rp[i + 1]]] == pytest.approx(want, rel=0, abs=0)


def test_select2nd_ignores_a_values():
    A = gen.random_csr(25, 20, 0.3, seed=47, semiring="sel2nd_min_i32")
    B = gen.random_csr(20, 22, 0.3, seed=48, semiring="sel2nd_min_i32")
    r1 = oracle.spgemm("sel2nd_min_i32", A, B)
    A2 = A.with_values(gen.random_values("sel2nd_min_i32", A.nnz, 49))
    r2 = oracle.spgemm("sel2nd_min_i32", A2, B)
    for x, y in zip(r1[:3], r2[:3]):
        assert np.array_equal(x, y)


# ----------------------------------------------------------------------------
# invariants and laws
# ----------------------------------------------------------------------------

def test_size_bounds_and_shared_pattern():
    P = gen.rmat(9, 8, *gen.RMAT_ABCD, seed=50)
    flops, maxb = oracle.row_stats(P, P)
    pats = []
    for sr in SR:
        A = P.with_values(gen.random_values(sr, P.nnz, 51))
        rp, col, val, _ = oracle.spgemm(sr, A, A)
        nz = np.diff(rp)
        assert nz.sum() <= flops.sum()
        assert np.all(nz >= maxb) and np.all(nz <= np.minimum(flops, P.ncols))
        pats.append((rp, col))
        if sr == "or_and_bool":
            assert np.all(val == 1)
    for rp, col in pats[1:]:
        assert np.array_equal(rp, pats[0][0]) and np.array_equal(col, pats[0][1])


def _csr_of(d, m, k, dt):
    keys = sorted(d)
    rows = np.array([i for i, _ in keys], dtype=np.int64)
    counts = np.bincount(rows, minlength=m) if keys else np.zeros(m, np.int64)
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    return gen.CSR(m, k, rp, np.array([j for _, j in keys], dtype=np.int32),
                   np.array([d[x][0] for x in keys], dtype=dt))


@pytest.mark.parametrize("sr", EXACT)
def test_associativity(sr):
    dt = gen.VALUE_DTYPE[sr]
    A = gen.random_csr(14, 12, 0.25, seed=52, semiring=sr)
    B = gen.random_csr(12, 15, 0.25, seed=53, semiring=sr)
    Cm = gen.random_csr(15, 11, 0.25, seed=54, semiring=sr)
    AB = _csr_of(to_dict(*oracle.spgemm(sr, A, B)), 14, 15, dt)
    BC = _csr_of(to_dict(*oracle.spgemm(sr, B, Cm)), 12, 11, dt)
    left = to_dict(*oracle.spgemm(sr, AB, Cm))
    right = to_dict(*oracle.spgemm(sr, A, BC))
    assert_same(sr, left, right)


@pytest.mark.parametrize("sr", EXACT)
def test_distributivity(sr):
    dt = gen.VALUE_DTYPE[sr]
    A = gen.random_csr(13, 10, 0.3, seed=55, semiring=sr)
    B1 = gen.random_csr(10, 12, 0.25, seed=56, semiring=sr)
    B2 = gen.random_csr(10, 12, 0.25, seed=57, semiring=sr)
    d1 = to_dict(*oracle.spgemm(sr, A, B1))
    d2 = to_dict(*oracle.spgemm(sr, A, B2))
    # B1 (+) B2 elementwise on the union pattern.
    dB = to_dict(B1.row_ptr, B1.col, B1.val, np.zeros(B1.nnz))
    for key, v in to_dict(B2.row_ptr, B2.col, B2.val, np.zeros(B2.nnz)).items():
        dB[key] = (_finish(sr, _add(sr, dB[key][0], v[0])), 0.0) if key in dB else v
    Bs = _csr_of(dB, 10, 12, dt)
    lhs = to_dict(*oracle.spgemm(sr, A, Bs))
    rhs = dict(d1)
    for key, v in d2.items():
        rhs[key] = (_finish(sr, _add(sr, rhs[key][0], v[0])), 0.0) if key in rhs else v
    assert_same(sr, lhs, rhs)


def _transpose(M):
    d = to_dict(M.row_ptr, M.col, M.val, np.zeros(M.nnz))
    return _csr_of({(j, i): v for (i, j), v in d.items()}, M.ncols, M.nrows, M.val.dtype)


@pytest.mark.parametrize("sr", ("plus_times_i64", "plus_times_f64", "min_plus_u32", "or_and_bool"))
def test_transposition(sr):
    A = gen.random_csr(16, 14, 0.25, seed=58, semiring=sr)
    B = gen.random_csr(14, 17, 0.25, seed=59, semiring=sr)
    C = to_dict(*oracle.spgemm(sr, A, B))
    Ct = to_dict(*oracle.spgemm(sr, _transpose(B), _transpose(A)))
    assert_same(sr, {(j, i): v for (i, j), v in C.items()}, Ct)


def test_min_plus_is_one_bellman_ford_step():
    A = gen.rmat(8, 6, *gen.RMAT_ABCD, seed=60)
    A = A.with_values(gen.random_values("min_plus_u32", A.nnz, 61))
    rp, col, val, _ = oracle.spgemm("min_plus_u32", A, A)
    # Edge list relaxation: from each source s, distances after exactly two hops.
    src = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    edges = list(zip(src.tolist(), A.col.tolist(), A.val.tolist()))
    for s in range(0, A.nrows, 7):
        d1 = {int(v): int(w) for (u, v, w) in edges if u == s}
        d2 = {}
        for (u, v, w) in edges:
            if u in d1:
                cand = min(d1[u] + w, U32MAX)
                d2[v] = min(d2.get(v, U32MAX + 1), cand)
        got = {int(col[p]): int(val[p]) for p in range(rp[s], rp[s + 1])}
        assert got == d2


@pytest.mark.parametrize("sr", ("plus_times_i64", "plus_times_f64"))
def test_scipy_cross_check(sr):
    sp = pytest.importorskip("scipy.sparse")
    P = gen.rmat(10, 8, *gen.RMAT_ABCD, seed=62)
    lo, hi = (-5, 5) if sr == "plus_times_i64" else (-1.0, 1.0)
    A = P.with_values(gen.random_values(sr, P.nnz, 63, lo, hi))
    rp, col, val, ab = oracle.spgemm(sr, A, A)
    S = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.nrows, A.ncols))
    T = (S @ S).tocsr()
    T.sort_indices()
    dense_got = sp.csr_matrix((val, col, rp), shape=T.shape).toarray()
    if sr == "plus_times_i64":
        assert np.array_equal(dense_got, T.toarray())
    else:
        dense_abs = sp.csr_matrix((ab, col, rp), shape=T.shape).toarray()
        assert np.all(np.abs(dense_got - T.toarray()) <= 1e-12 * dense_abs + 1e-300)


# ----------------------------------------------------------------------------
# hand-derived worked example (tests/golden/)
# ----------------------------------------------------------------------------

def test_golden_worked_example():
    with open(os.path.join(GOLDEN, "two_hop_example.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        sr = case["semiring"]
        dt = gen.VALUE_DTYPE[sr]
        A = gen.CSR(*case["A"]["shape"], np.array(case["A"]["row_ptr"], np.int64),
                    np.array(case["A"]["col"], np.int32), np.array(case["A"]["val"], dt))
        B = gen.CSR(*case["B"]["shape"], np.array(case["B"]["row_ptr"], np.int64),
                    np.array(case["B"]["col"], np.int32), np.array(case["B"]["val"], dt))
        rp, col, val, _ = oracle.spgemm(sr, A, B)
        assert rp.tolist() == case["C"]["row_ptr"], sr
        assert col.tolist() == case["C"]["col"], sr
        assert [v.item() for v in val] == case["C"]["val"], sr


# ----------------------------------------------------------------------------
# the comparison itself catches planted slips (mutations of the oracle's output)
# ----------------------------------------------------------------------------

def test_planted_mistakes_are_caught():
    sr = "plus_times_i64"
    A = gen.random_csr(12, 10, 0.4, seed=70, semiring=sr)
    B = gen.random_csr(10, 10, 0.4, seed=71, semiring=sr)
    want = dense_product(sr, A, B)
    rp, col, val, ab = oracle.spgemm(sr, A, B)
    bad = val.copy()
    bad[len(bad) // 2] += 1                                             # a dropped/extra term
    with pytest.raises(AssertionError):
        assert_same(sr, to_dict(rp, col, bad, ab), want)
    BT = _transpose(B)                                                  # a transposed operand
    BT = gen.CSR(B.nrows, B.ncols, BT.row_ptr, BT.col, BT.val)
    with pytest.raises(AssertionError):
        assert_same(sr, to_dict(*oracle.spgemm(sr, A, BT)), want)


def test_counter_generator_rows_are_exact_degree_and_sorted():
    A = gen.er_counter(12345, 300, 257, 40)
    assert np.all(np.diff(A.row_ptr) == 40)
    for r in range(A.nrows):
        c = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(c.astype(np.int64)) > 0) and c.min() >= 0 and c.max() < 257
    v = gen.counter_values_u32(7, 1000, 1, 1000)
    assert v.min() >= 1 and v.max() <= 1000
    f = gen.counter_values_f64(8, 1000, -1.0, 1.0)
    assert f.min() >= -1.0 and f.max() < 1.0
    # the draw is the published splitmix64 output function of seed + golden * (c + 1)
    x = int(gen.counter_draw(0, np.array([0], np.uint64))[0])
    assert x == gen.splitmix64(0)
