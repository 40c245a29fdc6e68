"""Pins of the oracle's heterogeneous semiring (paper Sec. 1: operations over
three value types, two for the inputs and one for the output).

maxw_label: A holds float32 weights, B int32 labels, C (weight, label)
records; (x)(w, l) = (w, l); (+) keeps the larger weight in IEEE 754
totalOrder, and of equal weights the smaller label.

The pins do not reuse oracle.cpp's comparison: a dense brute force over
Python floats with a case-by-case totalOrder key (sign, class, magnitude),
a numpy max over dense weight matrices, closed forms (equal weights reduce
to (select2nd, min); one-entry rows gather B's labels), the shared pattern
of every semiring, and a planted slip (ties resolved to the larger label)
that the brute force rejects.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.spmspv import spmspv as spmspv_oracle
from paper_2106_14402_gb300 import gen

SR = "maxw_label"


def total_key(w):
    """IEEE 754 totalOrder as a tuple: negative-signed values first, and
    among them larger classes (NaN > inf > finite) and magnitudes first."""
    bits = int(np.asarray(w, dtype=np.float32).view(np.uint32))   # the stored bits, NaN payload kept
    w = float(np.float32(w))
    neg = bits >> 31 == 1
    if math.isnan(w):
        cls, mag = 3, bits & 0x7FFFFF
    elif math.isinf(w):
        cls, mag = 2, 0.0
    else:
        cls, mag = 1, abs(w)
    return (0, -cls, -mag) if neg else (1, cls, mag)


def brute(A, B, lose_ties_to_larger=False):
    """Dense enumeration over Python values: for every (i, j) the stored
    pairs (A(i,k), B(k,j)); the winner is the heaviest weight, ties to the
    smaller label (or, for the planted slip, the larger)."""
    m, k = A.nrows, B.ncols
    out = {}
    for i in range(m):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            kk = int(A.col[p])
            w = A.val[p]                      # np.float32, bits kept
            for q in range(B.row_ptr[kk], B.row_ptr[kk + 1]):
                j = int(B.col[q])
                lab = int(B.val[q])
                cand = (total_key(w), -lab if not lose_ties_to_larger else lab, w, lab)
                cur = out.get((i, j))
                if cur is None or cand[:2] > cur[:2]:
                    out[(i, j)] = cand
    return {key: (v[2], v[3]) for key, v in out.items()}


def as_dict(res):
    rp, col, val, _ = res
    d = {}
    for i in range(rp.size - 1):
        for e in range(rp[i], rp[i + 1]):
            d[(i, int(col[e]))] = (val["w"][e], int(val["label"][e]))
    return d


def same(d1, d2):
    if d1.keys() != d2.keys():
        return False
    for key in d1:
        w1, l1 = d1[key]
        w2, l2 = d2[key]
        if np.float32(w1).view(np.uint32) != np.float32(w2).view(np.uint32) or l1 != l2:
            return False
    return True


def hetero_csr(m, n, density, seed, duplicates=False, shuffle=False):
    """A pattern (no values) with empty and full rows."""
    return gen.random_csr(m, n, density, seed, empty_rows=0.15, full_rows=0.05,
                          duplicates=duplicates, shuffle=shuffle)


def with_weights(M, seed, levels=4):
    return M.with_values(gen.hetero_values(SR, "A", M.nnz, seed, levels=levels))


def with_labels(M, seed, lo=0, hi=50):
    rng = np.random.default_rng(seed)
    return M.with_values(rng.integers(lo, hi, size=M.nnz).astype(np.int32))


@pytest.mark.parametrize("shape", [(1, 1, 1, 1.0), (6, 5, 7, 0.5), (20, 15, 25, 0.3), (3, 40, 2, 0.4)])
@pytest.mark.parametrize("levels", [0, 3])
def test_brute_force_small(shape, levels):
    m, n, k, d = shape
    A = with_weights(hetero_csr(m, n, d, seed=m + 3 * n), seed=11, levels=levels)
    B = with_labels(hetero_csr(n, k, d, seed=k + 5 * n), seed=12)
    got = as_dict(oracle.spgemm(SR, A, B))
    assert same(got, brute(A, B))


def test_duplicates_and_unsorted():
    A = with_weights(hetero_csr(30, 25, 0.2, seed=3, duplicates=True, shuffle=True), seed=4, levels=2)
    B = with_labels(hetero_csr(25, 35, 0.2, seed=5, duplicates=True, shuffle=True), seed=6, hi=5)
    assert same(as_dict(oracle.spgemm(SR, A, B)), brute(A, B))


def test_special_weights_follow_total_order():
    specials = np.array([-0.0, 0.0, np.inf, -np.inf, 1.5, -1.5, 3e-45, -3e-45], dtype=np.float32)
    nans = np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFFFFFFF], dtype=np.uint32).view(np.float32)
    pool = np.concatenate([specials, nans])
    M = hetero_csr(40, 12, 0.5, seed=21)
    rng = np.random.default_rng(22)
    A = M.with_values(pool[rng.integers(0, pool.size, M.nnz)])
    B = with_labels(hetero_csr(12, 30, 0.5, seed=23), seed=24, hi=4)
    assert same(as_dict(oracle.spgemm(SR, A, B)), brute(A, B))


def test_total_order_key_facts():
    # the order the reading states: -NaN < -inf < -1 < -0 < +0 < 1 < inf < +NaN
    seq = [np.uint32(0xFFC00000).view(np.float32), -np.inf, -1.0, -0.0, 0.0, 1.0, np.inf,
           np.uint32(0x7FC00000).view(np.float32)]
    keys = [total_key(w) for w in seq]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_planted_tie_slip_is_caught():
    A = with_weights(hetero_csr(25, 20, 0.4, seed=31), seed=32, levels=2)
    B = with_labels(hetero_csr(20, 25, 0.4, seed=33), seed=34, hi=100)
    got = as_dict(oracle.spgemm(SR, A, B))
    assert same(got, brute(A, B))
    assert not same(got, brute(A, B, lose_ties_to_larger=True))


def test_weight_is_the_masked_row_max():
    """C(i,j).w = max over k with B(k,j) stored of A(i,k) (finite weights), by
    a numpy max over dense matrices."""
    A = with_weights(hetero_csr(50, 40, 0.2, seed=41), seed=42, levels=0)
    B = with_labels(hetero_csr(40, 60, 0.2, seed=43), seed=44)
    Wa = np.full((50, 40), -np.inf)
    for i in range(50):
        for p in range(A.row_ptr[i], A.row_ptr[i + 1]):
            Wa[i, A.col[p]] = A.val[p]
    Pb = np.zeros((40, 60), bool)
    for kk in range(40):
        Pb[kk, B.col[B.row_ptr[kk]:B.row_ptr[kk + 1]]] = True
    dense = np.where(Pb[None, :, :], Wa[:, :, None], -np.inf).max(axis=1)
    rp, col, val, _ = oracle.spgemm(SR, A, B)
    for i in range(50):
        cols = col[rp[i]:rp[i + 1]]
        assert np.array_equal(val["w"][rp[i]:rp[i + 1]].astype(np.float64), dense[i, cols])
        assert np.all(np.isfinite(dense[i, cols]))
        others = np.setdiff1d(np.arange(60), cols)
        assert np.all(np.isneginf(dense[i, others]))


def test_equal_weights_reduce_to_select2nd_min():
    """With every weight equal, the label is min over k of B(k,j): the
    (select2nd, min) product."""
    P = hetero_csr(60, 50, 0.15, seed=51)
    A = P.with_values(np.full(P.nnz, 0.25, np.float32))
    B = with_labels(hetero_csr(50, 70, 0.15, seed=52), seed=53, lo=-1000, hi=1000)
    rp, col, val, _ = oracle.spgemm(SR, A, B)
    rp2, col2, val2, _ = oracle.spgemm("sel2nd_min_i32", P.with_values(np.ones(P.nnz, np.int32)), B)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    assert np.array_equal(val["label"], val2)
    assert np.all(val["w"] == np.float32(0.25))


def test_one_entry_rows_gather_labels():
    n, k = 30, 40
    B = with_labels(hetero_csr(n, k, 0.3, seed=61), seed=62)
    rng = np.random.default_rng(63)
    picks = rng.integers(0, n, 25)
    w = rng.random(25).astype(np.float32)
    A = gen.CSR(25, n, np.arange(26, dtype=np.int64), picks.astype(np.int32), w)
    rp, col, val, _ = oracle.spgemm(SR, A, B)
    for i, kk in enumerate(picks):
        lo, hi = B.row_ptr[kk], B.row_ptr[kk + 1]
        assert np.array_equal(col[rp[i]:rp[i + 1]], B.col[lo:hi])
        assert np.array_equal(val["label"][rp[i]:rp[i + 1]], B.val[lo:hi])
        assert np.all(val["w"][rp[i]:rp[i + 1]] == w[i])


def test_pattern_matches_the_other_semirings():
    P = hetero_csr(45, 35, 0.2, seed=71)
    Q = hetero_csr(35, 55, 0.2, seed=72)
    rp, col, _, _ = oracle.spgemm(SR, with_weights(P, 73), with_labels(Q, 74))
    rp2, col2, _, _ = oracle.spgemm("or_and_bool", P.with_values(np.ones(P.nnz, np.uint8)),
                                    Q.with_values(np.ones(Q.nnz, np.uint8)))
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_spmspv_oracle_agrees_with_one_row_spgemm():
    A = with_labels(hetero_csr(80, 90, 0.1, seed=81), seed=82)
    rng = np.random.default_rng(83)
    x_idx = rng.choice(80, 30, replace=False)
    x_val = gen.hetero_values(SR, "A", 30, 84, levels=3)
    y_idx, y_val, _ = spmspv_oracle(SR, A, x_idx, x_val)
    X = gen.CSR(1, 80, np.array([0, 30], np.int64), x_idx.astype(np.int32), x_val)
    rp, col, val, _ = oracle.spgemm(SR, X, A)
    assert np.array_equal(y_idx, col)
    assert np.array_equal(y_val.view(np.uint64), val.view(np.uint64))


def _record_parts(k, m, n, seed, levels=3, duplicates=False, shuffle=False):
    parts = []
    for l in range(k):
        P = gen.random_csr(m, n, 0.3, seed=seed + l, empty_rows=0.2, duplicates=duplicates,
                           shuffle=shuffle)
        rec = np.zeros(P.nnz, oracle.WLABEL)
        rec["w"] = gen.hetero_values(SR, "A", P.nnz, seed + 100 + l, levels=levels)
        rec["label"] = np.random.default_rng(seed + 200 + l).integers(0, 7, P.nnz)
        parts.append(P.with_values(rec))
    return parts


def test_merge_oracle_brute_force():
    """Merging (weight, label) records keeps per coordinate the heaviest
    weight (totalOrder) and then the smallest label: a dictionary walk."""
    parts = _record_parts(4, 12, 15, seed=900, duplicates=True, shuffle=True)
    want = {}
    for P in parts:
        for i in range(P.nrows):
            for q in range(P.row_ptr[i], P.row_ptr[i + 1]):
                rec = P.val[q]
                cand = (total_key(rec["w"]), -int(rec["label"]), rec["w"], int(rec["label"]))
                key = (i, int(P.col[q]))
                if key not in want or cand[:2] > want[key][:2]:
                    want[key] = cand
    got = as_dict(oracle.merge(SR, parts))
    assert same(got, {key: (v[2], v[3]) for key, v in want.items()})


def test_merge_of_partial_products_is_the_product():
    """Splitting the inner dimension into blocks and merging the partial
    products gives A.B, with the SpGEMM oracle on both sides."""
    A = with_weights(hetero_csr(40, 60, 0.15, seed=910), seed=911, levels=3)
    B = with_labels(hetero_csr(60, 50, 0.15, seed=912), seed=913, hi=9)
    cuts = [0, 13, 31, 60]
    parts = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        keep = (A.col >= lo) & (A.col < hi)
        rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))[keep]
        rp = np.zeros(A.nrows + 1, np.int64)
        np.add.at(rp, rows + 1, 1)
        L = gen.CSR(A.nrows, A.ncols, np.cumsum(rp), A.col[keep], A.val[keep])
        prp, pcol, pval, _ = oracle.spgemm(SR, L, B)
        parts.append(gen.CSR(A.nrows, B.ncols, prp, pcol, pval))
    merged = oracle.merge(SR, parts)
    full = oracle.spgemm(SR, A, B)
    assert np.array_equal(merged[0], full[0]) and np.array_equal(merged[1], full[1])
    assert np.array_equal(merged[2].view(np.uint64), full[2].view(np.uint64))


def test_golden_worked_example():
    """The hand-derived example in tests/golden/maxw_label_example.json
    (derivation in its "about" field), bit for bit, -0.0 included."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "maxw_label_example.json")))
    A = gen.CSR(*g["A"]["shape"], np.array(g["A"]["row_ptr"], np.int64), np.array(g["A"]["col"], np.int32),
                np.array(g["A"]["val"], np.float32))
    B = gen.CSR(*g["B"]["shape"], np.array(g["B"]["row_ptr"], np.int64), np.array(g["B"]["col"], np.int32),
                np.array(g["B"]["val"], np.int32))
    rp, col, val, _ = oracle.spgemm(SR, A, B)
    assert np.array_equal(rp, g["C"]["row_ptr"]) and np.array_equal(col, g["C"]["col"])
    want_w = np.array(g["C"]["w"], np.float32)
    assert np.array_equal(val["w"].view(np.uint32), want_w.view(np.uint32))
    assert np.array_equal(val["label"], g["C"]["label"])
    assert same(as_dict((rp, col, val, None)), brute(A, B))
