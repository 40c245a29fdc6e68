"""Property-based pins of the oracle (hypothesis, CPU only): for random
small CSR inputs (any shape, density, duplicate coordinates, unsorted rows,
extreme values) the oracle's SpGEMM equals the enumeration of stored entry
pairs, its merge equals a dictionary walk, and its SpMSpV equals the SpGEMM
of a one-row matrix.  Skipped where hypothesis is not installed."""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from test_oracle_pins import assert_same, pairs_product, to_dict

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SR = oracle.SEMIRINGS
EXTREMES = {"plus_times_i64": (-(1 << 62), 1 << 62), "plus_times_f64": (-1.0, 1.0),
            "min_plus_u32": (0xFFFFFF00, 0xFFFFFFFF), "or_and_bool": (0, 1),
            "sel2nd_min_i32": (-(1 << 31), (1 << 31) - 1)}


@st.composite
def csr_pair(draw):
    sr = draw(st.sampled_from(SR))
    m = draw(st.integers(0, 9))
    n = draw(st.integers(1, 9))
    k = draw(st.integers(1, 9))
    d = draw(st.floats(0.0, 1.0))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    extreme = draw(st.booleans())
    lo, hi = EXTREMES[sr] if extreme else (None, None)
    kw = dict(semiring=sr, duplicates=draw(st.booleans()), shuffle=draw(st.booleans()),
              empty_rows=draw(st.floats(0.0, 0.5)), lo=lo, hi=hi)
    A = gen.random_csr(m, n, d, seed=seed, **kw)
    B = gen.random_csr(n, k, d, seed=seed + 1, **kw)
    return sr, A, B


@settings(max_examples=150, deadline=None)
@given(csr_pair())
def test_spgemm_equals_pair_enumeration(case):
    sr, A, B = case
    got = to_dict(*oracle.spgemm(sr, A, B))
    assert_same(sr, got, pairs_product(sr, A, B))


@settings(max_examples=60, deadline=None)
@given(csr_pair(), st.integers(1, 4))
def test_merge_equals_dictionary_walk(case, k):
    sr, A, _ = case
    parts = [A] + [gen.random_csr(A.nrows, A.ncols, 0.4, seed=900 + t, semiring=sr, duplicates=True,
                                  shuffle=True) for t in range(k - 1)]
    rp, col, val, ab = oracle.merge(sr, parts)
    got = to_dict(rp, col, val, ab)
    # the merge of parts is the product of [I I ... I] with the stacked parts
    # under (x) = select2nd, enumerated as pairs: each stored entry once
    want = {}
    for P in parts:
        rows = np.repeat(np.arange(P.nrows), np.diff(P.row_ptr))
        for q in range(int(P.row_ptr[-1])):
            key = (int(rows[q]), int(P.col[q]))
            v = P.val[q]
            v = float(v) if sr == "plus_times_f64" else int(v)
            if sr == "or_and_bool":
                v = 1 if v else 0
            if key not in want:
                want[key] = (v, abs(float(v)))
            else:
                x, s = want[key]
                if sr == "plus_times_i64":
                    x = (x + v + (1 << 63)) % (1 << 64) - (1 << 63)
                elif sr == "plus_times_f64":
                    x = x + v
                elif sr == "or_and_bool":
                    x = 1 if (x or v) else 0
                else:
                    x = min(x, v)
                want[key] = (x, s + abs(float(v)))
    assert_same(sr, got, want)


@settings(max_examples=60, deadline=None)
@given(csr_pair(), st.integers(0, 2 ** 31 - 1))
def test_spmspv_equals_one_row_spgemm(case, seed):
    sr, _, B = case
    rng = np.random.default_rng(seed)
    nx = int(rng.integers(0, 2 * B.nrows + 1))
    idx = rng.integers(0, B.nrows, nx)
    val = gen.random_values(sr, nx, seed % 1000)
    yi, yv, ya = oracle.spmspv(sr, B, idx, val)
    X = gen.CSR(1, B.nrows, np.array([0, nx], np.int64), idx.astype(np.int32), val)
    rp, col, cv, ca = oracle.spgemm(sr, X, B)
    assert np.array_equal(yi, col)
    if sr == "plus_times_f64":
        assert np.all(np.abs(yv - cv) <= 1e-12 * ca + 1e-300)
    else:
        assert np.array_equal(yv, cv)
