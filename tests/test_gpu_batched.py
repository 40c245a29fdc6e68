"""Column-batched SpGEMM (paper Sec. 7.2): C is formed in column ranges that
each fit an output budget; reassembled, the batches must equal the oracle's
C bit for bit (fp64 within the per-entry bound)."""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def run_batches(cb, sr, A, B, budget, stop_after=None, **kw):
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = dA if B is A else cb.DeviceCSR.from_host(B, sr)
    got = []

    def on_batch(b, lo, hi, Cb):
        rp, col, val = Cb.to_host()
        assert Cb.nrows == A.nrows
        if col.size:
            assert col.min() >= lo and col.max() < hi
        got.append((b, lo, hi, rp, col, val))
        return stop_after is not None and len(got) >= stop_after

    st = cb.spgemm_column_batches(sr, dA, dB, budget, on_batch, **kw)
    return got, st


def assemble(batches, m):
    """Merge batches (in column order) into one CSR."""
    batches = sorted(batches, key=lambda t: t[1])
    rows_col = [[] for _ in range(m)]
    rows_val = [[] for _ in range(m)]
    for _, lo, hi, rp, col, val in batches:
        for i in range(m):
            rows_col[i].append(col[rp[i]:rp[i + 1]])
            rows_val[i].append(val[rp[i]:rp[i + 1]])
    rp = np.zeros(m + 1, np.int64)
    rp[1:] = np.cumsum([sum(len(c) for c in rc) for rc in rows_col])
    col = np.concatenate([np.concatenate(rc) for rc in rows_col]) if m else np.zeros(0, np.int32)
    val = np.concatenate([np.concatenate(rv) for rv in rows_val])
    return rp, col, val


def bytes_of(sr, m, nnz):
    return 8 * (m + 1) + nnz * (4 + np.dtype(gen.VALUE_DTYPE[sr]).itemsize)


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "or_and_bool", "sel2nd_min_i32",
                                "plus_times_i64"))
def test_batches_reassemble_to_the_product(cb, sr):
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=300)
    A = P.with_values(gen.random_values(sr, P.nnz, 301))
    B = P.with_values(gen.random_values(sr, P.nnz, 302))
    want = oracle.spgemm(sr, A, B)
    nnz = int(want[0][-1])
    budget = bytes_of(sr, A.nrows, nnz // 5)        # about six batches
    batches, st = run_batches(cb, sr, A, B, budget)
    assert st["batches"] == len(batches) >= 5
    assert st["nnz_total"] == nnz
    for b in batches:
        assert bytes_of(sr, A.nrows, b[4].size) <= budget
    compare_rows(sr, assemble(batches, A.nrows), want)


def test_batches_with_unsorted_b_filter_rows(cb):
    sr = "plus_times_f64"
    P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=310)
    A = P.with_values(gen.random_values(sr, P.nnz, 311))
    rng = np.random.default_rng(312)
    col, val = P.col.copy(), gen.random_values(sr, P.nnz, 313)
    for r in range(P.nrows):
        s, e = P.row_ptr[r], P.row_ptr[r + 1]
        perm = rng.permutation(e - s) + s
        col[s:e], val[s:e] = col[perm], val[perm]
    B = gen.CSR(P.nrows, P.ncols, P.row_ptr, col, val)
    want = oracle.spgemm(sr, A, B)
    budget = bytes_of(sr, A.nrows, int(want[0][-1]) // 4)
    batches, st = run_batches(cb, sr, A, B, budget)
    assert len(batches) >= 4
    compare_rows(sr, assemble(batches, A.nrows), want)


def test_skewed_columns_force_a_split(cb):
    # all of B's columns fall in the first tenth of the range: equal-width
    # batches overflow at the front and must be halved
    sr = "min_plus_u32"
    n, ncols = 3000, 100000
    rng = np.random.default_rng(320)
    lens = rng.integers(1, 60, n)
    cols = [np.sort(rng.choice(ncols // 10, size=l, replace=False)) for l in lens]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    B = gen.CSR(n, ncols, rp, np.concatenate(cols).astype(np.int32))
    B = B.with_values(gen.random_values(sr, B.nnz, 321))
    A = gen.random_csr(400, n, 0.01, seed=322, semiring=sr)
    want = oracle.spgemm(sr, A, B)
    nnz = int(want[0][-1])
    budget = bytes_of(sr, A.nrows, nnz // 3)
    batches, st = run_batches(cb, sr, A, B, budget)
    assert len(batches) > 4                      # more batches than the 4 equal-width ones
    compare_rows(sr, assemble(batches, A.nrows), want)


def test_early_stop_and_budget_errors(cb):
    sr = "plus_times_i64"
    P = gen.rmat(11, 8, *gen.RMAT_ABCD, seed=330)
    A = P.with_values(gen.random_values(sr, P.nnz, 331))
    want = oracle.spgemm(sr, A, A)
    budget = bytes_of(sr, A.nrows, int(want[0][-1]) // 4)
    batches, st = run_batches(cb, sr, A, A, budget, stop_after=1)
    assert len(batches) == 1 and st["batches"] == 1
    with pytest.raises(cb.CBError) as e:
        run_batches(cb, sr, A, A, 8 * (A.nrows + 1))            # no room for a single entry
    assert e.value.code == 6
    # a budget that fits everything gives one batch equal to the product
    batches, st = run_batches(cb, sr, A, A, 1 << 34)
    assert len(batches) == 1
    compare_rows(sr, assemble(batches, A.nrows), want)


def same_batch(x, y):
    """Same index, column range, row pointers and columns; the same values
    (fp64 within summation-order rounding: atomics combine in any order)."""
    if (x[0], x[1], x[2]) != (y[0], y[1], y[2]):
        return False
    if not (np.array_equal(x[3], y[3]) and np.array_equal(x[4], y[4])):
        return False
    if x[5].dtype.kind == "f":
        return bool(np.allclose(x[5], y[5], rtol=1e-12, atol=1e-12))
    return np.array_equal(x[5], y[5])


@pytest.mark.parametrize("stop", [1, 3, 5])
def test_resume_at_batch_b_repeats_the_remaining_batches(cb, stop):
    """A call stopped after `stop` batches and resumed at the next batch's
    col_lo and index gives exactly the full call's remaining batches (exact
    sizing), and the two parts together are the product."""
    sr = "plus_times_f64"
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=340)
    A = P.with_values(gen.random_values(sr, P.nnz, 341))
    want = oracle.spgemm(sr, A, A)
    budget = bytes_of(sr, A.nrows, int(want[0][-1]) // 6)
    full, st = run_batches(cb, sr, A, A, budget)
    assert len(full) > stop + 1
    head, _ = run_batches(cb, sr, A, A, budget, stop_after=stop)
    assert all(same_batch(x, y) for x, y in zip(head, full[:stop]))
    nxt = full[stop]
    tail, st2 = run_batches(cb, sr, A, A, budget, resume_col=nxt[1], resume_batch=nxt[0])
    assert st2["batches"] == len(tail) == len(full) - stop
    assert all(same_batch(x, y) for x, y in zip(tail, full[stop:]))
    compare_rows(sr, assemble(head + tail, A.nrows), want)


def test_resume_after_a_split_and_with_learned_sizing(cb):
    """Resuming inside the skewed product whose front ranges are halved
    (exact sizing), and resuming a learned-sizing call (its remaining
    columns are cut afresh): the parts still reassemble to the product."""
    sr = "min_plus_u32"
    n, ncols = 3000, 100000
    rng = np.random.default_rng(350)
    lens = rng.integers(1, 60, n)
    cols = [np.sort(rng.choice(ncols // 10, size=l, replace=False)) for l in lens]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    B = gen.CSR(n, ncols, rp, np.concatenate(cols).astype(np.int32))
    B = B.with_values(gen.random_values(sr, B.nnz, 351))
    A = gen.random_csr(400, n, 0.01, seed=352, semiring=sr)
    want = oracle.spgemm(sr, A, B)
    budget = bytes_of(sr, A.nrows, int(want[0][-1]) // 3)
    full, _ = run_batches(cb, sr, A, B, budget)
    k = 2
    tail, _ = run_batches(cb, sr, A, B, budget, resume_col=full[k][1], resume_batch=k)
    assert all(same_batch(x, y) for x, y in zip(tail, full[k:])) and len(tail) == len(full) - k
    # learned sizing: stop after two batches, resume where they ended
    from paper_2106_14402_gb300 import sizer
    model, _ = sizer.load()
    dA, dB = cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(B, sr)
    parts = []

    def keep(limit):
        def on_batch(b, lo, hi, Cb):
            parts.append((b, lo, hi) + tuple(Cb.to_host()))
            return limit is not None and len(parts) >= limit
        return on_batch

    cb.spgemm_column_batches(sr, dA, dB, budget, keep(2), sizing="learned", mlp=model)
    assert len(parts) == 2
    cb.spgemm_column_batches(sr, dA, dB, budget, keep(None), sizing="learned", mlp=model,
                             resume_col=parts[-1][2], resume_batch=2)
    assert [p[0] for p in parts] == list(range(len(parts)))
    assert parts[-1][2] == B.ncols
    compare_rows(sr, assemble(parts, A.nrows), want)


def test_resume_arguments_are_checked(cb):
    sr = "plus_times_i64"
    P = gen.rmat(10, 8, *gen.RMAT_ABCD, seed=360)
    A = P.with_values(gen.random_values(sr, P.nnz, 361))
    for kw in ({"resume_col": -1}, {"resume_col": A.ncols + 1}, {"resume_batch": -1}):
        with pytest.raises(cb.CBError) as e:
            run_batches(cb, sr, A, A, 1 << 30, **kw)
        assert e.value.code == 1
    got, st = run_batches(cb, sr, A, A, 1 << 30, resume_col=A.ncols)   # nothing left
    assert got == [] and st["batches"] == 0
