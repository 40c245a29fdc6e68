"""Parity of the work-queue kernel (k_queue_rows: one persistent launch,
rows dequeued in order, each formed in one pass with a bitmap of its columns
and a rank-indexed accumulator, offsets by look-back) with the CPU oracle.

It runs when every output row has at most 4096 products and at most 65536
columns and the one-launch kernel's lane bounds do not hold: ER rows with up
to 64 entries (the batched workload's rows), all semirings, duplicates and
unsorted rows, empty rows, column windows (column batches), stacked batched
products in every mode, a row that never publishes (bounded waits run out:
CB_ERR_TIMEOUT), and repeated launches (launch epochs of the row status
words).
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import check_structure, compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SR = gen.SEMIRINGS + gen.HETERO_SEMIRINGS


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def er_pair(sr, n, deg_a, deg_b, seed):
    A = gen.er_exact(n, n, deg_a, seed)
    B = gen.er_exact(n, n, deg_b, seed + 1)
    if sr in gen.HETERO_SEMIRINGS:
        return (A.with_values(gen.hetero_values(sr, "A", A.nnz, seed + 2, levels=16)),
                B.with_values(gen.hetero_values(sr, "B", B.nnz, seed + 3)))
    return (A.with_values(gen.random_values(sr, A.nnz, seed + 2)),
            B.with_values(gen.random_values(sr, B.nnz, seed + 3)))


def run(cb, sr, A, B, ctx=None, **kw):
    dA = cb.DeviceCSR.from_host(A, sr, operand="A")
    dB = cb.DeviceCSR.from_host(B, sr, operand="B")
    ctx = ctx or cb.context()
    C = cb.spgemm(sr, dA, dB, ctx=ctx, **kw)
    return C.to_host(), ctx.stats()


@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("shape", [(3000, 40, 40), (70000 // 2, 20, 64), (5000, 64, 64)])
def test_queue_rows_match_oracle(cb, sr, shape):
    n, da, db = shape
    A, B = er_pair(sr, n, da, db, seed=500 + n + da)
    got, st = run(cb, sr, A, B)
    # validation (2) + flops and binning (3) + the one work-queue launch
    assert st["kernels"] == 6, st["kernels"]
    check_structure(got[0], got[1], B.ncols)
    compare_rows(sr, got, oracle.spgemm(sr, A, B))


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "or_and_bool"))
def test_queue_rows_duplicates_unsorted_empty(cb, sr):
    A = gen.random_csr(4000, 3000, 0.012, seed=601, semiring=sr, duplicates=True, shuffle=True,
                       empty_rows=0.2)
    B = gen.random_csr(3000, 9000, 0.003, seed=602, semiring=sr, duplicates=True, shuffle=True,
                       empty_rows=0.2)
    flops, _ = oracle.row_stats(A, B)
    assert flops.max() <= 4096 and np.diff(A.row_ptr).max() > 32
    got, st = run(cb, sr, A, B)
    check_structure(got[0], got[1], B.ncols)
    compare_rows(sr, got, oracle.spgemm(sr, A, B))


def test_queue_rows_repeated_launches_and_two_phase_agree(cb):
    sr = "sel2nd_min_i32"
    A, B = er_pair(sr, 20000, 30, 30, seed=610)
    want = oracle.spgemm(sr, A, B)
    ctx = cb.Context()
    for _ in range(3):                       # launch epochs advance; nothing reset
        got, st = run(cb, sr, A, B, ctx=ctx)
        compare_rows(sr, got, want)
    got, st = run(cb, sr, A, B, ctx=ctx, fused=False)   # the two-phase path
    assert st["kernels"] > 6
    compare_rows(sr, got, want)


def test_queue_rows_in_column_batches(cb):
    """Column batches of 20000 columns each run through the queue."""
    sr = "plus_times_f64"
    A, B = er_pair(sr, 60000, 24, 24, seed=620)
    want = oracle.spgemm(sr, A, B)
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = cb.DeviceCSR.from_host(B, sr)
    parts = []
    budget = 8 * (A.nrows + 1) + int(want[0][-1]) * 12 // 3 + 1
    st = cb.spgemm_column_batches(sr, dA, dB, budget, lambda b, lo, hi, Cb: parts.append((lo, hi, Cb.to_host())))
    assert st["batches"] >= 3
    rows_c = [[] for _ in range(A.nrows)]
    rows_v = [[] for _ in range(A.nrows)]
    for lo, hi, (rp, col, val) in sorted(parts, key=lambda p: p[0]):
        assert hi - lo <= 65536
        for i in range(A.nrows):
            rows_c[i].append(col[rp[i]:rp[i + 1]])
            rows_v[i].append(val[rp[i]:rp[i + 1]])
    cols = [np.concatenate(c) for c in rows_c]
    rp = np.zeros(A.nrows + 1, np.int64)
    rp[1:] = np.cumsum([c.size for c in cols])
    compare_rows(sr, (rp, np.concatenate(cols), np.concatenate([np.concatenate(v) for v in rows_v])), want)


@pytest.mark.parametrize("row", [0, 7, 1500])
def test_queue_row_that_never_publishes(cb, row):
    sr = "min_plus_u32"
    A, B = er_pair(sr, 3000, 40, 40, seed=630)
    ctx = cb.Context()
    ctx.set_fault(cb.FAULT_SILENT_TILE, row, 32)
    dA, dB = cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(B, sr)
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, dB, ctx=ctx)
    assert e.value.code == 7 and "wait expired" in ctx.error()
    ctx.set_fault(cb.FAULT_SILENT_TILE, -1)
    C = cb.spgemm(sr, dA, dB, ctx=ctx)
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, B))
