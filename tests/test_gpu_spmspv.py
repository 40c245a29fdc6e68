"""Parity of the semiring SpMSpV (cb_spmspv, y^T = x^T A) with its oracle,
in both forms (dense accumulator; buckets / propagation blocking): all five
semirings, unsorted and duplicate x indices, empty rows, long rows (chunks
of one row on several warps), outputs spanning many buckets with a ragged
last bucket, repeated calls and a change of semiring on one context (the
dense accumulator is reset between calls), error paths."""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SR = gen.SEMIRINGS


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def run(cb, sr, A, idx, val, dA=None, ctx=None, bucket=False):
    dA = dA or cb.DeviceCSR.from_host(A, sr)
    xi = torch.from_numpy(np.asarray(idx, np.int32)).cuda()
    xv = torch.from_numpy(np.asarray(val).view(np.int32) if np.asarray(val).dtype == np.uint32
                          else np.asarray(val)).cuda()
    if cb.SEMIRING[sr][1] == torch.uint32:
        xv = xv.view(torch.uint32)
    yi, yv = cb.spmspv(sr, dA, xi, xv, ctx=ctx, bucket=bucket)
    torch.cuda.synchronize()
    yv = yv.view(torch.int32).cpu().numpy().view(np.uint32) if yv.dtype == torch.uint32 else yv.cpu().numpy()
    return yi.cpu().numpy(), yv


def check(sr, got, want):
    yi, yv = got
    wi, wv, wa = want
    compare_rows(sr, (np.array([0, yi.size]), yi, yv), (np.array([0, wi.size]), wi, wv, wa))


@pytest.mark.parametrize("bucket", [False, True])
@pytest.mark.parametrize("nx", [1, 37, 2000])
@pytest.mark.parametrize("sr", SR)
def test_matches_oracle(cb, sr, nx, bucket):
    P = gen.rmat(14, 16, *gen.RMAT_ABCD, seed=150)
    A = P.with_values(gen.random_values(sr, P.nnz, 151))
    rng = np.random.default_rng(152 + nx)
    idx = rng.integers(0, A.nrows, nx)                 # unsorted, duplicates for large nx
    val = gen.random_values(sr, nx, 153 + nx)
    check(sr, run(cb, sr, A, idx, val, bucket=bucket), oracle.spmspv(sr, A, idx, val))


@pytest.mark.parametrize("bucket", [False, True])
@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "or_and_bool"))
def test_long_rows_and_adversarial_matrix(cb, sr, bucket):
    A = gen.random_csr(64, 5000, 0.3, seed=160, semiring=sr, duplicates=True, shuffle=True,
                       empty_rows=0.2, full_rows=0.1)
    idx = np.arange(64)[::-1]
    val = gen.random_values(sr, 64, 161)
    check(sr, run(cb, sr, A, idx, val, bucket=bucket), oracle.spmspv(sr, A, idx, val))


@pytest.mark.parametrize("sr", ("plus_times_i64", "sel2nd_min_i32"))
def test_bucket_form_wide_output(cb, sr):
    """Columns over 96 buckets of 1024 and a ragged last one (n = 98,765):
    every bucket, its first and last column, and empty buckets in between."""
    n = 98765
    A = gen.random_csr(40, n, 0.01, seed=165, semiring=sr, empty_rows=0.1)
    rng = np.random.default_rng(166)
    idx = rng.integers(0, 40, 60)
    val = gen.random_values(sr, 60, 167)
    want = oracle.spmspv(sr, A, idx, val)
    check(sr, run(cb, sr, A, idx, val, bucket=True), want)
    # columns only at bucket edges
    cols = np.array([0, 4095, 4096, 8191, 3 * 4096, n - 1], np.int32)
    E = gen.CSR(2, n, np.array([0, 6, 6], np.int64), cols,
                gen.random_values(sr, 6, 168))
    idx = np.array([0, 1, 0])
    val = gen.random_values(sr, 3, 169)
    check(sr, run(cb, sr, E, idx, val, bucket=True), oracle.spmspv(sr, E, idx, val))


def test_repeated_calls_and_semiring_switch(cb):
    """The accumulator persists in the context: consecutive calls, of different
    semirings and widths, must each start from a clean state."""
    ctx = cb.Context()
    P = gen.rmat(12, 8, *gen.RMAT_ABCD, seed=170)
    rng = np.random.default_rng(171)
    for rep, sr in enumerate(("min_plus_u32", "min_plus_u32", "plus_times_f64", "or_and_bool",
                              "min_plus_u32", "sel2nd_min_i32", "plus_times_i64")):
        A = P.with_values(gen.random_values(sr, P.nnz, 172 + rep))
        idx = rng.integers(0, A.nrows, 300)
        val = gen.random_values(sr, 300, 180 + rep)
        check(sr, run(cb, sr, A, idx, val, ctx=ctx), oracle.spmspv(sr, A, idx, val))
    # a narrower matrix on the same context
    B = gen.random_csr(100, 77, 0.2, seed=190, semiring="plus_times_i64")
    idx = np.array([5, 99, 0, 5])
    val = gen.random_values("plus_times_i64", 4, 191)
    check("plus_times_i64", run(cb, "plus_times_i64", B, idx, val, ctx=ctx),
          oracle.spmspv("plus_times_i64", B, idx, val))


def test_bucket_form_many_buckets(cb):
    """More buckets than shared memory holds per-CTA counters for (n over
    2048 buckets of 1024 columns): the globally counted form."""
    sr = "min_plus_u32"
    n = 2048 * 4096 + 5003
    rng = np.random.default_rng(175)
    rows = []
    for i in range(30):
        rows.append(np.sort(rng.choice(n, 200, replace=False)))
    rp = np.zeros(31, np.int64)
    rp[1:] = np.cumsum([r.size for r in rows])
    A = gen.CSR(30, n, rp, np.concatenate(rows).astype(np.int32),
                gen.random_values(sr, int(rp[-1]), 176))
    idx = rng.integers(0, 30, 50)
    val = gen.random_values(sr, 50, 177)
    check(sr, run(cb, sr, A, idx, val, bucket=True), oracle.spmspv(sr, A, idx, val))


@pytest.mark.parametrize("bucket", [False, True])
def test_empty_and_errors(cb, bucket):
    sr = "plus_times_f64"
    A = gen.random_csr(50, 40, 0.2, seed=200, semiring=sr)
    yi, yv = run(cb, sr, A, np.zeros(0, np.int32), np.zeros(0), bucket=bucket)
    assert yi.size == 0 and yv.size == 0
    E = gen.random_csr(50, 40, 0.0, seed=201, semiring=sr)
    yi, _ = run(cb, sr, E, np.array([1, 2]), np.array([1.0, 2.0]), bucket=bucket)
    assert yi.size == 0
    with pytest.raises(cb.CBError) as e:
        run(cb, sr, A, np.array([3, 50]), np.array([1.0, 1.0]), bucket=bucket)
    assert e.value.code == 4
    # the context is still clean afterwards
    idx = np.array([3, 7, 3])
    val = np.array([0.5, -1.0, 2.0])
    check(sr, run(cb, sr, A, idx, val, bucket=bucket), oracle.spmspv(sr, A, idx, val))
