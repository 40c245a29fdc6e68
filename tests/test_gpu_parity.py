"""Parity of the CUDA SpGEMM (called through the C ABI) with the CPU oracle.

Covers every tier of the path (the one-launch kernel for small rows, warp /
256-thread / 512-thread hash teams, rank windows of heavy rows), all five
semirings, the adversarial inputs the ABI
accepts (unsorted and duplicate columns, empty and full rows, rectangular
shapes, explicit zeros, saturation), the edge cases (no rows, no entries,
one column, the largest column index), the two workloads at full size, and
the error paths.
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import check_structure, compare_rows, sample_rows

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


def run_pair(cb, sr, A, B, check=True, fused=True):
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = dA if B is A else cb.DeviceCSR.from_host(B, sr)
    C = cb.spgemm(sr, dA, dB, check=check, fused=fused)
    torch.cuda.synchronize()
    return C.to_host()


def assert_parity(cb, sr, A, B, rows=None, fused=True):
    got = run_pair(cb, sr, A, B, fused=fused)
    check_structure(got[0], got[1], B.ncols)
    want = oracle.spgemm(sr, A, B, rows=rows)
    return compare_rows(sr, got, want, rows=rows)


# ---------------------------------------------------------------------------
# small adversarial inputs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("shape", [(1, 1, 1, 1.0), (7, 5, 9, 0.5), (40, 33, 50, 0.2),
                                   (200, 150, 300, 0.05), (64, 1, 64, 0.9), (3, 100, 1, 0.3)])
def test_small_random(cb, sr, shape, fused):
    m, n, k, d = shape
    A = gen.random_csr(m, n, d, seed=m * 7 + n, semiring=sr, empty_rows=0.15, full_rows=0.05)
    B = gen.random_csr(n, k, d, seed=k * 11 + n, semiring=sr, empty_rows=0.15, full_rows=0.05)
    assert_parity(cb, sr, A, B, fused=fused)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("sr", SR)
def test_duplicates_unsorted_and_zeros(cb, sr, fused):
    lo, hi = {"plus_times_i64": (-3, 3), "plus_times_f64": (-1.0, 1.0), "min_plus_u32": (0, 5),
              "or_and_bool": (0, 1), "sel2nd_min_i32": (-4, 4)}[sr]
    A = gen.random_csr(120, 90, 0.08, seed=5, semiring=sr, duplicates=True, shuffle=True,
                       empty_rows=0.1, lo=lo, hi=hi)
    B = gen.random_csr(90, 140, 0.08, seed=6, semiring=sr, duplicates=True, shuffle=True,
                       empty_rows=0.1, lo=lo, hi=hi)
    assert_parity(cb, sr, A, B, fused=fused)


def test_wrap_and_saturation(cb):
    A = gen.random_csr(50, 40, 0.3, seed=8, semiring="plus_times_i64", lo=1 << 61, hi=1 << 62)
    B = gen.random_csr(40, 60, 0.3, seed=9, semiring="plus_times_i64", lo=-(1 << 62), hi=1 << 62)
    assert_parity(cb, "plus_times_i64", A, B)
    A = gen.random_csr(50, 40, 0.3, seed=10, semiring="min_plus_u32", lo=0xFFFFFFF0, hi=0xFFFFFFFF)
    B = gen.random_csr(40, 60, 0.3, seed=11, semiring="min_plus_u32", lo=0, hi=40)
    assert_parity(cb, "min_plus_u32", A, B)


def _tiered_inputs(sr, seed=0, ncols=70000):
    """A has rows hitting every tier: empty, a few products, ~1k, ~4k and
    heavy (tens of thousands of distinct columns over several slices)."""
    rng = np.random.default_rng(seed)
    n = 3000
    B = gen.random_csr(n, ncols, 0.0, seed=seed + 1, semiring=sr)
    # B rows of varied length (1..400) with random distinct columns
    lens = rng.integers(1, 400, n)
    lens[:20] = 3000
    cols = [np.sort(rng.choice(ncols, size=l, replace=False)) for l in lens]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    B = gen.CSR(n, ncols, rp, np.concatenate(cols).astype(np.int32))
    B = B.with_values(gen.random_values(sr, B.nnz, seed + 2))
    a_lens = [0, 1, 2, 3, 5, 8, 12, 20, 40, 60, 100, 150, 250, 400, 0, 1, 30, 700, 2, 900]
    a_cols = [np.sort(rng.choice(n, size=l, replace=False)) for l in a_lens]
    arp = np.zeros(len(a_lens) + 1, np.int64)
    arp[1:] = np.cumsum(a_lens)
    A = gen.CSR(len(a_lens), n, arp, np.concatenate(a_cols).astype(np.int32))
    A = A.with_values(gen.random_values(sr, A.nnz, seed + 3))
    return A, B


@pytest.mark.parametrize("sr", SR)
def test_every_tier(cb, sr):
    A, B = _tiered_inputs(sr)
    flops, _ = oracle.row_stats(A, B)
    assert flops.max() > 100_000          # reaches the heavy slice path
    assert_parity(cb, sr, A, B)
    ctx = cb.context()
    assert ctx.stats()["heavy_units"] > 0


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "sel2nd_min_i32"))
def test_heavy_rows_unsorted_b(cb, sr):
    # B rows shuffled: window passes must filter whole rows instead of searching them
    A, B = _tiered_inputs(sr, seed=5)
    rng = np.random.default_rng(6)
    col = B.col.copy()
    val = B.val.copy()
    for r in range(B.nrows):
        s, e = B.row_ptr[r], B.row_ptr[r + 1]
        perm = rng.permutation(e - s) + s
        col[s:e], val[s:e] = col[perm], val[perm]
    B = gen.CSR(B.nrows, B.ncols, B.row_ptr, col, val)
    assert_parity(cb, sr, A, B)


@pytest.mark.parametrize("sr", ("plus_times_f64", "or_and_bool"))
def test_heavy_rows_several_spans(cb, sr):
    # 600000 columns = 3 bitmap spans; the widest rows need several windows per span
    A, B = _tiered_inputs(sr, seed=7, ncols=600000)
    assert_parity(cb, sr, A, B)
    assert cb.context().stats()["heavy_units"] > A.nrows


@pytest.mark.parametrize("sr", SR)
def test_rank_window_columns_dense_and_sparse(cb, sr):
    """Heavy rows whose rank windows are dense (on average 8 or more output
    columns per bitmap word: columns read out a word per warp step) and
    sparse (fewer: a word per thread), on one span of 8192 columns and on a
    row spread over two spans, against the oracle."""
    rng = np.random.default_rng(71)
    n, ncols = 2000, 8192
    lens = rng.integers(50, 400, n)
    cols = [np.sort(rng.choice(ncols, size=l, replace=False)) for l in lens]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    B = gen.CSR(n, ncols, rp, np.concatenate(cols).astype(np.int32))
    B = B.with_values(gen.random_values(sr, B.nnz, 72))
    # A rows of 3 .. 300 entries: 600 .. 8192 distinct output columns
    a_lens = [3, 4, 5, 6, 8, 10, 14, 20, 40, 80, 300, 0, 1]
    a_cols = [np.sort(rng.choice(n, size=l, replace=False)) for l in a_lens]
    arp = np.zeros(len(a_lens) + 1, np.int64)
    arp[1:] = np.cumsum(a_lens)
    A = gen.CSR(len(a_lens), n, arp, np.concatenate(a_cols).astype(np.int32))
    A = A.with_values(gen.random_values(sr, A.nnz, 73))
    want = oracle.spgemm(sr, A, B)
    nnz = np.diff(want[0])
    words = ncols // 32          # one window per row: every row holds < kWcut entries
    heavy = nnz > 512            # rows past the hash tiers
    assert np.any(heavy & (nnz >= 8 * words)) and np.any(heavy & (nnz < 8 * words))
    got = run_pair(cb, sr, A, B)
    check_structure(got[0], got[1], B.ncols)
    compare_rows(sr, got, want)
    assert cb.context().stats()["heavy_units"] >= int(heavy.sum())
    # the same rows with their columns spread over two spans (sparse windows)
    B2 = gen.CSR(n, 2 * (1 << 18), rp, (B.col.astype(np.int64) * 61).astype(np.int32), B.val)
    assert_parity(cb, sr, A, B2)


def test_single_hot_column(cb):
    # every product of every row lands in column 7: maximal atomic contention
    n = 5000
    B = gen.CSR(n, 10, np.arange(n + 1, dtype=np.int64), np.full(n, 7, np.int32))
    A = gen.random_csr(30, n, 0.3, seed=12)
    for sr in ("plus_times_f64", "plus_times_i64", "min_plus_u32"):
        Av = A.with_values(gen.random_values(sr, A.nnz, 13))
        Bv = B.with_values(gen.random_values(sr, B.nnz, 14))
        assert_parity(cb, sr, Av, Bv)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("sr", ("plus_times_f64", "or_and_bool"))
def test_empty_shapes(cb, sr):
    for (m, n, k) in [(0, 5, 5), (5, 0, 5), (5, 5, 0), (4, 6, 3)]:
        A = gen.random_csr(m, n, 0.0, seed=1, semiring=sr)
        B = gen.random_csr(n, k, 0.5, seed=2, semiring=sr)
        got = run_pair(cb, sr, A, B)
        assert got[0].shape == (m + 1,) and np.all(got[0] == 0) and got[1].size == 0


def test_largest_column_index(cb):
    sr = "plus_times_i64"
    ncols = 2**31 - 1
    rng = np.random.default_rng(3)
    # 6 B rows with columns spread over the whole int32 range, incl. the last one
    cols = [np.unique(np.concatenate([rng.integers(0, ncols, 2000), [ncols - 1, 0]])) for _ in range(6)]
    rp = np.zeros(7, np.int64)
    rp[1:] = np.cumsum([c.size for c in cols])
    B = gen.CSR(6, ncols, rp, np.concatenate(cols).astype(np.int32))
    B = B.with_values(gen.random_values(sr, B.nnz, 4))
    A = gen.random_csr(5, 6, 0.7, seed=5, semiring=sr, full_rows=0.4)
    assert_parity(cb, sr, A, B)


# ---------------------------------------------------------------------------
# workloads at full size
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fused", [True, False])
def test_er_square_bit_exact(cb, fused):
    (sr, A, B), = gen.er_square()
    assert_parity(cb, sr, A, B, fused=fused)
    if fused:  # validation (2) + the one-launch kernel, tried first (mean rows fit 8 lanes)
        assert cb.context().stats()["kernels"] == 3


@pytest.fixture(scope="module")
def rmat18():
    return gen.rmat_square(18, 16, cfg=2)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_rmat_square_sampled(cb, rmat18, k):
    sr, A, B = rmat18[k]
    flops, maxb = oracle.row_stats(A, B)
    rows = sample_rows(A.nrows, flops, frac=0.004, top=40, seed=k)
    got = run_pair(cb, sr, A, B)
    rp, col, val = got
    check_structure(rp, col, B.ncols)
    nz = np.diff(rp)
    assert np.all(nz >= maxb) and np.all(nz <= np.minimum(flops, B.ncols))
    if sr == "or_and_bool":
        assert np.all(val == 1)
    compare_rows(sr, got, oracle.spgemm(sr, A, B, rows=rows), rows=rows)


def test_rmat_patterns_agree_across_semirings(cb, rmat18):
    pats = []
    for sr, A, B in rmat18:
        rp, col, _ = run_pair(cb, sr, A, B, check=False)
        pats.append((rp, col))
    for rp, col in pats[1:]:
        assert np.array_equal(rp, pats[0][0]) and np.array_equal(col, pats[0][1])


def test_integer_results_are_deterministic(cb):
    A = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=77)
    A = A.with_values(gen.random_values("plus_times_i64", A.nnz, 78))
    r1 = run_pair(cb, "plus_times_i64", A, A)
    r2 = run_pair(cb, "plus_times_i64", A, A)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# individual steps through the C ABI
# ---------------------------------------------------------------------------

def test_row_stats_and_row_nnz(cb):
    A = gen.rmat(14, 16, *gen.RMAT_ABCD, seed=80)
    A = A.with_values(gen.random_values("plus_times_f64", A.nnz, 81))
    dA = cb.DeviceCSR.from_host(A, "plus_times_f64")
    f, mb = cb.row_stats(dA, dA)
    nz = cb.row_nnz(dA, dA)
    wf, wmb = oracle.row_stats(A, A)
    assert np.array_equal(f.cpu().numpy(), wf)
    assert np.array_equal(mb.cpu().numpy().astype(np.int64), wmb)
    rp = oracle.spgemm("or_and_bool", A.with_values(np.ones(A.nnz, np.uint8)),
                       A.with_values(np.ones(A.nnz, np.uint8)))[0]
    assert np.array_equal(nz.cpu().numpy(), np.diff(rp))


# 5,000,011 entries take 1,221 tiles: the scan of tile sums carries across
# two chunks of 1,024 tiles.
@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 1_000_003, 5_000_011])
def test_exclusive_scan(cb, n):
    x = torch.randint(0, 1 << 20, (n,), dtype=torch.int64, device="cuda")
    out = cb.exclusive_scan(x).cpu().numpy()
    want = np.zeros(n + 1, np.int64)
    want[1:] = np.cumsum(x.cpu().numpy())
    assert np.array_equal(out, want)


# ---------------------------------------------------------------------------
# caller-provided output and error paths
# ---------------------------------------------------------------------------

def test_caller_buffers_and_capacity(cb):
    sr = "plus_times_f64"
    A = gen.random_csr(100, 80, 0.1, seed=20, semiring=sr)
    B = gen.random_csr(80, 90, 0.1, seed=21, semiring=sr)
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = cb.DeviceCSR.from_host(B, sr)
    want = oracle.spgemm(sr, A, B)
    nnz = int(want[0][-1])
    out = cb.DeviceCSR(100, 90, torch.empty(101, dtype=torch.int64, device="cuda"),
                       torch.empty(nnz, dtype=torch.int32, device="cuda"),
                       torch.empty(nnz, dtype=torch.float64, device="cuda"))
    C = cb.spgemm(sr, dA, dB, out=out)
    compare_rows(sr, C.to_host(), want)
    small = cb.DeviceCSR(100, 90, out.row_ptr, out.col[: nnz - 1], out.val[: nnz - 1])
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, dB, out=small)
    assert e.value.code == 9


def test_invalid_inputs_are_rejected(cb):
    sr = "plus_times_i64"
    A = gen.random_csr(20, 10, 0.3, seed=30, semiring=sr)
    B = gen.random_csr(10, 12, 0.3, seed=31, semiring=sr)
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = cb.DeviceCSR.from_host(B, sr)
    # shape mismatch (host check)
    dB_bad = cb.DeviceCSR(11, 12, dB.row_ptr, dB.col, dB.val)
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, dB_bad)
    assert e.value.code == 2
    # column out of range (device validation runs before any other kernel)
    col = dB.col.clone()
    col[0] = 12
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, cb.DeviceCSR(10, 12, dB.row_ptr, col, dB.val))
    assert e.value.code == 4
    # decreasing row pointers
    rp = dA.row_ptr.clone()
    rp[5] = rp[6] + 1
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, cb.DeviceCSR(20, 10, rp, dA.col, dA.val), dB)
    assert e.value.code == 4
    # the context is still usable afterwards
    compare_rows(sr, cb.spgemm(sr, dA, dB).to_host(), oracle.spgemm(sr, A, B))


def test_drop_result_without_sync(cb):
    # The library-allocated C is released in stream order, so dropping it
    # while its kernels are still queued is safe.
    sr = "plus_times_f64"
    A = gen.rmat(14, 16, *gen.RMAT_ABCD, seed=90)
    A = A.with_values(gen.random_values(sr, A.nnz, 91))
    dA = cb.DeviceCSR.from_host(A, sr)
    for _ in range(3):
        C = cb.spgemm(sr, dA, dA)
        del C
    got = cb.spgemm(sr, dA, dA).to_host()
    rows = np.arange(0, A.nrows, 97)
    compare_rows(sr, got, oracle.spgemm(sr, A, A, rows=rows), rows=rows)


# ---------------------------------------------------------------------------
# high compression (block-clustered, shaped like protein-similarity networks)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bounds", [(512, 512), (4096, 4096)])
@pytest.mark.parametrize("sr", SR)
def test_high_compression_block_clustered(cb, sr, bounds):
    P = gen.block_clustered(1 << 13, 256, 0.5, 1.0, seed=31)
    vals = gen.random_values(sr, P.nnz, 32)
    A = P.with_values(vals if sr != "sel2nd_min_i32" else np.ones(P.nnz, np.int32))
    B = P.with_values(vals)
    flops, _ = oracle.row_stats(A, B)
    ctx = cb.context()
    ctx.set_tune(bounds[0], bounds[1], 512)
    try:
        got = run_pair(cb, sr, A, B)
    finally:
        ctx.set_tune(512, 512, 512)
    check_structure(got[0], got[1], B.ncols)
    want = oracle.spgemm(sr, A, B)
    assert flops.sum() > 20 * int(want[0][-1])      # compression ratio above 20
    compare_rows(sr, got, want)
