"""Parity of the semiring merge of k partial results (cb_merge) with the
merge oracle, over all five semirings: small parts (the one-launch kernel
and the two-phase path), parts with long rows (the rank windows), unsorted
and duplicate entries, empty parts; and, at scale, the partial products of
an R-MAT square merged back into the product."""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import check_structure, compare_rows

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


def run_merge(cb, sr, parts, fused=True):
    dparts = [cb.DeviceCSR.from_host(P, sr) for P in parts]
    C = cb.merge(sr, dparts, fused=fused)
    torch.cuda.synchronize()
    return C.to_host()


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("k", [1, 2, 5, 32])
@pytest.mark.parametrize("sr", SR)
def test_small_parts(cb, sr, k, fused):
    lo, hi = {"plus_times_i64": (-5, 5), "plus_times_f64": (-1.0, 1.0), "min_plus_u32": (0, 9),
              "or_and_bool": (0, 1), "sel2nd_min_i32": (-9, 9)}[sr]
    parts = []
    for l in range(k):
        P = gen.random_csr(300, 500, 0.01, seed=1000 + 17 * k + l, semiring=sr, duplicates=True,
                           shuffle=True, empty_rows=0.2)
        parts.append(P.with_values(gen.random_values(sr, P.nnz, 2000 + l, lo=lo, hi=hi)))
    got = run_merge(cb, sr, parts, fused)
    check_structure(got[0], got[1], 500)
    compare_rows(sr, got, oracle.merge(sr, parts))


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "or_and_bool"))
def test_long_rows(cb, sr):
    # rows of ~3000 entries over 100k columns in each of 4 parts: heavy rows
    parts = [gen.random_csr(120, 100_000, 0.03, seed=3000 + l, semiring=sr, empty_rows=0.1)
             for l in range(4)]
    got = run_merge(cb, sr, parts)
    check_structure(got[0], got[1], 100_000)
    compare_rows(sr, got, oracle.merge(sr, parts))
    assert cb.context().stats()["heavy_units"] > 0


def test_empty_parts_and_shapes(cb):
    sr = "min_plus_u32"
    E = gen.random_csr(50, 40, 0.0, seed=1, semiring=sr)
    P = gen.random_csr(50, 40, 0.2, seed=2, semiring=sr)
    got = run_merge(cb, sr, [E, P, E])
    compare_rows(sr, got, oracle.merge(sr, [P]))
    got = run_merge(cb, sr, [E, E])
    assert got[0].shape == (51,) and np.all(got[0] == 0)
    Q = gen.random_csr(50, 41, 0.2, seed=3, semiring=sr)
    with pytest.raises(cb.CBError) as e:
        run_merge(cb, sr, [P, Q])
    assert e.value.code == 2


def _column_block(A, lo, hi):
    keep = (A.col >= lo) & (A.col < hi)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))[keep]
    rp = np.zeros(A.nrows + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return gen.CSR(A.nrows, A.ncols, np.cumsum(rp), A.col[keep], A.val[keep])


def _row_block(B, lo, hi):
    lens = np.diff(B.row_ptr).copy()
    lens[:lo] = 0
    lens[hi:] = 0
    rp = np.zeros(B.nrows + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    s, e = B.row_ptr[lo], B.row_ptr[hi]
    return gen.CSR(B.nrows, B.ncols, rp, B.col[s:e], B.val[s:e])


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "plus_times_i64"))
def test_partial_products_merge_to_the_product(cb, sr):
    """A SUMMA-style split of the inner dimension into 6 blocks: the merge of
    the 6 partial products (each formed on the GPU) is A.A."""
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=140)
    A = P.with_values(gen.random_values(sr, P.nnz, 141))
    cuts = np.linspace(0, A.ncols, 7).astype(int)
    dparts = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        dL = cb.DeviceCSR.from_host(_column_block(A, lo, hi), sr)
        dR = cb.DeviceCSR.from_host(_row_block(A, lo, hi), sr)
        dparts.append(cb.spgemm(sr, dL, dR))
    C = cb.merge(sr, dparts)
    torch.cuda.synchronize()
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A))
