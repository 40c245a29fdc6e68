"""Host-side parts of the Python binding (no GPU, CPU tensors): scipy
interop round trips keep the stored entries and the value dtypes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")

from paper_2106_14402_gb300 import cb, gen  # noqa: E402


@pytest.mark.parametrize("sr", gen.SEMIRINGS)
def test_scipy_round_trip(sr):
    A = gen.random_csr(30, 40, 0.2, seed=3, semiring=sr, empty_rows=0.2)
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.nrows, A.ncols))
    d = cb.DeviceCSR.from_scipy(M, sr, device="cpu")
    assert d.val.dtype == cb.SEMIRING[sr][1]
    rp, col, val = d.to_host()
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
    assert np.array_equal(val, A.val.astype(val.dtype))
    back = d.to_scipy()
    assert back.shape == M.shape and (back != M).nnz == 0


def test_scipy_operand_dtypes_of_the_heterogeneous_semiring():
    A = gen.random_csr(10, 12, 0.3, seed=4)
    M = sp.csr_matrix((np.linspace(0, 1, A.nnz), A.col, A.row_ptr), shape=(10, 12))
    assert cb.DeviceCSR.from_scipy(M, "maxw_label", device="cpu", operand="A").val.dtype == torch.float32
    L = sp.csr_matrix((np.arange(A.nnz), A.col, A.row_ptr), shape=(10, 12))
    assert cb.DeviceCSR.from_scipy(L, "maxw_label", device="cpu", operand="B").val.dtype == torch.int32


def test_scipy_duplicates_in_csr_are_kept():
    """A CSR built from arrays keeps duplicate and unsorted columns; the copy
    keeps them too (the ABI combines duplicates by the semiring's (+))."""
    M = sp.csr_matrix((np.array([1.0, 2.0, 3.0]), np.array([2, 2, 0]), np.array([0, 2, 3])),
                      shape=(2, 3))
    d = cb.DeviceCSR.from_scipy(M, "plus_times_f64", device="cpu")
    rp, col, val = d.to_host()
    assert d.nnz == 3 and np.array_equal(col, [2, 2, 0]) and np.array_equal(val, [1.0, 2.0, 3.0])
