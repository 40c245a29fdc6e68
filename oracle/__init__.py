"""CPU oracle for the semiring SpGEMM -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The library's product path never does,
and this package imports nothing from the library (it shares no code with
the CUDA path).

`spgemm` wraps oracle.cpp: a plain Gustavson SpGEMM with one ordered map per
output row (paper Sec. 4.1), over the six semirings named below (five with
one value type, one heterogeneous: Sec. 1).
`row_stats` gives flops_i and max_p nnz(B(p,:)) per row (Sec. 4.1, phase (1);
Table 1 defines flops).  `mlp` holds the FP64 reference of the learned row
size predictor.  `merge` is the semiring sum of k partial results (Sec. 3.2),
stated directly in numpy; `spmspv` the sparse-vector x sparse-matrix
product (Sec. 4.3), likewise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# (weight, label) pairs of the heterogeneous semiring, as oracle.cpp lays them out.
WLABEL = np.dtype([("w", "<f4"), ("label", "<i4")])

# Semiring names -> this file's own codes (oracle.cpp's enum) and the value
# dtypes of A, B and C.
_CODES = {
    "plus_times_i64": (1, np.int64, np.int64, np.int64),
    "plus_times_f64": (2, np.float64, np.float64, np.float64),
    "min_plus_u32": (3, np.uint32, np.uint32, np.uint32),
    "or_and_bool": (4, np.uint8, np.uint8, np.uint8),
    "sel2nd_min_i32": (5, np.int32, np.int32, np.int32),
    "maxw_label": (6, np.float32, np.int32, WLABEL),
}
SEMIRINGS = tuple(s for s in _CODES if s != "maxw_label")   # one value type each
HETERO_SEMIRINGS = ("maxw_label",)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (plain g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.orc_row_stats.argtypes = [I64, P, P, P, P, P]
            lib.orc_row_stats.restype = ctypes.c_int
            lib.orc_spgemm.argtypes = [ctypes.c_int, I64, P, P, P, P, P, P, I64, P, ctypes.c_int,
                                       ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                       ctypes.POINTER(P)]
            lib.orc_spgemm.restype = ctypes.c_int
            lib.orc_free.argtypes = [P]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def row_stats(A, B):
    """(flops_i, maxb_i) per row of A.B: products per output row and the longest B row touched."""
    lib = _load()
    m = A.nrows
    flops = np.zeros(m, dtype=np.int64)
    maxb = np.zeros(m, dtype=np.int64)
    arp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    acol = np.ascontiguousarray(A.col, dtype=np.int32)
    brp = np.ascontiguousarray(B.row_ptr, dtype=np.int64)
    lib.orc_row_stats(m, _ptr(arp), _ptr(acol), _ptr(brp), _ptr(flops), _ptr(maxb))
    return flops, maxb


def spgemm(semiring: str, A, B, rows=None, threads: int = 0):
    """C = A (+).(x) B on the CPU.

    A and B are objects with nrows, ncols, row_ptr (int64), col (int32) and
    val arrays.  `rows` (optional int64 array) restricts the output to those
    rows of C, in that order.  Returns (row_ptr, col, val, absum): a CSR over
    the selected rows with sorted unique columns, and for fp64 the sum of
    |products| of every entry (zeros for the other semirings).  A's and B's
    values are taken in the semiring's A and B types (maxw_label: float32
    weights and int32 labels); its C values come back as WLABEL records.
    """
    code, adt, bdt, dt = _CODES[semiring]
    if A.ncols != B.nrows:
        raise ValueError("shape mismatch: A.ncols != B.nrows")
    lib = _load()
    arp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    acol = np.ascontiguousarray(A.col, dtype=np.int32)
    aval = np.ascontiguousarray(A.val, dtype=adt)
    brp = np.ascontiguousarray(B.row_ptr, dtype=np.int64)
    bcol = np.ascontiguousarray(B.col, dtype=np.int32)
    bval = np.ascontiguousarray(B.val, dtype=bdt)
    if rows is None:
        nsel, rp_rows = A.nrows, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nsel, rp_rows = rows.shape[0], _ptr(rows)
    o_rp, o_col, o_val, o_abs = (ctypes.c_void_p() for _ in range(4))
    rc = lib.orc_spgemm(code, A.nrows, _ptr(arp), _ptr(acol), _ptr(aval), _ptr(brp), _ptr(bcol),
                        _ptr(bval), nsel, rp_rows, int(threads), ctypes.byref(o_rp),
                        ctypes.byref(o_col), ctypes.byref(o_val), ctypes.byref(o_abs))
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    try:
        rp = np.ctypeslib.as_array(ctypes.cast(o_rp, ctypes.POINTER(ctypes.c_int64)), (nsel + 1,)).copy()
        nnz = int(rp[-1])
        n_alloc = max(nnz, 1)
        col = np.ctypeslib.as_array(ctypes.cast(o_col, ctypes.POINTER(ctypes.c_int32)), (n_alloc,))[:nnz].copy()
        raw = (ctypes.c_char * (n_alloc * np.dtype(dt).itemsize)).from_address(o_val.value)
        val = np.frombuffer(raw, dtype=dt, count=nnz).copy()
        absum = np.ctypeslib.as_array(ctypes.cast(o_abs, ctypes.POINTER(ctypes.c_double)), (n_alloc,))[:nnz].copy()
    finally:
        for p in (o_rp, o_col, o_val, o_abs):
            lib.orc_free(p)
    return rp, col, val, absum


from .merge import merge  # noqa: E402,F401
from .spmspv import spmspv  # noqa: E402,F401
