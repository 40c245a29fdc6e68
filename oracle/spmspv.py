"""CPU reference of the semiring sparse-vector x sparse-matrix product -- TEST
INFRASTRUCTURE ONLY (loaded by tests/, the smoke check and bench.py's CPU
legs; never by the library).

Sec. 4.3 of the paper (SpMSpV, the kernel of graph traversals such as BFS)
multiplies a sparse matrix by a sparse vector over a semiring.  This file
states the row form used with CSR matrices: y^T = x^T A, i.e.

    y_c = (+) over every stored x entry (i, x_i) and every stored A(i, c)
          of  x_i (x) A(i, c),

combined in x's storage order, then A's row storage order.  The pattern is
structural (an entry exists when some product exists, whatever its value).
Duplicate indices in x contribute separately.  (x) and (+) are those of
oracle.cpp: wrapping int64 multiply/add, IEEE fp64, uint32 saturating add /
min, boolean and / or (uint8, output 0/1), select2nd (the matrix value) /
int32 min, and the heterogeneous maxw_label: x holds float32 weights, A int32
labels, y (weight, label) records; y_c is the pair of the heaviest x entry
reaching c (IEEE 754 totalOrder on weights), the smaller label on ties.
For fp64 the sum of |products| per entry is returned beside it.
"""
from __future__ import annotations

import numpy as np

_DT = {"plus_times_i64": np.int64, "plus_times_f64": np.float64, "min_plus_u32": np.uint32,
       "or_and_bool": np.uint8, "sel2nd_min_i32": np.int32}
WLABEL = np.dtype([("w", "<f4"), ("label", "<i4")])


def total_order_rank(w) -> np.ndarray:
    """Integers ordered as IEEE 754 totalOrder orders the float32 weights w:
    a weight with its sign bit clear keeps its magnitude encoding m, one with
    the sign bit set maps to -m - 1 (so -0 < +0 and -NaN < -inf)."""
    bits = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.int64)
    mag = bits & 0x7FFFFFFF
    return np.where(bits >> 31 != 0, -mag - 1, mag)


def _spmspv_maxw_label(A, x_idx, x_val):
    x_idx = np.asarray(x_idx, dtype=np.int64)
    x_val = np.asarray(x_val, dtype=np.float32)
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    cols, w, lab = [], [], []
    for p, i in enumerate(x_idx):            # every product x_i (x) A(i, c) = (x_i, A(i, c))
        for q in range(rp[i], rp[i + 1]):
            cols.append(int(A.col[q]))
            w.append(x_val[p])
            lab.append(int(A.val[q]))
    if not cols:
        return np.zeros(0, np.int32), np.zeros(0, WLABEL), np.zeros(0)
    cols = np.array(cols, np.int64)
    w = np.array(w, np.float32)
    lab = np.array(lab, np.int64)
    order = np.lexsort((lab, -total_order_rank(w), cols))   # by column, heaviest first, then label
    cols, w, lab = cols[order], w[order], lab[order]
    head = np.ones(cols.size, dtype=bool)
    head[1:] = cols[1:] != cols[:-1]
    out = np.zeros(int(head.sum()), WLABEL)
    out["w"] = w[head]
    out["label"] = lab[head]
    return cols[head].astype(np.int32), out, np.zeros(out.size)


def _mul(semiring, a, b):
    if semiring == "plus_times_i64":
        return (a.astype(np.uint64) * b.astype(np.uint64)).view(np.int64)
    if semiring == "plus_times_f64":
        return a * b
    if semiring == "min_plus_u32":
        s = a.astype(np.uint64) + b.astype(np.uint64)
        return np.minimum(s, 0xFFFFFFFF).astype(np.uint32)
    if semiring == "or_and_bool":
        return ((a != 0) & (b != 0)).astype(np.uint8)
    if semiring == "sel2nd_min_i32":
        return b.astype(np.int32)
    raise ValueError(semiring)


def spmspv(semiring: str, A, x_idx, x_val):
    """y^T = x^T A: A is a CSR object (nrows, ncols, row_ptr, col, val), x a
    sparse vector of length A.nrows.  Returns (idx, val, absum), idx sorted."""
    if semiring == "maxw_label":
        return _spmspv_maxw_label(A, x_idx, x_val)
    dt = _DT[semiring]
    x_idx = np.asarray(x_idx, dtype=np.int64)
    x_val = np.asarray(x_val, dtype=dt)
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    lens = rp[x_idx + 1] - rp[x_idx]
    if lens.sum() == 0:
        return np.zeros(0, np.int32), np.zeros(0, dt), np.zeros(0)
    owner = np.repeat(np.arange(x_idx.size), lens)                    # x entry of each product
    first = np.repeat(rp[x_idx] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    q = first + np.arange(owner.size)                                  # A position of each product
    cols = np.asarray(A.col, dtype=np.int64)[q]
    prod = _mul(semiring, x_val[owner], np.asarray(A.val, dtype=dt)[q])
    order = np.lexsort((np.arange(owner.size), cols))                 # by column, then product order
    cols, prod = cols[order], prod[order]
    head = np.ones(cols.size, dtype=bool)
    head[1:] = cols[1:] != cols[:-1]
    starts = np.nonzero(head)[0]
    if semiring == "plus_times_i64":
        out = np.add.reduceat(prod.view(np.uint64), starts).view(np.int64)
        ab = np.zeros(starts.size)
    elif semiring == "plus_times_f64":
        out = np.add.reduceat(prod, starts)
        ab = np.add.reduceat(np.abs(prod), starts)
    elif semiring == "or_and_bool":
        out = np.maximum.reduceat(prod, starts)
        ab = np.zeros(starts.size)
    else:
        out = np.minimum.reduceat(prod, starts)
        ab = np.zeros(starts.size)
    return cols[starts].astype(np.int32), out.astype(dt), ab
