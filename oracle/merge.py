"""CPU reference of the semiring merge of k partial results -- TEST
INFRASTRUCTURE ONLY (loaded by tests/, the smoke check and bench.py's CPU
legs; never by the library).

After the local multiplies of a SUMMA stage, and across the layers of the
communication-avoiding SpGEMM, the partial products of one block are
combined by the semiring's addition (Sec. 3.2): C = P_0 (+) P_1 (+) ...
(+) P_{k-1}, entry by entry over the union of the patterns.  Stated here
directly: every stored entry of every part, in part order and then storage
order, is (+)-combined into its coordinate; coordinates come out sorted.
Duplicate coordinates inside one part combine the same way.

Semirings as in oracle.cpp: (+) is wrapping int64 add, IEEE fp64 add, uint32
min, boolean or (uint8, nonzero = true, output 0/1), int32 min, and for the
heterogeneous maxw_label (parts hold (weight, label) records) the record
with the larger weight in IEEE 754 totalOrder, the smaller label on ties
(the rank of a weight in that order is spmspv.total_order_rank).  For fp64 the
sum of |values| per entry is returned for the tolerance test (the order of
an fp64 sum changes it by far less than that tolerance).
"""
from __future__ import annotations

import numpy as np

_DT = {"plus_times_i64": np.int64, "plus_times_f64": np.float64, "min_plus_u32": np.uint32,
       "or_and_bool": np.uint8, "sel2nd_min_i32": np.int32}


def merge(semiring: str, parts):
    """C = (+) over parts (objects with nrows, ncols, row_ptr, col, val).
    Returns (row_ptr, col, val, absum) with sorted unique columns per row."""
    if not parts:
        raise ValueError("merge needs at least one part")
    m, n = parts[0].nrows, parts[0].ncols
    for P in parts:
        if (P.nrows, P.ncols) != (m, n):
            raise ValueError("all parts must have the same shape")
    if semiring == "maxw_label":
        return _merge_maxw_label(parts, m)
    dt = _DT[semiring]
    rows, cols, vals, order = [], [], [], []
    base = 0
    for P in parts:
        rp = np.asarray(P.row_ptr, dtype=np.int64)
        nnz = int(rp[-1])
        rows.append(np.repeat(np.arange(m, dtype=np.int64), np.diff(rp)))
        cols.append(np.asarray(P.col[:nnz], dtype=np.int64))
        vals.append(np.asarray(P.val[:nnz], dtype=dt))
        order.append(base + np.arange(nnz, dtype=np.int64))   # part order, then storage order
        base += nnz
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    o = np.concatenate(order)
    idx = np.lexsort((o, c, r))          # by row, then column, then part/storage order
    r, c, v = r[idx], c[idx], v[idx]
    if r.size == 0:
        return np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, dt), np.zeros(0)
    head = np.ones(r.size, dtype=bool)
    head[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    starts = np.nonzero(head)[0]
    if semiring == "plus_times_i64":
        out = np.add.reduceat(v.view(np.uint64), starts).view(np.int64)     # wrapping
        ab = np.zeros(starts.size)
    elif semiring == "plus_times_f64":
        out = np.add.reduceat(v, starts)
        ab = np.add.reduceat(np.abs(v), starts)
    elif semiring in ("min_plus_u32", "sel2nd_min_i32"):
        out = np.minimum.reduceat(v, starts)
        ab = np.zeros(starts.size)
    elif semiring == "or_and_bool":
        out = (np.maximum.reduceat((v != 0).astype(np.uint8), starts) != 0).astype(np.uint8)
        ab = np.zeros(starts.size)
    else:
        raise ValueError(semiring)
    row_of = r[starts]
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, row_of + 1, 1)
    rp = np.cumsum(rp)
    return rp, c[starts].astype(np.int32), out.astype(dt), ab



def _merge_maxw_label(parts, m):
    from .spmspv import WLABEL, total_order_rank
    rows, cols, vals = [], [], []
    for P in parts:
        rp = np.asarray(P.row_ptr, dtype=np.int64)
        nnz = int(rp[-1])
        rows.append(np.repeat(np.arange(m, dtype=np.int64), np.diff(rp)))
        cols.append(np.asarray(P.col[:nnz], dtype=np.int64))
        vals.append(np.asarray(P.val[:nnz]).view(WLABEL))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals) if vals else np.zeros(0, WLABEL)
    if r.size == 0:
        return np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, WLABEL), np.zeros(0)
    # per coordinate: heaviest weight first, then the smaller label; keep the first
    idx = np.lexsort((v["label"].astype(np.int64), -total_order_rank(v["w"]), c, r))
    r, c, v = r[idx], c[idx], v[idx]
    head = np.ones(r.size, dtype=bool)
    head[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
    rp = np.zeros(m + 1, np.int64)
    np.add.at(rp, r[head] + 1, 1)
    return np.cumsum(rp), c[head].astype(np.int32), v[head].copy(), np.zeros(int(head.sum()))
