"""Seeded synthetic sparse inputs shared by the CUDA path and the CPU oracle.

This module holds no SpGEMM arithmetic: it only draws random sparse matrices
in CSR form (int64 row_ptr, int32 col, typed values) with numpy's PCG64, so
that both sides of a parity test see the same bytes.  Every matrix it emits
has strictly increasing column indices within a row (sorted, no duplicates).

Shapes follow the paper's workloads:
  * R-MAT with Graph500-style quadrant probabilities (the sparsity study of
    Sec. 4.5 uses an R-MAT with the Graph500 parameters), symmetrised,
    duplicates removed, vertices randomly permuted (Sec. 3.1 balances load by
    permuting matrices at assembly);
  * Erdos-Renyi rows with an exact number of distinct uniform columns;
  * banded matrices (a family with strong locality).
The paper's own matrices (Table 4) are not available; these stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20210628
_M64 = (1 << 64) - 1

# Semiring value types, by name.  bool values are stored as uint8 0/1.
VALUE_DTYPE = {
    "plus_times_i64": np.int64,
    "plus_times_f64": np.float64,
    "min_plus_u32": np.uint32,
    "or_and_bool": np.uint8,
    "sel2nd_min_i32": np.int32,
}
SEMIRINGS = tuple(VALUE_DTYPE)

# The heterogeneous semiring: A, B and C value types (C = (weight, label)
# records, 8 bytes).
WLABEL = np.dtype([("w", "<f4"), ("label", "<i4")])
HETERO_DTYPES = {"maxw_label": (np.float32, np.int32, WLABEL)}
HETERO_SEMIRINGS = tuple(HETERO_DTYPES)


def splitmix64(x: int) -> int:
    """One step of the splitmix64 output function (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def subseed(*parts: int) -> int:
    """Derive a 64-bit seed from a tuple of integers by chained splitmix64."""
    h = MASTER_SEED
    for p in parts:
        h = splitmix64(h ^ (int(p) & _M64))
    return h


def rng_for(*parts: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(subseed(*parts)))


@dataclass
class CSR:
    """Host CSR matrix: row_ptr int64[nrows+1], col int32[nnz], val typed[nnz] (or None)."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def with_values(self, val: np.ndarray) -> "CSR":
        assert val.shape == (self.nnz,)
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col, val)

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values (same result as np.unique, via one sort and a mask)."""
    s = np.sort(keys)
    if s.size == 0:
        return s
    keep = np.empty(s.size, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _csr_from_sorted_keys(keys: np.ndarray, nrows: int, ncols: int) -> CSR:
    rows = keys // ncols
    cols = (keys - rows * ncols).astype(np.int32)
    counts = np.bincount(rows, minlength=nrows).astype(np.int64)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(nrows, ncols, row_ptr, cols)


def csr_from_coo(rows: np.ndarray, cols: np.ndarray, nrows: int, ncols: int) -> CSR:
    """Sorted, de-duplicated CSR pattern from COO coordinates."""
    keys = sorted_unique(rows.astype(np.int64) * ncols + cols.astype(np.int64))
    return _csr_from_sorted_keys(keys, nrows, ncols)


def rmat(scale: int, edgefactor: int, a: float, b: float, c: float, seed: int,
         symmetrize: bool = True, permute: bool = True) -> CSR:
    """R-MAT pattern on n = 2**scale vertices with n*edgefactor directed edges.

    Each edge descends `scale` levels of the adjacency quadtree, picking the
    quadrants (0,0), (0,1), (1,0), (1,1) with probabilities a, b, c, d=1-a-b-c
    and no per-level noise.  Then (optionally) the transpose is added, the
    vertices are relabelled by one seeded random permutation, and duplicate
    edges are dropped.  Self-loops are kept.
    """
    n = 1 << scale
    m = n * edgefactor
    rng = rng_for(seed, 1)
    i = np.zeros(m, dtype=np.int64)
    j = np.zeros(m, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    for _ in range(scale):
        u = rng.random(m)
        ibit = u >= ab
        jbit = ((u >= a) & (u < ab)) | (u >= abc)
        i <<= 1
        j <<= 1
        i |= ibit
        j |= jbit
        del u, ibit, jbit
    if permute:
        perm = rng_for(seed, 2).permutation(n).astype(np.int64)
        i = perm[i]
        j = perm[j]
    if symmetrize:
        i, j = np.concatenate([i, j]), np.concatenate([j, i])
    keys = sorted_unique(i * n + j)
    del i, j
    return _csr_from_sorted_keys(keys, n, n)


def block_clustered(n: int, cluster: int, density: float, inter: float, seed: int) -> CSR:
    """High-compression pattern shaped like the paper's protein-similarity
    networks (dense groups of similar sequences, few links between groups):
    the n vertices form clusters of `cluster` consecutive vertices; every
    ordered pair inside a cluster is an edge with probability `density`, and
    each vertex gets Poisson(`inter`) edges to uniformly random vertices.
    Symmetrised, vertices relabelled by one seeded permutation, duplicates
    dropped, self-loops kept.  Squaring it gives compression ratios of
    order density^2 * cluster."""
    rng = rng_for(seed, 7)
    nc = n // cluster
    # intra-cluster pairs: per cluster a Bernoulli(density) cluster x cluster block
    blocks = rng.random((nc, cluster, cluster)) < density
    cb, ib, jb = np.nonzero(blocks)
    del blocks
    i = cb.astype(np.int64) * cluster + ib
    j = cb.astype(np.int64) * cluster + jb
    del cb, ib, jb
    k = rng.poisson(inter, nc * cluster)
    src = np.repeat(np.arange(nc * cluster, dtype=np.int64), k)
    dst = rng.integers(0, n, src.size, dtype=np.int64)
    i = np.concatenate([i, src])
    j = np.concatenate([j, dst])
    perm = rng_for(seed, 8).permutation(n).astype(np.int64)
    i, j = perm[i], perm[j]
    i, j = np.concatenate([i, j]), np.concatenate([j, i])
    keys = sorted_unique(i * n + j)
    del i, j
    return _csr_from_sorted_keys(keys, n, n)


def high_compression(n: int = 1 << 17, cluster: int = 256, density: float = 0.5, inter: float = 1.0,
                     cfg: int = 6, semiring: str = "plus_times_f64"):
    """C = A.A on a block-clustered matrix (compression ratio ~40)."""
    P = block_clustered(n, cluster, density, inter, seed=subseed(cfg, 0))
    A = P.with_values(random_values(semiring, P.nnz, subseed(cfg, 1)))
    return [(semiring, A, A)]


def er_exact(nrows: int, ncols: int, deg: int, seed: int) -> CSR:
    """Each row gets exactly min(deg, ncols) distinct uniformly random columns."""
    d = min(deg, ncols)
    rng = rng_for(seed, 3)
    cols = np.sort(rng.integers(0, ncols, size=(nrows, d), dtype=np.int64), axis=1)
    if d > 1:
        bad = np.nonzero((np.diff(cols, axis=1) == 0).any(axis=1))[0]
        for r in bad:
            # Sequential rejection: the first d distinct draws form a uniform d-subset.
            got: list[int] = []
            seen: set[int] = set()
            while len(got) < d:
                for x in rng.integers(0, ncols, size=2 * d):
                    x = int(x)
                    if x not in seen:
                        seen.add(x)
                        got.append(x)
                        if len(got) == d:
                            break
            cols[r] = np.sort(np.array(got, dtype=np.int64))
    row_ptr = np.arange(nrows + 1, dtype=np.int64) * d
    return CSR(nrows, ncols, row_ptr, cols.reshape(-1).astype(np.int32))


def banded(n: int, bw: int, deg: int, seed: int) -> CSR:
    """Row i gets min(deg, |window|) distinct random columns in [i-bw, i+bw] clipped to [0, n)."""
    rng = rng_for(seed, 4)
    width = 2 * bw + 1
    k = min(deg, width)
    offsets = np.arange(width, dtype=np.int64) - bw
    rows_out, cols_out = [], []
    for r0 in range(0, n, 4096):
        r1 = min(n, r0 + 4096)
        rows = np.arange(r0, r1, dtype=np.int64)
        cand = rows[:, None] + offsets[None, :]
        key = rng.random((r1 - r0, width))
        key[(cand < 0) | (cand >= n)] = 2.0          # positions outside [0, n) never win
        pick = np.argpartition(key, k - 1, axis=1)[:, :k] if k < width else np.tile(np.arange(width), (r1 - r0, 1))
        ok = np.take_along_axis(key, pick, axis=1) < 2.0
        c = np.take_along_axis(cand, pick, axis=1)
        rows_out.append(np.broadcast_to(rows[:, None], c.shape)[ok])
        cols_out.append(c[ok])
    return csr_from_coo(np.concatenate(rows_out), np.concatenate(cols_out), n, n)


def random_values(semiring: str, nnz: int, seed: int, lo=None, hi=None) -> np.ndarray:
    """Value streams per semiring (bounds inclusive for integers, [lo, hi) for floats)."""
    rng = rng_for(seed, 5)
    if semiring == "plus_times_i64":
        lo, hi = (1, 10) if lo is None else (lo, hi)
        return rng.integers(lo, hi + 1, size=nnz, dtype=np.int64)
    if semiring == "plus_times_f64":
        lo, hi = (0.0, 1.0) if lo is None else (lo, hi)
        return lo + (hi - lo) * rng.random(nnz)
    if semiring == "min_plus_u32":
        lo, hi = (1, 255) if lo is None else (lo, hi)
        return rng.integers(lo, hi + 1, size=nnz, dtype=np.uint32)
    if semiring == "or_and_bool":
        if lo is None:
            return np.ones(nnz, dtype=np.uint8)
        return rng.integers(0, 2, size=nnz, dtype=np.uint8)
    if semiring == "sel2nd_min_i32":
        lo, hi = (0, (1 << 30) - 1) if lo is None else (lo, hi)
        return rng.integers(lo, hi + 1, size=nnz, dtype=np.int32)
    raise ValueError(semiring)


def hetero_values(semiring: str, operand: str, nnz: int, seed: int, levels: int = 0) -> np.ndarray:
    """Values of a heterogeneous semiring's operand.  maxw_label: A = float32
    weights in [0, 1) (with levels > 0 drawn from the `levels` values k/levels,
    so equal weights are common), B = int32 labels uniform in [0, 2^30)."""
    rng = rng_for(seed, 6 if operand == "A" else 7)
    if semiring != "maxw_label":
        raise ValueError(semiring)
    if operand == "A":
        if levels > 0:
            return (rng.integers(0, levels, size=nnz) / levels).astype(np.float32)
        return rng.random(nnz, dtype=np.float32)
    return rng.integers(0, 1 << 30, size=nnz, dtype=np.int32)


# ---------------------------------------------------------------------------
# The workloads.  Each returns (semiring, A, B) triples; A and B share the
# pattern when the product is a square (C = A.A).
# ---------------------------------------------------------------------------

RMAT_ABCD = (0.57, 0.19, 0.19)


def er_square(n: int = 16384, deg: int = 8, cfg: int = 1):
    """Plain C = A.A over (+,x) int64; A is ER with exactly `deg` distinct columns per row."""
    A = er_exact(n, n, deg, subseed(cfg, 0))
    A = A.with_values(random_values("plus_times_i64", A.nnz, subseed(cfg, 1)))
    return [("plus_times_i64", A, A)]


def rmat_square(scale: int = 18, edgefactor: int = 16, cfg: int = 2,
                semirings=("plus_times_f64", "min_plus_u32", "or_and_bool")):
    """C = A.A on a symmetrised R-MAT, one value stream per semiring."""
    P = rmat(scale, edgefactor, *RMAT_ABCD, seed=subseed(cfg, 0))
    out = []
    for k, sr in enumerate(semirings):
        if sr == "sel2nd_min_i32":
            A = P.with_values(np.ones(P.nnz, dtype=np.int32))
            B = P.with_values(random_values(sr, P.nnz, subseed(cfg, 10 + k)))
        elif sr in HETERO_DTYPES:
            A = P.with_values(hetero_values(sr, "A", P.nnz, subseed(cfg, 10 + k)))
            B = P.with_values(hetero_values(sr, "B", P.nnz, subseed(cfg, 10 + k)))
        else:
            A = P.with_values(random_values(sr, P.nnz, subseed(cfg, 10 + k)))
            B = A
        out.append((sr, A, B))
    return out


def rmat_column_batched(scale: int = 21, edgefactor: int = 16, cfg: int = 3):
    """Memory-constrained workload: C = A.A over (+,x) fp64 U(0,1) on a
    symmetrised R-MAT of scale 21, edgefactor 16 (formed in column batches
    under a 24 GB output budget)."""
    return rmat_square(scale, edgefactor, cfg=cfg, semirings=("plus_times_f64",))


def rmat_held_out(scale: int = 20, edgefactor: int = 32, cfg: int = 5):
    """Held-out product of the learned sizer: (select2nd,min) int32 on a
    symmetrised R-MAT of scale 20, edgefactor 32 (A's values 1, B's values
    uniform in [0, 2^30))."""
    return rmat_square(scale, edgefactor, cfg=cfg, semirings=("sel2nd_min_i32",))


def training_family(index: int, cfg: int = 5) -> CSR:
    """Matrix `index` of the learned-sizer training mix (R-MAT / ER / banded, 2000 in all).

    Indices 0..666 are R-MAT (scale 12..16, a in [0.45, 0.65], d = 0.05,
    b = c = (0.95 - a)/2, edgefactor 16), 667..1333 are ER (n log-uniform in
    [2^12, 2^16], degree 4..64), 1334..1999 are banded (bandwidth 8..256,
    degree 4..64).  All are squared (C = A.A).
    """
    rng = rng_for(cfg, 100, index)
    if index < 667:
        scale = int(rng.integers(12, 17))
        a = float(rng.uniform(0.45, 0.65))
        bc = (0.95 - a) / 2
        return rmat(scale, 16, a, bc, bc, seed=subseed(cfg, 101, index))
    if index < 1334:
        n = int(math.exp(rng.uniform(math.log(1 << 12), math.log(1 << 16))))
        deg = int(rng.integers(4, 65))
        return er_exact(n, n, deg, seed=subseed(cfg, 102, index))
    n = int(math.exp(rng.uniform(math.log(1 << 12), math.log(1 << 16))))
    bw = int(rng.integers(8, 257))
    deg = int(rng.integers(4, 65))
    return banded(n, bw, deg, seed=subseed(cfg, 103, index))


def random_csr(nrows: int, ncols: int, density: float, seed: int, semiring: str | None = None,
               duplicates: bool = False, shuffle: bool = False, empty_rows: float = 0.0,
               full_rows: float = 0.0, lo=None, hi=None) -> CSR:
    """Small adversarial CSR inputs for parity tests.

    Each row independently is empty (prob. empty_rows), full (prob.
    full_rows) or Bernoulli(density) per column.  With `duplicates`, some
    stored entries are repeated (same coordinate, new value); with `shuffle`
    the columns inside a row are left in random order.  Values come from
    random_values(semiring, ...).
    """
    rng = rng_for(seed, 6)
    rows, cols = [], []
    for i in range(nrows):
        u = rng.random()
        if u < empty_rows:
            c = np.zeros(0, dtype=np.int64)
        elif u < empty_rows + full_rows:
            c = np.arange(ncols, dtype=np.int64)
        else:
            c = np.nonzero(rng.random(ncols) < density)[0].astype(np.int64)
        if duplicates and c.size:
            extra = rng.choice(c, size=int(rng.integers(0, c.size + 1)), replace=True)
            c = np.concatenate([c, extra])
        if shuffle:
            rng.shuffle(c)
        else:
            c = np.sort(c, kind="stable")
        rows.append(np.full(c.size, i, dtype=np.int64))
        cols.append(c)
    counts = np.array([c.size for c in cols], dtype=np.int64)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.concatenate(cols).astype(np.int32) if nrows else np.zeros(0, np.int32)
    out = CSR(nrows, ncols, row_ptr, col)
    if semiring is not None:
        out = out.with_values(random_values(semiring, out.nnz, subseed(seed, 7), lo, hi))
    return out


# ---------------------------------------------------------------------------
# Counter-based generator (same definition as csrc_gen/cbgen.cu, which
# generates the large batched workload on the device):
#   draw(s, c) = mix(s + 0x9E3779B97F4A7C15 * (c + 1)), mix = splitmix64 output
#   ER row r: candidates (draw(s, (r << 32) | t) >> 32) * ncols >> 32, first
#   `deg` distinct in draw order, sorted.
# ---------------------------------------------------------------------------

_GOLD = 0x9E3779B97F4A7C15


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_draw(seed: int, counters: np.ndarray) -> np.ndarray:
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(seed & _M64) + np.uint64(_GOLD) * (c + np.uint64(1)))


def er_counter(seed: int, nrows: int, ncols: int, deg: int) -> CSR:
    """Exact-degree ER pattern from the counter-based draw (matches cbgen_er)."""
    cols = np.zeros((nrows, deg), dtype=np.int64)
    for r in range(nrows):
        got: list[int] = []
        seen: set[int] = set()
        t = 0
        while len(got) < deg:
            ts = np.arange(t, t + 2 * deg, dtype=np.uint64)
            x = counter_draw(seed, (np.uint64(r) << np.uint64(32)) | ts)
            cand = ((x >> np.uint64(32)) * np.uint64(ncols)) >> np.uint64(32)
            for c in cand.tolist():
                if c not in seen:
                    seen.add(c)
                    got.append(c)
                    if len(got) == deg:
                        break
            t += 2 * deg
        cols[r] = np.sort(np.array(got, dtype=np.int64))
    return CSR(nrows, ncols, np.arange(nrows + 1, dtype=np.int64) * deg,
               cols.reshape(-1).astype(np.int32))


def counter_values_u32(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    x = counter_draw(seed, np.arange(n, dtype=np.uint64))
    return (np.uint64(lo) + (((x >> np.uint64(32)) * np.uint64(hi - lo + 1)) >> np.uint64(32))).astype(np.uint32)


def counter_values_f64(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    x = counter_draw(seed, np.arange(n, dtype=np.uint64))
    return lo + (hi - lo) * ((x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)


def batched_plan(count: int = 4096, cfg: int = 4):
    """Shapes of the batched workload: product i has n_i = floor(exp U(ln 256,
    ln 65536)), ER degree d_i uniform in 4..64, semiring (min,+) u32 in [1,1000]
    for the first half and (+,x) fp64 U(-1,1) for the second; A_i and B_i
    are n_i x n_i with independent seeds."""
    out = []
    for i in range(count):
        rng = rng_for(cfg, 200, i)
        n = int(math.exp(rng.uniform(math.log(256), math.log(65536))))
        d = int(rng.integers(4, 65))
        sr = "min_plus_u32" if i < count // 2 else "plus_times_f64"
        out.append({"i": i, "n": n, "deg": d, "semiring": sr,
                    "seed_a": subseed(cfg, 201, i), "seed_b": subseed(cfg, 202, i),
                    "seed_va": subseed(cfg, 203, i), "seed_vb": subseed(cfg, 204, i)})
    return out


def batched_product_host(p: dict):
    """One product of the batched workload on the host (for the oracle)."""
    A = er_counter(p["seed_a"], p["n"], p["n"], p["deg"])
    B = er_counter(p["seed_b"], p["n"], p["n"], p["deg"])
    if p["semiring"] == "min_plus_u32":
        A = A.with_values(counter_values_u32(p["seed_va"], A.nnz, 1, 1000))
        B = B.with_values(counter_values_u32(p["seed_vb"], B.nnz, 1, 1000))
    else:
        A = A.with_values(counter_values_f64(p["seed_va"], A.nnz, -1.0, 1.0))
        B = B.with_values(counter_values_f64(p["seed_vb"], B.nnz, -1.0, 1.0))
    return A, B
