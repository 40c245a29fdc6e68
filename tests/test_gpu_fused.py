"""Parity of the one-launch SpGEMM for small rows (cb_spgemm_fused, and the
automatic branch of cb_spgemm_ex) with the CPU oracle.

Covers the three lane widths (8, 16, 32 lanes per row: rows of A up to 8 /
16 / 32 entries, up to 64 / 128 / 256 products), all five semirings,
duplicate and unsorted columns (long runs of one column spanning several
lanes), empty rows and ragged tile tails, more tiles than resident CTAs
(each CTA walks several tiles, look-backs longer than one window), the
error bits (row beyond the bounds, capacity), repeated launches (the
launch epoch of the tile status words) and replay inside a CUDA graph.
"""
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


def bounded_rows(nrows, ncols, max_len, seed, sr, duplicates=False, shuffle=False, empty=0.1):
    """Rows of 0..max_len stored entries (columns drawn with replacement when
    `duplicates`, else distinct), seeded."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len + 1, nrows)
    lens[rng.random(nrows) < empty] = 0
    cols = []
    for ln in lens:
        if duplicates:
            c = rng.integers(0, ncols, ln)
        else:
            c = rng.choice(ncols, size=min(int(ln), ncols), replace=False)
        cols.append(c if shuffle else np.sort(c))
    lens = np.array([c.size for c in cols], np.int64)
    rp = np.zeros(nrows + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate(cols).astype(np.int32) if nrows else np.zeros(0, np.int32)
    M = gen.CSR(nrows, ncols, rp, col)
    return M.with_values(gen.random_values(sr, M.nnz, seed + 1))


def run_fused(cb, sr, A, B, lanes, capacity=None):
    dA = cb.DeviceCSR.from_host(A, sr)
    dB = dA if B is A else cb.DeviceCSR.from_host(B, sr)
    flops, _ = oracle.row_stats(A, B)
    cap = int(flops.sum()) if capacity is None else capacity
    dt = cb.SEMIRING[sr][1]
    out = cb.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                       torch.empty(cap, dtype=torch.int32, device="cuda"),
                       torch.empty(cap, dtype=dt, device="cuda"))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cb.spgemm_fused(sr, dA, dB, out, status, lanes=lanes)
    torch.cuda.synchronize()
    rp = out.row_ptr.cpu().numpy()
    n = int(rp[-1])
    C = cb.DeviceCSR(A.nrows, B.ncols, out.row_ptr, out.col[:min(n, cap)], out.val[:min(n, cap)])
    return C.to_host(), int(status.item())


# (lanes, max A row, max B row, ncols)
SHAPES = [(8, 8, 8, 20000), (16, 16, 8, 5000), (32, 32, 8, 300), (32, 16, 16, 100000)]


@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_matches_oracle(cb, sr, shape):
    lanes, amax, bmax, ncols = shape
    A = bounded_rows(1000 + lanes * 3 + 1, 700, amax, seed=lanes + amax, sr=sr)
    B = bounded_rows(700, ncols, bmax, seed=lanes + bmax + 50, sr=sr)
    got, st = run_fused(cb, sr, A, B, lanes)
    assert st == 0
    check_structure(got[0], got[1], B.ncols)
    compare_rows(sr, got, oracle.spgemm(sr, A, B))


@pytest.mark.parametrize("sr", SR)
@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_fused_duplicates_and_long_runs(cb, sr, lanes):
    # B over 6 columns: a row's products collapse into runs of one column that
    # cross lane boundaries; A and B hold repeated, unsorted columns
    lo, hi = {"plus_times_i64": (-3, 3), "plus_times_f64": (-1.0, 1.0), "min_plus_u32": (0, 5),
              "or_and_bool": (0, 1), "sel2nd_min_i32": (-4, 4)}[sr]
    A = bounded_rows(517, 40, lanes, seed=3 * lanes, sr=sr, duplicates=True, shuffle=True)
    B = bounded_rows(40, 6, 8, seed=3 * lanes + 1, sr=sr, duplicates=True, shuffle=True)
    A = A.with_values(gen.random_values(sr, A.nnz, 11, lo=lo, hi=hi))
    B = B.with_values(gen.random_values(sr, B.nnz, 12, lo=lo, hi=hi))
    got, st = run_fused(cb, sr, A, B, lanes)
    assert st == 0
    compare_rows(sr, got, oracle.spgemm(sr, A, B))


def test_fused_er_square_workload(cb):
    # n = 16384, exactly 8 distinct columns per row, C = A.A over (+,x) int64
    (sr, A, B), = gen.er_square()
    assert cb.fused_lanes(cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(A, sr))[0] == 8
    got, st = run_fused(cb, sr, A, A, 8)
    assert st == 0
    compare_rows(sr, got, oracle.spgemm(sr, A, A))


def test_fused_many_tiles(cb):
    # 8 rows per tile at 32 lanes: ~40k tiles, far more than resident CTAs,
    # so CTAs walk several tiles and look-backs cross 256-tile windows
    sr = "plus_times_i64"
    A = bounded_rows(320_003, 50_000, 32, seed=71, sr=sr)
    B = bounded_rows(50_000, 1_000_000, 8, seed=72, sr=sr)
    got, st = run_fused(cb, sr, A, B, 32)
    assert st == 0
    check_structure(got[0], got[1], B.ncols)
    compare_rows(sr, got, oracle.spgemm(sr, A, B))


def test_fused_error_bits(cb):
    sr = "plus_times_f64"
    A = bounded_rows(300, 100, 8, seed=80, sr=sr, empty=0.0)
    B = bounded_rows(100, 500, 8, seed=81, sr=sr)
    want = oracle.spgemm(sr, A, B)
    nnz = int(want[0][-1])
    # capacity one short: the bit is set, row pointers are still complete
    got, st = run_fused(cb, sr, A, B, 8, capacity=nnz - 1)
    assert st & cb.FUSED_CAPACITY and not st & cb.FUSED_ROW_TOO_LARGE
    assert np.array_equal(got[0], want[0])
    # a row of A with 9 entries is beyond 8 lanes
    A9 = bounded_rows(300, 100, 9, seed=82, sr=sr, empty=0.0)
    assert np.diff(A9.row_ptr).max() == 9
    _, st = run_fused(cb, sr, A9, B, 8)
    assert st & cb.FUSED_ROW_TOO_LARGE
    # a B row of 9 entries under an A row of 8 makes > 64 products
    B9 = bounded_rows(100, 500, 9, seed=83, sr=sr, empty=0.0)
    f, _ = oracle.row_stats(A, B9)
    if f.max() > 64:
        _, st = run_fused(cb, sr, A, B9, 8)
        assert st & cb.FUSED_ROW_TOO_LARGE
    # the context still works afterwards
    got, st = run_fused(cb, sr, A, B, 8)
    assert st == 0
    compare_rows(sr, got, want)


def test_fused_empty(cb):
    sr = "min_plus_u32"
    for m, n, k in [(0, 5, 5), (7, 0, 5), (7, 5, 0), (33, 5, 5)]:
        A = bounded_rows(m, n, 0 if n == 0 else 4, seed=90, sr=sr, empty=1.0 if m == 33 else 0.0)
        B = bounded_rows(n, k, 0 if k == 0 else 4, seed=91, sr=sr)
        got, st = run_fused(cb, sr, A, B, 8)
        assert st == 0 and got[0].shape == (m + 1,) and np.all(got[0] == 0)


def test_fused_lanes_choice(cb):
    sr = "plus_times_i64"
    for amax, bmax, want in [(8, 8, 8), (9, 8, 16), (16, 8, 16), (8, 16, 16), (32, 8, 32),
                             (33, 1, 0), (8, 40, 0)]:
        A = bounded_rows(200, 300, amax, seed=amax * 100 + bmax, sr=sr, empty=0.0)
        B = bounded_rows(300, 1000, bmax, seed=amax * 100 + bmax + 1, sr=sr, empty=0.0)
        f, _ = oracle.row_stats(A, B)
        la = np.diff(A.row_ptr).max()
        expect = next((L for L in (8, 16, 32) if la <= L and f.max() <= 8 * L), 0)
        lanes, flops = cb.fused_lanes(cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(B, sr))
        assert lanes == expect and flops == int(f.sum())


def test_fused_repeated_launches_and_graph_replay(cb):
    """Tile status words are reused across launches through the launch epoch;
    the launch also replays correctly from a CUDA graph."""
    sr = "plus_times_i64"
    ctx = cb.Context(torch.cuda.Stream())
    mats = [bounded_rows(n, 3000, 8, seed=n, sr=sr) for n in (5000, 300, 9000, 5000)]
    B = bounded_rows(3000, 3000, 8, seed=7, sr=sr)
    dB = cb.DeviceCSR.from_host(B, sr)
    with torch.cuda.stream(ctx.stream):
        for A in mats:
            dA = cb.DeviceCSR.from_host(A, sr)
            cap = int(oracle.row_stats(A, B)[0].sum())
            out = cb.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                               torch.empty(cap, dtype=torch.int32, device="cuda"),
                               torch.empty(cap, dtype=torch.int64, device="cuda"))
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            cb.spgemm_fused(sr, dA, dB, out, status, lanes=8, ctx=ctx)
            ctx.stream.synchronize()
            assert int(status.item()) == 0
            n = int(out.row_ptr[-1].item())
            got = cb.DeviceCSR(A.nrows, B.ncols, out.row_ptr, out.col[:n], out.val[:n]).to_host()
            compare_rows(sr, got, oracle.spgemm(sr, A, B))

    # graph: capture once (status reset + launch), replay with new A values
    A = mats[0]
    dA = cb.DeviceCSR.from_host(A, sr)
    cap = int(oracle.row_stats(A, B)[0].sum())
    out = cb.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                       torch.empty(cap, dtype=torch.int32, device="cuda"),
                       torch.empty(cap, dtype=torch.int64, device="cuda"))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=ctx.stream):
        status.zero_()
        cb.spgemm_fused(sr, dA, dB, out, status, lanes=8, ctx=ctx)
    for rep in range(4):
        vals = gen.random_values(sr, A.nnz, 1000 + rep)
        dA.val.copy_(torch.from_numpy(vals))
        graph.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        n = int(out.row_ptr[-1].item())
        got = cb.DeviceCSR(A.nrows, B.ncols, out.row_ptr, out.col[:n], out.val[:n]).to_host()
        compare_rows(sr, got, oracle.spgemm(sr, A.with_values(vals), B))


@pytest.mark.parametrize("sr", ("plus_times_f64", "or_and_bool"))
def test_automatic_branch_matches_two_phase(cb, sr):
    A = bounded_rows(4097, 4000, 16, seed=120, sr=sr)
    B = bounded_rows(4000, 9000, 8, seed=121, sr=sr)
    dA, dB = cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(B, sr)
    ctx = cb.context()
    C1 = cb.spgemm(sr, dA, dB, fused=True)
    k1 = ctx.stats()["kernels"]
    C2 = cb.spgemm(sr, dA, dB, fused=False)
    k2 = ctx.stats()["kernels"]
    # the operands' mean row lengths fit 8 lanes, so the one-launch kernel is
    # tried first; rows of 16 entries exceed them and the call falls back to
    # the classified path: validation (2) + the tried launch (1) + sortedness,
    # flops and binning (3) + the one-launch kernel at 16 lanes (1)
    assert k1 == 7 and k2 > k1
    want = oracle.spgemm(sr, A, B)
    compare_rows(sr, C1.to_host(), want)
    compare_rows(sr, C2.to_host(), want)


def test_speculative_launch_falls_back_on_one_large_row(cb):
    """Mean row lengths small enough for 8 lanes, but one dense row of A
    (300 entries): the speculative one-launch pass reports it, nothing of its
    output is kept, and the classified path computes the exact product."""
    sr = "plus_times_i64"
    (_, A, _), = gen.er_square(n=2048, deg=4, cfg=81)
    rng = np.random.default_rng(82)
    dense = np.sort(rng.choice(2048, 300, replace=False)).astype(np.int32)
    rp = A.row_ptr.copy()
    col = np.concatenate([A.col[:rp[5]], dense, A.col[rp[6]:]])
    rp[6:] += 300 - (rp[6] - rp[5])
    M = gen.CSR(2048, 2048, rp, col)
    M = M.with_values(gen.random_values(sr, M.nnz, 83))
    dM = cb.DeviceCSR.from_host(M, sr)
    ctx = cb.context()
    C = cb.spgemm(sr, dM, dM, ctx=ctx)
    assert ctx.stats()["kernels"] > 3
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, M, M))


def test_speculative_launch_into_caller_buffers(cb):
    """Exact-degree ER: the speculative pass alone forms C (validation + one
    launch), into caller buffers; a buffer one entry short is reported as a
    capacity error."""
    (sr, A, _), = gen.er_square(n=4096, deg=8, cfg=84)
    dA = cb.DeviceCSR.from_host(A, sr)
    want = oracle.spgemm(sr, A, A)
    nnz = int(want[0][-1])
    ctx = cb.context()
    out = cb.DeviceCSR(A.nrows, A.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                       torch.empty(nnz, dtype=torch.int32, device="cuda"),
                       torch.empty(nnz, dtype=torch.int64, device="cuda"))
    C = cb.spgemm(sr, dA, dA, out=out, ctx=ctx)
    st = ctx.stats()
    assert st["kernels"] == 3 and st["nnz"] == nnz and st["flops"] == A.nrows * 64
    compare_rows(sr, C.to_host(), want)
    short = cb.DeviceCSR(A.nrows, A.ncols, out.row_ptr, out.col[:nnz - 1], out.val[:nnz - 1])
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, dA, out=short, ctx=ctx)
    assert e.value.code == 9
