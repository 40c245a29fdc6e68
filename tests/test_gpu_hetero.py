"""Parity of the heterogeneous semiring on the GPU with the CPU oracle
(paper Sec. 1: operations over three value types).

maxw_label: A float32 weights, B int32 labels, C cb_wlabel (weight, label)
records, bit-exact (the (+) only compares).  Covers every tier (the
one-launch kernel, the hash teams, the rank windows of heavy rows with
their L2 accumulators), exact / learned / upper-bound sizing, column
batches, stacked batches next to a one-type semiring in every mode,
SpMSpV, IEEE special weights, and the merge of partial results.
"""
import numpy as np
import pytest

import oracle
from oracle.spmspv import spmspv as spmspv_oracle
from paper_2106_14402_gb300 import gen
from parity import check_structure, compare_rows, sample_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SR = "maxw_label"


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def weights(M, seed, levels=4):
    return M.with_values(gen.hetero_values(SR, "A", M.nnz, seed, levels=levels))


def labels(M, seed, hi=None):
    if hi is None:
        return M.with_values(gen.hetero_values(SR, "B", M.nnz, seed))
    return M.with_values(np.random.default_rng(seed).integers(0, hi, M.nnz).astype(np.int32))


def run(cb, A, B, **kw):
    dA = cb.DeviceCSR.from_host(A, SR, operand="A")
    dB = cb.DeviceCSR.from_host(B, SR, operand="B")
    C = cb.spgemm(SR, dA, dB, **kw)
    torch.cuda.synchronize()
    return C


def parity(cb, A, B, rows=None, **kw):
    got = run(cb, A, B, check=True, **kw).to_host()
    check_structure(got[0], got[1], B.ncols)
    compare_rows(SR, got, oracle.spgemm(SR, A, B, rows=rows), rows=rows)
    return got


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("levels", [0, 3])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1.0), (7, 5, 9, 0.5), (40, 33, 50, 0.2),
                                   (200, 150, 300, 0.05), (64, 1, 64, 0.9), (3, 100, 1, 0.3)])
def test_small_random(cb, shape, levels, fused):
    m, n, k, d = shape
    A = weights(gen.random_csr(m, n, d, seed=m * 7 + n, empty_rows=0.15, full_rows=0.05), 1, levels)
    B = labels(gen.random_csr(n, k, d, seed=k * 11 + n, empty_rows=0.15, full_rows=0.05), 2, hi=20)
    parity(cb, A, B, fused=fused)


@pytest.mark.parametrize("fused", [True, False])
def test_duplicates_unsorted_and_special_weights(cb, fused):
    pool = np.concatenate([np.array([-0.0, 0.0, np.inf, -np.inf, 0.5, -0.5, 1e-45], np.float32),
                           np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFFFFFFF],
                                    np.uint32).view(np.float32)])
    P = gen.random_csr(150, 90, 0.08, seed=5, duplicates=True, shuffle=True, empty_rows=0.1)
    A = P.with_values(pool[np.random.default_rng(6).integers(0, pool.size, P.nnz)])
    B = labels(gen.random_csr(90, 160, 0.08, seed=7, duplicates=True, shuffle=True), 8, hi=6)
    parity(cb, A, B, fused=fused)


SPECIAL = np.concatenate([np.array([-0.0, 0.0, np.inf, -np.inf, 0.5, -0.5, 1e-45], np.float32),
                          np.array([0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFFFFFFF],
                                   np.uint32).view(np.float32)])


@pytest.mark.parametrize("case", ["one_launch", "queue", "rank_windows"])
def test_special_weights_on_every_path(cb, case):
    """NaN payloads, infinities and signed zeros as weights through the
    one-launch kernel (ER, 8 per row), the work-queue kernel (ER rows of 40
    entries) and the hash tiers plus rank windows (R-MAT scale 12)."""
    if case == "one_launch":
        P = gen.er_exact(4096, 4096, 8, gen.subseed(90, 0))
    elif case == "queue":
        P = gen.er_exact(3000, 3000, 40, gen.subseed(90, 1))
    else:
        P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=gen.subseed(90, 2))
    A = P.with_values(SPECIAL[np.random.default_rng(91).integers(0, SPECIAL.size, P.nnz)])
    B = labels(P, 92, hi=6)
    got = parity(cb, A, B)
    if case == "rank_windows":
        assert np.diff(got[0]).max() > 512


@pytest.mark.parametrize("fused", [True, False])
def test_er_small_rows(cb, fused):
    P = gen.er_exact(16384, 16384, 8, gen.subseed(60, 0))
    A, B = weights(P, 61, levels=16), labels(P, 62)
    C = run(cb, A, B, fused=fused)
    got = C.to_host()
    compare_rows(SR, got, oracle.spgemm(SR, A, B))


@pytest.mark.parametrize("sizing", ["exact", "learned", "upper_bound"])
def test_rmat_all_tiers(cb, sizing):
    """R-MAT scale 14: warp, 256- and 512-thread hash teams and rank windows
    (rows with more than 512 output entries), every row compared."""
    P = gen.rmat(14, 16, *gen.RMAT_ABCD, seed=gen.subseed(70, 0))
    A, B = weights(P, 71, levels=8), labels(P, 72, hi=1000)
    mlp = None
    if sizing == "learned":
        from paper_2106_14402_gb300 import sizer
        mlp, _ = sizer.load()
    got = parity(cb, A, B, sizing=sizing, mlp=mlp)
    assert np.diff(got[0]).max() > 512   # heavy rows reach the rank windows


def test_rmat_s16_sampled(cb):
    P = gen.rmat(16, 16, *gen.RMAT_ABCD, seed=gen.subseed(80, 0))
    A, B = weights(P, 81), labels(P, 82)
    flops, _ = oracle.row_stats(A, B)
    rows = sample_rows(A.nrows, flops, frac=0.01, top=50, seed=83)
    parity(cb, A, B, rows=rows)


def test_column_batches(cb):
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=gen.subseed(90, 0))
    A, B = weights(P, 91, levels=5), labels(P, 92)
    want = oracle.spgemm(SR, A, B)
    nnz = int(want[0][-1])
    budget = 8 * (A.nrows + 1) + (nnz // 5) * 12
    dA = cb.DeviceCSR.from_host(A, SR, operand="A")
    dB = cb.DeviceCSR.from_host(B, SR, operand="B")
    parts = []
    st = cb.spgemm_column_batches(SR, dA, dB, budget,
                                  lambda b, lo, hi, Cb: parts.append((lo, Cb.to_host())) and False)
    assert st["batches"] >= 5 and len(parts) == st["batches"]
    m = A.nrows
    rows_col = [[] for _ in range(m)]
    rows_val = [[] for _ in range(m)]
    for lo, (rp, col, val) in sorted(parts, key=lambda t: t[0]):
        for i in range(m):
            rows_col[i].append(col[rp[i]:rp[i + 1]])
            rows_val[i].append(val[rp[i]:rp[i + 1]])
    rp = np.zeros(m + 1, np.int64)
    rp[1:] = np.cumsum([sum(len(c) for c in rc) for rc in rows_col])
    col = np.concatenate([np.concatenate(rc) for rc in rows_col])
    val = np.concatenate([np.concatenate(rv) for rv in rows_val])
    compare_rows(SR, (rp, col, val), want)


@pytest.mark.parametrize("mode", ["host", "sync_free", "graph"])
def test_stacked_batches_beside_fp64(cb, mode):
    """Batched products mixing the heterogeneous semiring with (+,x) fp64:
    the stacking copies A's and B's values with their own sizes."""
    plan = []
    for t in range(6):
        P = gen.er_exact(300 + 50 * t, 300 + 50 * t, 6 + t, gen.subseed(100, t))
        if t % 2 == 0:
            plan.append((SR, weights(P, 200 + t, levels=4), labels(P, 300 + t, hi=50)))
        else:
            plan.append(("plus_times_f64", P.with_values(gen.random_values("plus_times_f64", P.nnz, 400 + t)),
                         P.with_values(gen.random_values("plus_times_f64", P.nnz, 500 + t))))
    As = [cb.DeviceCSR.from_host(A, sr, operand="A") for sr, A, _ in plan]
    Bs = [cb.DeviceCSR.from_host(B, sr, operand="B") for sr, _, B in plan]
    want = [oracle.spgemm(sr, A, B) for sr, A, B in plan]
    if mode == "graph":
        seen = []
        st = cb.spgemm_batched([p[0] for p in plan], As, Bs, lambda *a: seen.append(a), mode="graph")
        assert st["nnz"] == sum(int(w[0][-1]) for w in want)
        return
    got = {}

    def on_wave(w, first, end, Cw):
        rp, col, val = Cw.to_host()
        r0 = 0
        for i in range(first, end):
            n = plan[i][1].nrows
            got[i] = (rp[r0:r0 + n + 1] - rp[r0], col[rp[r0]:rp[r0 + n]], val[rp[r0]:rp[r0 + n]])
            r0 += n

    cb.spgemm_batched([p[0] for p in plan], As, Bs, on_wave, mode=mode)
    assert sorted(got) == list(range(len(plan)))
    for i, (sr, _, _) in enumerate(plan):
        compare_rows(sr, got[i], want[i])


def test_spmspv(cb):
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=gen.subseed(110, 0))
    A = labels(P, 111, hi=100)
    dA = cb.DeviceCSR.from_host(A, SR, operand="B")
    rng = np.random.default_rng(112)
    for nx in (1, 50, 2000):
        x_idx = rng.choice(A.nrows, nx, replace=False).astype(np.int32)
        x_val = gen.hetero_values(SR, "A", nx, 113 + nx, levels=4)
        w_idx, w_val, _ = spmspv_oracle(SR, A, x_idx, x_val)
        for bucket in (False, True):
            y_idx, y_val = cb.spmspv(SR, dA, torch.from_numpy(x_idx).cuda(), torch.from_numpy(x_val).cuda(),
                                     bucket=bucket)
            assert np.array_equal(y_idx.cpu().numpy(), w_idx)
            assert np.array_equal(y_val.cpu().numpy().view(np.uint64), w_val.view(np.uint64))


def test_wlabel_split(cb):
    P = gen.random_csr(30, 30, 0.2, seed=120)
    A, B = weights(P, 121), labels(P, 122, hi=9)
    C = run(cb, A, B)
    w, lab = cb.wlabel_split(C.val)
    want = oracle.spgemm(SR, A, B)
    assert np.array_equal(w.cpu().numpy(), want[2]["w"])
    assert np.array_equal(lab.cpu().numpy(), want[2]["label"])


def test_merge_of_partial_products(cb):
    """The merge combines (weight, label) records (the selector product in
    the semiring's merge form): the partial products of a split inner
    dimension merge back into the product; unsorted parts with duplicate
    coordinates merge as the oracle says."""
    P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=130)
    A, B = weights(P, 131, levels=3), labels(P, 132, hi=40)
    cuts = np.linspace(0, A.ncols, 6).astype(int)
    dB = cb.DeviceCSR.from_host(B, SR, operand="B")
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    parts = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        keep = (A.col >= lo) & (A.col < hi)
        rp = np.zeros(A.nrows + 1, np.int64)
        np.add.at(rp, rows[keep] + 1, 1)
        L = gen.CSR(A.nrows, A.ncols, np.cumsum(rp), A.col[keep], A.val[keep])
        parts.append(cb.spgemm(SR, cb.DeviceCSR.from_host(L, SR, operand="A"), dB))
    C = cb.merge(SR, parts)
    torch.cuda.synchronize()
    compare_rows(SR, C.to_host(), oracle.spgemm(SR, A, B))
    hparts = []
    for t in range(3):
        Q = gen.random_csr(300, 200, 0.05, seed=140 + t, shuffle=True, duplicates=True, empty_rows=0.2)
        rec = np.zeros(Q.nnz, oracle.WLABEL)
        rec["w"] = gen.hetero_values(SR, "A", Q.nnz, 150 + t, levels=3)
        rec["label"] = np.random.default_rng(160 + t).integers(0, 9, Q.nnz)
        hparts.append(Q.with_values(rec))
    for fused in (True, False):
        C = cb.merge(SR, [cb.DeviceCSR.from_host(Q, SR, operand="C") for Q in hparts], fused=fused)
        got = C.to_host()
        check_structure(got[0], got[1], 200)
        compare_rows(SR, got, oracle.merge(SR, hparts))


@pytest.mark.parametrize("fused", [True, False])
def test_golden_worked_example(cb, fused):
    """The hand-derived example of tests/golden/maxw_label_example.json."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "maxw_label_example.json")))
    A = gen.CSR(*g["A"]["shape"], np.array(g["A"]["row_ptr"], np.int64), np.array(g["A"]["col"], np.int32),
                np.array(g["A"]["val"], np.float32))
    B = gen.CSR(*g["B"]["shape"], np.array(g["B"]["row_ptr"], np.int64), np.array(g["B"]["col"], np.int32),
                np.array(g["B"]["val"], np.int32))
    rp, col, val = run(cb, A, B, fused=fused).to_host()
    assert np.array_equal(rp, g["C"]["row_ptr"]) and np.array_equal(col, g["C"]["col"])
    rec = val.view(oracle.WLABEL)
    assert np.array_equal(rec["w"].view(np.uint32), np.array(g["C"]["w"], np.float32).view(np.uint32))
    assert np.array_equal(rec["label"], g["C"]["label"])
