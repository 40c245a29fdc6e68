"""Learned sizing (paper Sec. 5: approximate memory estimation in place of
the symbolic phase; Sec. 7.4: batch count from such an estimate).

The MLP's predicted row sizes set hash-table capacities and the column-batch
count; rows that overflow their capacity are detected on the device and
recomputed exactly, so the output must equal the oracle's in every case,
including a deliberately bad predictor that overflows most rows.
"""
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


def small_family():
    out = []
    for s in (10, 11, 12):
        for k, a in enumerate((0.45, 0.55, 0.65)):
            bc = (0.95 - a) / 2
            out.append(gen.rmat(s, 16, a, bc, bc, seed=500 + 10 * s + k))
    for k, (n, d) in enumerate(((3000, 8), (5000, 24), (2000, 60))):
        out.append(gen.er_exact(n, n, d, seed=520 + k))
    for k, (n, bw, d) in enumerate(((3000, 16, 12), (4000, 100, 40))):
        out.append(gen.banded(n, bw, d, seed=530 + k))
    return out


@pytest.fixture(scope="module")
def trained(cb):
    from paper_2106_14402_gb300 import sizer
    feats, labels = zip(*(sizer.product_rows(A) for A in small_family()))
    feat, lab = torch.cat(feats), torch.cat(labels)
    model, losses = sizer.train(feat, lab, epochs=25, batch=2048, lr=3e-3, seed=1)
    assert losses[-1] < losses[0]
    return model


def held_out(sr, seed=600):
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=seed)
    if sr == "sel2nd_min_i32":
        return P.with_values(np.ones(P.nnz, np.int32)), P.with_values(gen.random_values(sr, P.nnz, seed + 2))
    A = P.with_values(gen.random_values(sr, P.nnz, seed + 1))
    return A, A


def dev(cb, sr, A, B):
    dA = cb.DeviceCSR.from_host(A, sr)
    return dA, (dA if B is A else cb.DeviceCSR.from_host(B, sr))


@pytest.mark.parametrize("sr", SR)
def test_learned_sizing_matches_oracle(cb, trained, sr):
    A, B = held_out(sr)
    dA, dB = dev(cb, sr, A, B)
    C = cb.spgemm(sr, dA, dB, sizing="learned", mlp=trained, check=True)
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, B))


def test_bad_predictor_overflows_and_falls_back(cb):
    from paper_2106_14402_gb300 import sizer
    params = sizer.init_params(3)
    params[-1] = -30.0                     # sigmoid(z) ~ 0: every capacity = max B row
    model = cb.MLP(params, np.array([0, 0, 0, 1, 1, 1], np.float32))
    sr = "plus_times_i64"
    A, B = held_out(sr, seed=610)
    dA, dB = dev(cb, sr, A, B)
    C = cb.spgemm(sr, dA, dB, sizing="learned", mlp=model, margin=0.0)
    st = cb.context().stats()
    assert st["overflow_rows"] > 100
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, B))


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32"))
def test_upper_bound_sizing(cb, sr):
    A, B = held_out(sr, seed=620)
    dA, dB = dev(cb, sr, A, B)
    C = cb.spgemm(sr, dA, dB, sizing="upper_bound")
    assert cb.context().stats()["overflow_rows"] == 0
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, B))


def test_learned_column_batches(cb, trained):
    sr = "plus_times_f64"
    A, B = held_out(sr, seed=630)
    dA, dB = dev(cb, sr, A, B)
    want = oracle.spgemm(sr, A, B)
    nnz = int(want[0][-1])
    budget = 8 * (A.nrows + 1) + (nnz // 4) * 12
    parts = []

    def on_batch(b, lo, hi, Cb):
        parts.append((lo, hi) + Cb.to_host())

    st = cb.spgemm_column_batches(sr, dA, dB, budget, on_batch, sizing="learned", mlp=trained)
    assert st["batches"] == len(parts) >= 4
    parts.sort()
    m = A.nrows
    rp = np.zeros(m + 1, np.int64)
    cols, vals = [], []
    for i in range(m):
        for lo, hi, prp, pcol, pval in parts:
            cols.append(pcol[prp[i]:prp[i + 1]])
            vals.append(pval[prp[i]:prp[i + 1]])
        rp[i + 1] = rp[i] + sum(len(c) for c in cols[-len(parts):])
    compare_rows(sr, (rp, np.concatenate(cols), np.concatenate(vals)), want)


def _column_batched(cb, sr, dA, dB, budget, sizing, mlp):
    parts = []

    def on_batch(b, lo, hi, Cb):
        parts.append((lo, hi) + Cb.to_host())

    st = cb.spgemm_column_batches(sr, dA, dB, budget, on_batch, sizing=sizing, mlp=mlp)
    assert st["batches"] == len(parts)
    parts.sort(key=lambda p: p[0])
    m = dA.nrows
    rp = np.zeros(m + 1, np.int64)
    cols, vals = [], []
    for i in range(m):
        n = 0
        for lo, hi, prp, pcol, pval in parts:
            cols.append(pcol[prp[i]:prp[i + 1]])
            vals.append(pval[prp[i]:prp[i + 1]])
            n += prp[i + 1] - prp[i]
        rp[i + 1] = rp[i] + n
    return (rp, np.concatenate(cols), np.concatenate(vals)), st


def test_learned_column_batches_unsorted_after_sorted(cb, trained):
    """Whether B's rows are sorted is decided per call: a call on a B with
    unsorted rows right after one on sorted rows must not reuse the slab
    offsets of sorted rows."""
    sr = "min_plus_u32"
    A, B = held_out(sr, seed=650)
    rng = np.random.default_rng(651)
    col, val = B.col.copy(), B.val.copy()
    for r in range(B.nrows):
        s0, e0 = B.row_ptr[r], B.row_ptr[r + 1]
        perm = rng.permutation(e0 - s0) + s0
        col[s0:e0], val[s0:e0] = col[perm], val[perm]
    Bu = gen.CSR(B.nrows, B.ncols, B.row_ptr, col, val)
    want = oracle.spgemm(sr, A, B)
    budget = 8 * (A.nrows + 1) + (int(want[0][-1]) // 5) * 8
    dA = cb.DeviceCSR.from_host(A, sr)
    for Bx in (B, Bu):
        got, st = _column_batched(cb, sr, dA, cb.DeviceCSR.from_host(Bx, sr), budget, "learned", trained)
        assert st["batches"] >= 4 and st["flops"] == int(oracle.row_stats(A, B)[0].sum())
        compare_rows(sr, got, want)


def test_what_the_trained_network_gains(cb, trained):
    """On a held-out product, the trained sizer (a 0.9-quantile estimate of
    each row's size) overflows on few rows while allocating clearly less
    than the flop bound min(flops_i, ncols), is closer to the exact sizes
    than that bound row by row, and scores a lower held-out training
    objective than the same network untrained."""
    from paper_2106_14402_gb300 import sizer
    A, _ = held_out("or_and_bool", seed=640)
    feat, y = sizer.product_rows(A)
    untrained = cb.MLP(sizer.init_params(1), sizer.normalisation(feat))
    good = sizer.evaluate(trained, feat, y, A.ncols)
    raw = sizer.evaluate(untrained, feat, y, A.ncols)
    assert good["sum_cap_over_sum_true"] < 2.0
    assert good["overflow_rows"] < 0.05
    assert good["sum_bound_over_sum_true"] > 1.8
    assert good["sum_cap_over_sum_true"] < 0.9 * good["sum_bound_over_sum_true"]
    live = feat[:, 1] > 0
    bound = torch.clamp(feat[live][:, 1].double(), max=A.ncols)
    yl = y[live].double()
    assert good["median_abs_log2_err"] < float(torch.median(torch.abs(torch.log2(bound) - torch.log2(yl))))
    # the pinball objective on the held-out rows, and the overflow rate
    _, loss_good = trained.grad(feat, y, tau=sizer.TAU)
    _, loss_raw = untrained.grad(feat, y, tau=sizer.TAU)
    assert float(loss_good.item()) < float(loss_raw.item())
    assert good["overflow_rows"] <= raw["overflow_rows"]
