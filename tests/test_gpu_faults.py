"""Failure paths under fault injection (cb_ctx_set_fault), with nothing that
faults, traps or hangs the GPU.

* A bounded device wait that runs out: the one-launch kernel's look-back
  waits on an earlier tile's published total.  With one tile made silent
  (it never publishes) and waits limited to a few polls, the waiting tiles
  give up, record CB_FUSED_STALLED and publish anyway, so the launch ends;
  cb_spgemm_ex returns CB_ERR_TIMEOUT with C zeroed, and the context works
  afterwards.
* Device allocations that fail: the k-th allocation the context makes
  returns out-of-memory; every call path returns CB_ERR_OOM with C zeroed
  (nothing leaked to the caller), and the same context then computes the
  product exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CB_ERR_OOM = 5
CB_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


@pytest.fixture(scope="module")
def er():
    (sr, A, _), = gen.er_square(n=4096, deg=8, cfg=71)
    return sr, A, oracle.spgemm(sr, A, A)


@pytest.mark.parametrize("tile", [0, 5, 100])
def test_wait_that_runs_out_returns_timeout(cb, er, tile):
    sr, A, want = er
    ctx = cb.Context()
    dA = cb.DeviceCSR.from_host(A, sr)
    ctx.set_fault(cb.FAULT_SILENT_TILE, tile, 64)
    with pytest.raises(cb.CBError) as e:
        cb.spgemm(sr, dA, dA, ctx=ctx)
    assert e.value.code == CB_ERR_TIMEOUT
    assert "wait expired" in ctx.error()
    torch.cuda.synchronize()
    # the context (and its tile status words) still serve a normal call
    ctx.set_fault(cb.FAULT_SILENT_TILE, -1)
    C = cb.spgemm(sr, dA, dA, ctx=ctx)
    compare_rows(sr, C.to_host(), want)


def test_wait_that_runs_out_sets_the_stall_bit(cb, er):
    sr, A, want = er
    ctx = cb.Context()
    dA = cb.DeviceCSR.from_host(A, sr)
    lanes, flops = cb.fused_lanes(dA, dA, ctx=ctx)
    assert lanes == 8
    out = cb.DeviceCSR(A.nrows, A.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device="cuda"),
                       torch.empty(flops, dtype=torch.int32, device="cuda"),
                       torch.empty(flops, dtype=torch.int64, device="cuda"))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.set_fault(cb.FAULT_SILENT_TILE, 3, 16)
    cb.spgemm_fused(sr, dA, dA, out, status, lanes=lanes, ctx=ctx)
    torch.cuda.synchronize()                      # the launch ends
    assert int(status.item()) & cb.FUSED_STALLED
    ctx.set_fault(cb.FAULT_SILENT_TILE, -1)
    status.zero_()
    cb.spgemm_fused(sr, dA, dA, out, status, lanes=lanes, ctx=ctx)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    n = int(out.row_ptr[-1].item())
    got = cb.DeviceCSR(A.nrows, A.ncols, out.row_ptr, out.col[:n], out.val[:n]).to_host()
    compare_rows(sr, got, want)


def test_fault_arguments_are_checked(cb):
    ctx = cb.Context()
    for kind, arg, arg2 in ((9, 1, 1), (cb.FAULT_ALLOC, -1, 0), (cb.FAULT_SILENT_TILE, 2, 0),
                            (cb.FAULT_SILENT_TILE, 2, (1 << 20) + 1)):
        with pytest.raises(cb.CBError) as e:
            ctx.set_fault(kind, arg, arg2)
        assert e.value.code == 1


@pytest.fixture(scope="module")
def heavy():
    sr = "plus_times_f64"
    P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=72)
    A = P.with_values(gen.random_values(sr, P.nnz, 73))
    flops, _ = oracle.row_stats(A, A)
    assert flops.max() > 4096          # hash tiers and rank windows both run
    return sr, A, oracle.spgemm(sr, A, A)


def _oom_sweep(cb, run, check, kmax=12):
    """Fail the k-th allocation for k = 1, 2, ... on fresh contexts until a call
    succeeds; every failure must be CB_ERR_OOM and leave the context usable."""
    failures = 0
    for k in range(1, kmax + 1):
        ctx = cb.Context()
        ctx.set_fault(cb.FAULT_ALLOC, k)
        try:
            res = run(ctx)
        except cb.CBError as e:
            assert e.code == CB_ERR_OOM, (k, e.code, str(e))
            failures += 1
            check(run(ctx))   # the fault fired once; the same context now succeeds
            continue
        check(res)
        return failures, k
    raise AssertionError("every allocation up to kmax failed")


def test_allocation_failures_two_phase(cb, heavy):
    sr, A, want = heavy
    dA = cb.DeviceCSR.from_host(A, sr)

    def run(ctx):
        return cb.spgemm(sr, dA, dA, ctx=ctx, fused=False).to_host()

    failures, k = _oom_sweep(cb, run, lambda got: compare_rows(sr, got, want))
    # workspaces, heavy-row workspace, C's row pointers, columns and values
    assert failures >= 4, failures


def test_allocation_failures_learned(cb, heavy):
    from paper_2106_14402_gb300 import sizer
    model, _ = sizer.load()
    sr, A, want = heavy
    dA = cb.DeviceCSR.from_host(A, sr)

    def run(ctx):
        return cb.spgemm(sr, dA, dA, ctx=ctx, sizing="learned", mlp=model).to_host()

    failures, _ = _oom_sweep(cb, run, lambda got: compare_rows(sr, got, want))
    assert failures >= 5, failures


def test_allocation_failures_column_batched(cb, heavy):
    sr, A, want = heavy
    dA = cb.DeviceCSR.from_host(A, sr)
    budget = 8 * (A.nrows + 1) + int(want[0][-1]) * 12 // 3

    def run(ctx):
        parts = []

        def on_batch(b, lo, hi, Cb):
            rp, col, val = Cb.to_host()
            parts.append((lo, rp, col, val))

        st = cb.spgemm_column_batches(sr, dA, dA, budget, on_batch, ctx=ctx)
        return st, parts

    def check(res):
        st, parts = res
        assert st["batches"] >= 3 and len(parts) == st["batches"]
        # reassemble the rows from the column batches and compare
        rows_col = [[] for _ in range(A.nrows)]
        rows_val = [[] for _ in range(A.nrows)]
        for lo, rp, col, val in sorted(parts, key=lambda p: p[0]):
            for i in range(A.nrows):
                rows_col[i].append(col[rp[i]:rp[i + 1]])
                rows_val[i].append(val[rp[i]:rp[i + 1]])
        cols = [np.concatenate(c) for c in rows_col]
        vals = [np.concatenate(v) for v in rows_val]
        rp = np.zeros(A.nrows + 1, np.int64)
        rp[1:] = np.cumsum([c.size for c in cols])
        compare_rows(sr, (rp, np.concatenate(cols), np.concatenate(vals)), want)

    failures, _ = _oom_sweep(cb, run, check)
    assert failures >= 2, failures


def test_allocation_failures_batched(cb):
    plan = []
    for p in gen.batched_plan(6, cfg=41):
        p = dict(p)
        p["n"] = 256 + (p["n"] % 1000)
        plan.append(p)
    from paper_2106_14402_gb300 import gen_device
    As = [gen_device.er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"]) for p in plan]
    Bs = [gen_device.er(p["seed_b"], p["n"], p["deg"], p["semiring"], p["seed_vb"]) for p in plan]
    want = [oracle.spgemm(p["semiring"], *gen.batched_product_host(p)) for p in plan]

    def run(ctx):
        got = {}

        def on_wave(w, first, end, Cw):
            rp, col, val = Cw.to_host()
            r0 = 0
            for i in range(first, end):
                n = plan[i]["n"]
                got[i] = (rp[r0:r0 + n + 1] - rp[r0], col[rp[r0]:rp[r0 + n]], val[rp[r0]:rp[r0 + n]])
                r0 += n

        cb.spgemm_batched([p["semiring"] for p in plan], As, Bs, on_wave, ctx=ctx)
        return got

    def check(got):
        assert len(got) == len(plan)
        for i, p in enumerate(plan):
            compare_rows(p["semiring"], got[i], want[i])

    failures, _ = _oom_sweep(cb, run, check, kmax=40)
    assert failures >= 3, failures
