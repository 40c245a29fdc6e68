"""The bounds-checking debug library (libcb_check.so, -DCB_CHECK): on valid
inputs no check fires and every path gives the oracle's result; with one
row's exact size made one short after the symbolic phase (fault injection),
the debug library reports the failed bound while the normal library stays
inside C's arrays (dropping the row's surplus entry, or reporting a
consistency failure under CB_FLAG_CHECK when a hash tier forms the row).

The debug library runs in a child process (CB_LIBRARY=check), one per test."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def run_child(body: str) -> dict:
    """Run body (which sets `out`, a JSON-able dict) under the debug library."""
    script = textwrap.dedent("""
        import json, sys
        import numpy as np, torch
        import oracle
        from paper_2106_14402_gb300 import cb, gen
        from parity import compare_rows
        lib = cb.load()
        assert cb.library_path().endswith("libcb_check.so")
        out = {}
    """) + textwrap.dedent(body) + "\nprint('RESULT ' + json.dumps(out))\n"
    env = dict(os.environ, CB_LIBRARY="check",
               PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", script], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[7:])


def test_debug_library_on_adversarial_cases(cb):
    """All products in one column, dense rows, ncols = 1, nrows = 0, an
    empty A, rows in every tier over several bitmap spans: no check fires,
    results equal the oracle."""
    out = run_child("""
        cases = 0
        n = 5000
        hot = gen.CSR(n, 10, np.arange(n + 1, dtype=np.int64), np.full(n, 7, np.int32))
        A = gen.random_csr(30, n, 0.3, seed=820)
        for sr in ("plus_times_f64", "min_plus_u32"):
            for fused in (True, False):
                Av = A.with_values(gen.random_values(sr, A.nnz, 821))
                Bv = hot.with_values(gen.random_values(sr, hot.nnz, 822))
                C = cb.spgemm(sr, cb.DeviceCSR.from_host(Av, sr), cb.DeviceCSR.from_host(Bv, sr),
                              fused=fused, check=True)
                compare_rows(sr, C.to_host(), oracle.spgemm(sr, Av, Bv))
                cases += 1
        # a dense row of A against a random B; ncols = 1; nrows = 0; an empty matrix
        shapes = [(gen.random_csr(40, 3000, 0.01, seed=823, full_rows=0.05), gen.random_csr(3000, 2000, 0.01, seed=824)),
                  (gen.random_csr(300, 200, 0.05, seed=825), gen.random_csr(200, 1, 0.5, seed=826)),
                  (gen.random_csr(0, 50, 0.1, seed=827), gen.random_csr(50, 60, 0.1, seed=828)),
                  (gen.random_csr(20, 30, 0.0, seed=829), gen.random_csr(30, 40, 0.2, seed=830))]
        for P, Q in shapes:
            for sr in ("plus_times_i64", "or_and_bool"):
                Av = P.with_values(gen.random_values(sr, P.nnz, 833))
                Bv = Q.with_values(gen.random_values(sr, Q.nnz, 834))
                C = cb.spgemm(sr, cb.DeviceCSR.from_host(Av, sr), cb.DeviceCSR.from_host(Bv, sr),
                              check=True)
                compare_rows(sr, C.to_host(), oracle.spgemm(sr, Av, Bv))
                cases += 1
        # rows in every tier over three bitmap spans (600000 columns)
        from test_gpu_parity import _tiered_inputs
        for sr in ("plus_times_i64", "or_and_bool"):
            Av, Bv = _tiered_inputs(sr, seed=835, ncols=600000)
            C = cb.spgemm(sr, cb.DeviceCSR.from_host(Av, sr), cb.DeviceCSR.from_host(Bv, sr), check=True)
            compare_rows(sr, C.to_host(), oracle.spgemm(sr, Av, Bv))
            cases += 1
        out["cases"] = cases
    """)
    assert out["cases"] == 14


def test_debug_library_is_silent_on_valid_products(cb):
    out = run_child("""
        checked = []
        # hash tiers and rank windows (R-MAT), every semiring
        for sr in gen.SEMIRINGS:
            P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=800)
            A = P.with_values(gen.random_values(sr, P.nnz, 801))
            dA = cb.DeviceCSR.from_host(A, sr)
            for fused in (True, False):
                C = cb.spgemm(sr, dA, dA, fused=fused, check=True)
                compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A))
            checked.append(sr)
        # small rows: the one-launch kernel and the work-queue kernel
        for sr, deg in (("min_plus_u32", 8), ("plus_times_f64", 40)):
            A = gen.er_exact(4000, 4000, deg, 802)
            A = A.with_values(gen.random_values(sr, A.nnz, 803))
            dA = cb.DeviceCSR.from_host(A, sr)
            C = cb.spgemm(sr, dA, dA)
            compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A))
            checked.append(sr + f"_er{deg}")
        # learned sizing (staging copy) and column batches
        from paper_2106_14402_gb300 import sizer
        model, _ = sizer.load()
        sr = "plus_times_f64"
        P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=804)
        A = P.with_values(gen.random_values(sr, P.nnz, 805))
        dA = cb.DeviceCSR.from_host(A, sr)
        want = oracle.spgemm(sr, A, A)
        C = cb.spgemm(sr, dA, dA, sizing="learned", mlp=model)
        compare_rows(sr, C.to_host(), want)
        n = []
        cb.spgemm_column_batches(sr, dA, dA, 8 * (A.nrows + 1) + int(want[0][-1]) * 12 // 3,
                                 lambda b, lo, hi, Cb: n.append(Cb.nnz))
        assert sum(n) == int(want[0][-1]) and len(n) >= 3
        checked.append("learned+batches")
        out["checked"] = checked
    """)
    assert len(out["checked"]) == len(gen.SEMIRINGS) + 3


@pytest.mark.parametrize("which", ["heavy", "hash"])
def test_short_row_is_reported_by_the_debug_library(cb, which):
    sr = "plus_times_f64"
    P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=810)
    A = P.with_values(gen.random_values(sr, P.nnz, 811))
    want = oracle.spgemm(sr, A, A)
    sizes = np.diff(want[0])
    # the largest row (rank windows) or a row of a hash tier (4 < nnz <= 512)
    row = int(np.argmax(sizes)) if which == "heavy" else int(np.flatnonzero((sizes > 4) & (sizes <= 512))[0])
    assert (sizes[row] > 512) == (which == "heavy")
    out = run_child(f"""
        sr = "{sr}"
        P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=810)
        A = P.with_values(gen.random_values(sr, P.nnz, 811))
        dA = cb.DeviceCSR.from_host(A, sr)
        ctx = cb.Context()
        ctx.set_fault(cb.FAULT_SHORT_ROW, {row})
        try:
            cb.spgemm(sr, dA, dA, ctx=ctx, fused=False)
            out["error"] = None
        except cb.CBError as e:
            out["error"] = e.code
            out["message"] = ctx.error()
        ctx.set_fault(cb.FAULT_SHORT_ROW, -1)      # the context stays usable
        C = cb.spgemm(sr, dA, dA, ctx=ctx, fused=False)
        compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A))
        out["after"] = "ok"
    """)
    assert out["error"] == 8 and "bounds check" in out["message"], out
    code = int(out["message"].split("bounds check ")[1].split()[0])
    assert code in ((37, 38, 39) if which == "heavy" else (34, 35)), out["message"]
    assert out["after"] == "ok"

    # the normal library: every write stays in C; the surplus entry is dropped,
    # and CB_FLAG_CHECK reports the hash tier's count mismatch
    dA = cb.DeviceCSR.from_host(A, sr)
    ctx = cb.Context()
    ctx.set_fault(cb.FAULT_SHORT_ROW, row)
    if which == "hash":
        with pytest.raises(cb.CBError) as e:
            cb.spgemm(sr, dA, dA, ctx=ctx, fused=False, check=True)
        assert e.value.code == 8 and "consistency" in ctx.error()
    rp, col, val = cb.spgemm(sr, dA, dA, ctx=ctx, fused=False).to_host()
    assert rp[-1] == want[0][-1] - 1 and rp[row + 1] - rp[row] == sizes[row] - 1
    rows = np.flatnonzero(np.arange(A.nrows) != row)     # every other row is intact
    compare_rows(sr, (rp, col, val), oracle.spgemm(sr, A, A, rows=rows), rows=rows)
