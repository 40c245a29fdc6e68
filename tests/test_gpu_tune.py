"""Tier bounds chosen at run time: every setting must give the oracle's
result (they only move rows between hash tables and bitmap/rank windows),
and the autotuner must leave a valid, timed setting in the context."""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import compare_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


@pytest.fixture(scope="module")
def problem():
    P = gen.rmat(14, 16, *gen.RMAT_ABCD, seed=700)
    return P


def test_set_tune_clamps(cb):
    ctx = cb.Context()
    t = ctx.set_tune(100, 50, 99999)
    assert t["sym_hash_max"] == 512 and t["num_hash_max"] == 512 and t["learn_max"] == 8192
    t = ctx.set_tune(9000, 9000, 64)
    assert t["sym_hash_max"] == 4096 and t["num_hash_max"] == 4096
    assert ctx.get_tune() == t


@pytest.mark.parametrize("sr", ("plus_times_f64", "min_plus_u32", "or_and_bool"))
@pytest.mark.parametrize("bounds", [(512, 512), (512, 4096), (4096, 4096), (2048, 2048), (1024, 4096)])
def test_every_bound_setting_matches_oracle(cb, problem, sr, bounds):
    A = problem.with_values(gen.random_values(sr, problem.nnz, 701))
    ctx = cb.Context()
    ctx.set_tune(bounds[0], bounds[1], 512)
    dA = cb.DeviceCSR.from_host(A, sr)
    C = cb.spgemm(sr, dA, dA, ctx=ctx, check=True)
    torch.cuda.synchronize()
    flops, _ = oracle.row_stats(A, A)
    rows = np.unique(np.concatenate([np.arange(0, A.nrows, 37), np.argsort(-flops)[:60]]))
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A, rows=rows), rows=rows)


def test_autotune_keeps_a_valid_setting(cb, problem):
    sr = "plus_times_f64"
    A = problem.with_values(gen.random_values(sr, problem.nnz, 702))
    ctx = cb.Context()
    dA = cb.DeviceCSR.from_host(A, sr)
    best, ms = cb.autotune(sr, dA, dA, ctx=ctx)
    assert ms > 0
    assert ctx.get_tune() == best
    assert 512 <= best["sym_hash_max"] <= best["num_hash_max"] <= 4096
    C = cb.spgemm(sr, dA, dA, ctx=ctx)
    rows = np.arange(0, A.nrows, 53)
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A, rows=rows), rows=rows)
