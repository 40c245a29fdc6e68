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
    assert 0.0 <= best["cf_esc"] <= 2.0 and best["cf_prereduce"] >= 1.0
    C = cb.spgemm(sr, dA, dA, ctx=ctx)
    rows = np.arange(0, A.nrows, 53)
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A, rows=rows), rows=rows)


# ---------------------------------------------------------------------------
# accumulator of hash-tier rows by compression ratio (expand-sort-compress,
# hash, hash with warp pre-reduction)
# ---------------------------------------------------------------------------

CF_SETTINGS = {"esc_all_low": (2.0, 1e30), "prereduce_all": (0.0, 1.0), "hash_only": (0.0, 1e30),
               "default": (1.25, 4.0)}


@pytest.mark.parametrize("setting", sorted(CF_SETTINGS))
@pytest.mark.parametrize("sr", gen.SEMIRINGS + gen.HETERO_SEMIRINGS)
def test_accumulator_by_compression_ratio(cb, sr, setting):
    """Every accumulator choice gives the oracle's result: R-MAT scale 12
    (hash-tier rows of low compression), a block-clustered matrix (high
    compression) and duplicate, unsorted inputs."""
    esc, pre = CF_SETTINGS[setting]
    ctx = cb.Context()
    t = ctx.set_tune(512, 4096, 512, esc, pre)
    assert abs(t["cf_esc"] - esc) < 1e-6 and (t["cf_prereduce"] == pre or pre >= 1e30)
    inputs = [gen.rmat(12, 16, *gen.RMAT_ABCD, seed=710), gen.block_clustered(1 << 11, 256, 0.5, 1.0, seed=711)]
    dup = gen.random_csr(500, 400, 0.02, seed=712, duplicates=True, shuffle=True, empty_rows=0.1)
    for k, P in enumerate(inputs + [dup]):
        B = P if k < 2 else gen.random_csr(400, 300, 0.03, seed=713, duplicates=True, shuffle=True)
        if sr in gen.HETERO_SEMIRINGS:
            A = P.with_values(gen.hetero_values(sr, "A", P.nnz, 714 + k, levels=4))
            Bv = B.with_values(gen.hetero_values(sr, "B", B.nnz, 715 + k))
        else:
            A = P.with_values(gen.random_values(sr, P.nnz, 714 + k))
            Bv = B.with_values(gen.random_values(sr, B.nnz, 715 + k))
        dA = cb.DeviceCSR.from_host(A, sr, operand="A")
        dB = cb.DeviceCSR.from_host(Bv, sr, operand="B")
        C = cb.spgemm(sr, dA, dB, ctx=ctx, check=True, fused=False)
        compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, Bv))


def test_set_tune_clamps_compression_bounds(cb):
    ctx = cb.Context()
    t = ctx.set_tune(512, 512, 512, 5.0, 0.5)
    assert t["cf_esc"] == 2.0 and t["cf_prereduce"] == 1.0
    t = ctx.set_tune(512, 512, 512, -1.0, float("nan"))
    assert t["cf_esc"] == 0.0 and t["cf_prereduce"] >= 1e30


def test_autotune_cache_hit_skips_the_grid(cb, problem, tmp_path):
    """The first cached autotune times the grid and stores the result under
    this device's key; a second call (fresh context) finds it, sets the same
    bounds and reports a hit; a foreign file is an argument error."""
    sr = "min_plus_u32"
    A = problem.with_values(gen.random_values(sr, problem.nnz, 720))
    dA = cb.DeviceCSR.from_host(A, sr)
    path = str(tmp_path / "tune.json")
    ctx1 = cb.Context()
    best, ms, hit = cb.autotune_cached(sr, dA, dA, path, ctx=ctx1)
    assert not hit and ms > 0 and ctx1.get_tune() == best
    key = cb.tune_key(torch.cuda.get_device_name(), sr, A.nrows, A.nnz, A.nnz)
    cached, cms = cb.tune_cache_get(path, key)
    assert cached == best and cms == ms
    ctx2 = cb.Context()
    best2, ms2, hit2 = cb.autotune_cached(sr, dA, dA, path, ctx=ctx2)
    assert hit2 and best2 == best and ms2 == ms and ctx2.get_tune() == best
    C = cb.spgemm(sr, dA, dA, ctx=ctx2)
    rows = np.arange(0, A.nrows, 61)
    compare_rows(sr, C.to_host(), oracle.spgemm(sr, A, A, rows=rows), rows=rows)
    bad = tmp_path / "bad.json"
    bad.write_text("not json")
    with pytest.raises(cb.CBError) as e:
        cb.autotune_cached(sr, dA, dA, str(bad), ctx=ctx2)
    assert e.value.code == 1 and "tune cache" in ctx2.error()
    assert bad.read_text() == "not json"
