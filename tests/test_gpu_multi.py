"""Batched SpGEMM of many independent products (stacked block-diagonal
launch, cut into waves by an output budget) and the device-side generator
of the batched workload."""
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


def small_plan(count=24):
    plan = []
    for p in gen.batched_plan(count, cfg=40):
        p = dict(p)
        p["n"] = 256 + (p["n"] % 1800)      # keep the host-side regeneration quick
        plan.append(p)
    return plan


def test_device_generator_matches_host_definition(cb):
    from paper_2106_14402_gb300 import gen_device
    for p in small_plan(4):
        dA = gen_device.er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"])
        A, _ = gen.batched_product_host(p)
        rp, col, val = dA.to_host()
        assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col)
        assert np.array_equal(val, A.val)


def run(cb, plan, budget, sizing="exact", mlp=None, mode="host"):
    from paper_2106_14402_gb300 import gen_device
    As, Bs, host = [], [], []
    for p in plan:
        As.append(gen_device.er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"]))
        Bs.append(gen_device.er(p["seed_b"], p["n"], p["deg"], p["semiring"], p["seed_vb"]))
    got = {}

    def on_wave(w, first, end, Cw):
        rp, col, val = Cw.to_host()
        r0 = 0
        for i in range(first, end):
            n = plan[i]["n"]
            sub = rp[r0:r0 + n + 1] - rp[r0]
            got[i] = (sub, col[rp[r0]:rp[r0 + n]], val[rp[r0]:rp[r0 + n]])
            r0 += n
        assert r0 == Cw.nrows

    st = cb.spgemm_batched([p["semiring"] for p in plan], As, Bs, on_wave, budget_bytes=budget,
                           sizing=sizing, mlp=mlp, mode=mode)
    return got, st


def reference(plan):
    out = []
    for p in plan:
        A, B = gen.batched_product_host(p)
        out.append(oracle.spgemm(p["semiring"], A, B))
    return out


def out_bytes(p, want):
    vsz = 4 if p["semiring"] == "min_plus_u32" else 8
    return 8 * (p["n"] + 1) + int(want[0][-1]) * (4 + vsz)


@pytest.mark.parametrize("waves", [False, True])
def test_batched_products_match_oracle(cb, waves):
    plan = small_plan()
    want = reference(plan)
    budget = int(1.3 * max(out_bytes(p, w) for p, w in zip(plan, want))) if waves else 0
    got, st = run(cb, plan, budget)
    assert len(got) == len(plan)
    if waves:
        assert st["batches"] > 3
    for i, p in enumerate(plan):
        compare_rows(p["semiring"], got[i], want[i])


def test_batched_with_learned_sizing(cb):
    from paper_2106_14402_gb300 import sizer
    model, _ = sizer.load()
    plan = small_plan(12)
    want = reference(plan)
    budget = int(1.6 * max(out_bytes(p, w) for p, w in zip(plan, want)))
    got, st = run(cb, plan, budget, sizing="learned", mlp=model)
    assert st["batches"] > 2
    for i, p in enumerate(plan):
        compare_rows(p["semiring"], got[i], want[i])


def test_batched_stops_early_and_rejects_tiny_budget(cb):
    plan = small_plan(8)
    from paper_2106_14402_gb300 import gen_device
    As = [gen_device.er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"]) for p in plan]
    Bs = [gen_device.er(p["seed_b"], p["n"], p["deg"], p["semiring"], p["seed_vb"]) for p in plan]
    seen = []
    big = max(out_bytes(p, w) for p, w in zip(plan, reference(plan)))
    st = cb.spgemm_batched([p["semiring"] for p in plan], As, Bs,
                           lambda w, f, e, C: seen.append(w) or True, budget_bytes=int(1.2 * big))
    assert seen == [0] and st["batches"] == 1
    with pytest.raises(cb.CBError) as e:
        cb.spgemm_batched([p["semiring"] for p in plan], As, Bs, lambda *a: False, budget_bytes=4096)
    assert e.value.code == 6


def bound_bytes(p):
    A, B = gen.batched_product_host(p)
    vsz = 4 if p["semiring"] == "min_plus_u32" else 8
    return 8 * (p["n"] + 1) + int(oracle.row_stats(A, B)[0].sum()) * (4 + vsz)


def flop_waves(plan, budget):
    """Waves when each run of same-semiring products is packed by its flop
    bound: a wave holds one row-pointer array and the flops of its products."""
    waves, rows, flops, sr = 0, 0, 0, None
    for p in plan:
        A, B = gen.batched_product_host(p)
        f = int(oracle.row_stats(A, B)[0].sum())
        per = 4 + (4 if p["semiring"] == "min_plus_u32" else 8)
        if p["semiring"] != sr or 8 * (rows + p["n"] + 1) + (flops + f) * per > budget:
            waves, rows, flops, sr = waves + 1, p["n"], f, p["semiring"]
        else:
            rows, flops = rows + p["n"], flops + f
    return waves


@pytest.mark.parametrize("waves", [False, True])
def test_sync_free_waves_match_oracle(cb, waves):
    """The launch sequence without host synchronisation (tier sizes on the
    device, C sized by the wave's flop bound) gives the exact products."""
    plan = small_plan()
    want = reference(plan)
    budget = int(1.3 * max(bound_bytes(p) for p in plan)) if waves else 0
    got, st = run(cb, plan, budget, mode="sync_free")
    assert len(got) == len(plan)
    if waves:
        assert st["batches"] == flop_waves(plan, budget) > 3   # cut by the flop bound
    for i, p in enumerate(plan):
        compare_rows(p["semiring"], got[i], want[i])


def test_graph_waves(cb):
    """All waves captured into one CUDA graph: the same waves, and every
    wave's nnz equal to the oracle's, as the sync-free run reports them."""
    from paper_2106_14402_gb300 import gen_device
    plan = small_plan()
    want = reference(plan)
    budget = int(1.3 * max(bound_bytes(p) for p in plan))
    As = [gen_device.er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"]) for p in plan]
    Bs = [gen_device.er(p["seed_b"], p["n"], p["deg"], p["semiring"], p["seed_vb"]) for p in plan]
    srs = [p["semiring"] for p in plan]
    waves = []
    st = cb.spgemm_batched(srs, As, Bs, lambda w, f, e, nr, nz: waves.append((w, f, e, nr, nz)),
                           budget_bytes=budget, mode="graph")
    free = []
    cb.spgemm_batched(srs, As, Bs, lambda w, f, e, C: free.append((w, f, e, C.nrows, C.nnz)),
                      budget_bytes=budget, mode="sync_free")
    assert waves == free and st["batches"] == len(waves) == flop_waves(plan, budget) > 3
    for w, f, e, nr, nz in waves:
        assert nr == sum(plan[i]["n"] for i in range(f, e))
        assert nz == sum(int(want[i][0][-1]) for i in range(f, e))
    assert st["nnz"] == sum(int(x[0][-1]) for x in want)


@pytest.mark.parametrize("sr", ("min_plus_u32", "plus_times_f64"))
def test_sync_free_heavy_rows(cb, sr):
    """Products with heavy rows (bitmap symbolic, rank-window numeric) in the
    launch sequence without host synchronisation: sortedness, heavy-row and
    window counts read on the device; exact results."""
    P = gen.rmat(13, 16, *gen.RMAT_ABCD, seed=300)
    A = P.with_values(gen.random_values(sr, P.nnz, 301))
    B = P.with_values(gen.random_values(sr, P.nnz, 302))
    flops, _ = oracle.row_stats(A, B)
    assert flops.max() > 4096
    dA, dB = cb.DeviceCSR.from_host(A, sr), cb.DeviceCSR.from_host(B, sr)
    got = []
    st = cb.spgemm_batched([sr, sr], [dA, dA], [dB, dB], lambda w, f, e, C: got.append(C.to_host()),
                           mode="sync_free")
    want = oracle.spgemm(sr, A, B)
    assert len(got) == 1 and st["nnz"] == 2 * int(want[0][-1])
    rp, col, val = got[0]
    m, n = A.nrows, int(want[0][-1])
    for k in range(2):
        sub = (rp[k * m:(k + 1) * m + 1] - rp[k * m], col[rp[k * m]:rp[k * m] + n], val[rp[k * m]:rp[k * m] + n])
        compare_rows(sr, sub, want)
    seen = []
    st = cb.spgemm_batched([sr, sr], [dA, dA], [dB, dB], lambda *a: seen.append(a), mode="graph")
    assert st["nnz"] == 2 * n and len(seen) == 1 and seen[0][4] == 2 * n
