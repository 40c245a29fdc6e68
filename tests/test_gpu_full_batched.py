"""The batched workload at full size: 4096 independent products (ER,
n_i = floor(exp U(ln 256, ln 65536)), degree U{4..64}; products 0..2047
(min,+) u32, 2048..4095 (+,x) fp64), generated on the device, run through
cb_spgemm_batched under a 24 GiB output budget in every mode: host (exact),
sync-free, graph, and learned sizing.

Every wave is checked against the oracle:
  * element by element (host, sync-free and learned modes, in the wave's
    callback): a seeded 1% of the products completely, and in every wave the
    product with most products on a seeded 1% of its rows plus its first and
    last rows;
  * by digest (all modes, graph mode included, whose callback cannot read C):
    the library's per-product digest words (cb.h, cb_spgemm_batched) of the
    seeded 1% and of every wave's smallest product against the same digest
    of the oracle's output: bit-exact for (min,+) u32 and for the fp64
    pattern, and the fp64 weighted checksum within its bound;
  * and across modes: every product's first digest word (values included for
    u32, the pattern for fp64) is the same in all four modes.
"""
import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen
from parity import CHECKSUM_TOL, compare_rows, digest, digest_words

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COUNT = 4096
BUDGET = 24 << 30
MODES = [("host", "exact"), ("sync_free", "exact"), ("graph", "exact"), ("host", "learned")]


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


class Workload:
    def __init__(self, cb):
        from paper_2106_14402_gb300 import gen_device
        self.plan, self.As, self.Bs = gen_device.batched_workload(COUNT)
        self.srs = [p["semiring"] for p in self.plan]
        self.flops = np.array([p["n"] * p["deg"] * p["deg"] for p in self.plan], np.int64)
        rng = np.random.default_rng(20210628)
        self.random = set(int(i) for i in rng.choice(COUNT, COUNT // 100, replace=False))
        self._host = {}
        self._full = {}
        self._rows = {}
        self._dig = {}
        self.digests = {}   # mode -> host int64 array of 2 * COUNT words

    def host(self, i):
        if i not in self._host:
            self._host[i] = gen.batched_product_host(self.plan[i])
        return self._host[i]

    def full(self, i):
        """The oracle's whole product i."""
        if i not in self._full:
            A, B = self.host(i)
            self._full[i] = oracle.spgemm(self.plan[i]["semiring"], A, B)
        return self._full[i]

    def digest(self, i):
        """The oracle's digest words of product i, and the sum of its |a b| sums."""
        if i not in self._dig:
            rp, col, val, absum = self.full(i)
            d0, V = digest(self.plan[i]["semiring"], rp, col, val)
            self._dig[i] = (d0, V, float(absum.sum()))
        return self._dig[i]

    def sample_rows(self, i):
        n = self.plan[i]["n"]
        rng = np.random.default_rng(1000 + i)
        pick = rng.choice(n, size=max(1, n // 100), replace=False)
        return np.unique(np.concatenate([pick, [0, n - 1]])).astype(np.int64)

    def rows(self, i):
        """The oracle on product i's sampled rows."""
        if i not in self._rows:
            A, B = self.host(i)
            self._rows[i] = oracle.spgemm(self.plan[i]["semiring"], A, B, rows=self.sample_rows(i))
        return self._rows[i]


@pytest.fixture(scope="module")
def work(cb):
    w = Workload(cb)
    torch.cuda.synchronize()
    yield w
    del w.As, w.Bs
    torch.cuda.empty_cache()


def _host_vals(v):
    """A device value tensor on the host (uint32 through an int32 view)."""
    if v.dtype == torch.uint32:
        return v.view(torch.int32).cpu().numpy().view(np.uint32)
    return v.cpu().numpy()


def _vals(Cw):
    return Cw.val.view(torch.int32) if Cw.val.dtype == torch.uint32 else Cw.val


def _gather_rows(Cw, r0, rows):
    """Rows r0 + rows of a wave's device output, copied to the host as a CSR
    over those rows."""
    rp = Cw.row_ptr
    sel = torch.as_tensor(rows + r0, device=rp.device)
    starts, ends = rp[sel], rp[sel + 1]
    lens = ends - starts
    out_rp = torch.zeros(len(rows) + 1, dtype=torch.int64, device=rp.device)
    out_rp[1:] = torch.cumsum(lens, 0)
    total = int(out_rp[-1].item())
    rel = torch.arange(total, device=rp.device) - torch.repeat_interleave(out_rp[:-1], lens)
    idx = torch.repeat_interleave(starts, lens) + rel
    val = _vals(Cw)[idx]
    if Cw.val.dtype == torch.uint32:
        val = val.view(torch.uint32)
    return out_rp.cpu().numpy(), Cw.col[idx].cpu().numpy(), _host_vals(val)


def _product_rows(Cw, r0, n):
    """Product rows [r0, r0 + n) of a wave's device output on the host (its
    entries are contiguous)."""
    rp = Cw.row_ptr[r0:r0 + n + 1].cpu().numpy()
    a, b = int(rp[0]), int(rp[-1])
    return rp - a, Cw.col[a:b].cpu().numpy(), _host_vals(Cw.val[a:b])


def run_mode(cb, work, mode, sizing, model):
    plan = work.plan
    row_off = {}
    got_full, got_rows, waves = {}, {}, []

    def on_wave(w, first, end, *rest):
        if mode == "graph":
            nrows, nnz = rest
            waves.append((w, first, end, nnz))
            return None
        (Cw,) = rest
        waves.append((w, first, end, Cw.nnz))
        r0 = 0
        for i in range(first, end):
            row_off[i] = r0
            r0 += plan[i]["n"]
        assert r0 == Cw.nrows
        for i in range(first, end):
            if i in work.random:
                got_full[i] = _product_rows(Cw, row_off[i], plan[i]["n"])
        big = first + int(np.argmax(work.flops[first:end]))
        got_rows[big] = _gather_rows(Cw, row_off[big], work.sample_rows(big))
        return False

    dig = torch.zeros(2 * COUNT, dtype=torch.int64, device="cuda")
    st = cb.spgemm_batched(work.srs, work.As, work.Bs, on_wave, budget_bytes=BUDGET, validate=False,
                           sizing=sizing, mlp=model if sizing == "learned" else None, mode=mode,
                           digests=dig)
    torch.cuda.synchronize()
    return st, waves, got_full, got_rows, dig.cpu().numpy()


def check_digest(work, i, words):
    sr = work.plan[i]["semiring"]
    d0, V, abs_total = work.digest(i)
    g0, gv = digest_words(words, i)
    assert g0 == d0, f"product {i}: digest {g0:#x} != oracle {d0:#x}"
    if sr == "plus_times_f64":
        tol = CHECKSUM_TOL * abs_total
        assert abs(gv - V) <= tol, f"product {i}: checksum {gv!r} vs oracle {V!r} (tol {tol:.3g})"


@pytest.mark.parametrize("mode,sizing", MODES, ids=[f"{m}-{s}" for m, s in MODES])
def test_full_batched_workload_every_wave(cb, work, mode, sizing):
    model = None
    if sizing == "learned":
        from paper_2106_14402_gb300 import sizer
        model, _ = sizer.load()
    st, waves, got_full, got_rows, words = run_mode(cb, work, mode, sizing, model)
    # the waves cover every product once, in order, each within the budget
    assert [w[0] for w in waves] == list(range(len(waves))) and len(waves) == st["batches"]
    assert waves[0][1] == 0 and waves[-1][2] == COUNT
    assert all(a[2] == b[1] for a, b in zip(waves, waves[1:]))
    assert len(waves) >= 20, len(waves)
    assert st["nnz"] == sum(w[3] for w in waves)
    assert st["flops"] == int(work.flops.sum())
    for w, first, end, nnz in waves:
        assert end > first
        rows = sum(work.plan[i]["n"] for i in range(first, end))
        per = 4 + (4 if work.plan[first]["semiring"] == "min_plus_u32" else 8)
        assert 8 * (rows + 1) + nnz * per <= BUDGET
        # one product of every wave against the oracle by digest: its smallest
        small = first + int(np.argmin(work.flops[first:end]))
        check_digest(work, small, words)
    for i in sorted(work.random):
        check_digest(work, i, words)
    if mode != "graph":
        # element by element: the seeded 1% completely, and every wave's
        # largest product on its sampled rows
        assert set(got_full) == work.random
        for i in sorted(got_full):
            compare_rows(work.plan[i]["semiring"], got_full[i], work.full(i))
        assert len(got_rows) == len(waves)
        for i in sorted(got_rows):
            compare_rows(work.plan[i]["semiring"], got_rows[i], work.rows(i))
    work.digests[mode + "-" + sizing] = words


def test_digests_agree_across_modes(work):
    """Every product's first digest word (u32: pattern and values; fp64:
    pattern) is the same in all four modes."""
    if len(work.digests) < len(MODES):
        pytest.skip("needs every mode's run")
    base = None
    for key, words in work.digests.items():
        d0 = words[0::2]
        if base is None:
            base = d0
        else:
            bad = np.nonzero(d0 != base)[0]
            assert bad.size == 0, f"{key}: products {bad[:8]} differ"
