"""Host-side arithmetic of bench.py (no GPU): the compulsory-bytes model of
the roofline, per operand value size, and the traffic figure it reads from
the committed ncu summary."""
import numpy as np

import bench
from paper_2106_14402_gb300 import gen


def _csr(rows, ncols):
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows]) if rows else np.zeros(0, np.int32)
    return gen.CSR(len(rows), ncols, rp, col)


def test_compulsory_bytes_counts_each_operand_once():
    # A: 3 rows, 4 entries; B: rows 0..3, rows 1 and 2 touched by A (lengths 2 and 3)
    A = _csr([[1], [1, 2], [2]], 4)
    B = _csr([[0], [0, 3], [1, 2, 3], []], 4)
    nnz_c = 5
    for sr, v in (("plus_times_f64", 8), ("min_plus_u32", 4), ("or_and_bool", 1)):
        a = 8 * 4 + 4 * (4 + v)
        b = 8 * (2 + 1) + 5 * (4 + v)
        c = 8 * 4 + nnz_c * (4 + v)
        assert bench.compulsory_bytes(sr, A, B, nnz_c, 3) == a + b + c
    # heterogeneous: A float32 weights, B int32 labels, C 8-byte records
    a = 8 * 4 + 4 * (4 + 4)
    b = 8 * 3 + 5 * (4 + 4)
    c = 8 * 4 + nnz_c * (4 + 8)
    assert bench.compulsory_bytes("maxw_label", A, B, nnz_c, 3) == a + b + c


def test_traffic_figure_holds_only_for_the_captured_kernel_sources(tmp_path, monkeypatch):
    """profiles/traffic.json's figure is used only while the numeric kernels'
    sources are the ones it was captured from."""
    import json
    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(path))
    assert bench.fp64_traffic_per_product() == (None, "no traffic capture")
    path.write_text(json.dumps({"fp64_numeric_bytes_per_product": 4.5, "capture": "s16",
                                "sources_digest": bench.sources_digest()}))
    assert bench.fp64_traffic_per_product() == (4.5, "s16")
    path.write_text(json.dumps({"fp64_numeric_bytes_per_product": 4.5, "capture": "s16",
                                "sources_digest": "0" * 16}))
    t, why = bench.fp64_traffic_per_product()
    assert t is None and "changed" in why
