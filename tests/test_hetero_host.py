"""Host-side pieces of the heterogeneous semiring that need no GPU: the ABI's
semiring ids and record layout agree across the header, the binding, the
generators and the oracle; the binding's record split; the value streams."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2106_14402_gb300 import gen

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_enum():
    text = open(os.path.join(ROOT, "include", "cb.h")).read()
    body = text[text.index("typedef enum {"):text.index("} cb_semiring;")]
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"(CB_[A-Z0-9_]+)\s*=\s*(\d+)", body)}


def test_semiring_ids_agree():
    from paper_2106_14402_gb300 import cb
    ids = header_enum()
    assert ids["CB_MAXW_LABEL"] == cb.SEMIRING["maxw_label"][0] == oracle._CODES["maxw_label"][0] == 6
    names = {"CB_PLUS_TIMES_I64": "plus_times_i64", "CB_PLUS_TIMES_F64": "plus_times_f64",
             "CB_MIN_PLUS_U32": "min_plus_u32", "CB_OR_AND_BOOL": "or_and_bool",
             "CB_SEL2ND_MIN_I32": "sel2nd_min_i32"}
    for c, name in names.items():
        assert ids[c] == cb.SEMIRING[name][0] == oracle._CODES[name][0]


def test_record_layout_agrees():
    from paper_2106_14402_gb300 import cb
    text = open(os.path.join(ROOT, "include", "cb.h")).read()
    rec = text[text.index("typedef struct {\n  float w;"):text.index("} cb_wlabel;")]
    assert re.search(r"float w;\s*int32_t label;", rec)
    assert oracle.WLABEL == gen.WLABEL
    assert oracle.WLABEL.itemsize == 8 and oracle.WLABEL.fields["w"][1] == 0
    assert oracle.WLABEL.fields["label"][1] == 4
    a, b, c = cb.OPERAND_DTYPES["maxw_label"]
    assert (a, b, c) == (torch.float32, torch.int32, torch.int64)
    assert gen.HETERO_DTYPES["maxw_label"][:2] == (np.float32, np.int32)


def test_wlabel_split_reads_records():
    from paper_2106_14402_gb300 import cb
    rec = np.zeros(5, oracle.WLABEL)
    rec["w"] = np.array([0.5, -0.0, np.inf, 1e-45, -3.25], np.float32)
    rec["label"] = np.array([7, -1, 2 ** 31 - 1, -2 ** 31, 0], np.int32)
    val = torch.from_numpy(rec.view(np.int64).copy())
    w, lab = cb.wlabel_split(val)
    assert np.array_equal(w.numpy().view(np.uint32), rec["w"].view(np.uint32))
    assert np.array_equal(lab.numpy(), rec["label"])


def test_hetero_values_streams():
    w = gen.hetero_values("maxw_label", "A", 10000, seed=5)
    assert w.dtype == np.float32 and w.min() >= 0 and w.max() < 1
    assert np.array_equal(w, gen.hetero_values("maxw_label", "A", 10000, seed=5))
    lv = gen.hetero_values("maxw_label", "A", 10000, seed=5, levels=4)
    assert set(np.unique(lv).tolist()) <= {0.0, 0.25, 0.5, 0.75}
    lab = gen.hetero_values("maxw_label", "B", 10000, seed=5)
    assert lab.dtype == np.int32 and lab.min() >= 0 and lab.max() < 2 ** 30
    with pytest.raises(ValueError):
        gen.hetero_values("plus_times_f64", "A", 3, seed=1)
