"""Error paths of the C ABI that need no GPU: status strings, option
defaults, the one-launch kernel's column bound, and calls with a null
context or (on a machine without a GPU) a context that cannot be created
return status codes instead of aborting."""
import ctypes

import pytest

from paper_2106_14402_gb300 import build, cb

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    lib = ctypes.CDLL(build.build())
    lib.cb_status_str.restype = ctypes.c_char_p
    lib.cb_fused_max_cols.restype = ctypes.c_int64
    return lib


def test_status_strings(lib):
    for code, name in cb.STATUS.items():
        s = lib.cb_status_str(code)
        assert s and s != b"unknown status", (code, name)
    assert lib.cb_status_str(99) == b"unknown status"


def test_option_defaults(lib):
    o = cb.cb_opts()
    lib.cb_opts_default(ctypes.byref(o))
    assert (o.sizing, o.validate, o.out_capacity, o.budget_bytes, o.flags) == (0, 1, 0, 0, 0)
    assert (o.resume_col, o.resume_batch, o.digests) == (0, 0, None)
    assert abs(o.margin - 0.25) < 1e-7


def test_binding_structs_match_the_library_layout(lib):
    lib.cb_struct_size.restype = ctypes.c_int64
    want = [cb.cb_csr, cb.cb_opts, cb.cb_tune, cb.cb_stats, cb.cb_spvec]
    for which, struct in enumerate(want):
        assert lib.cb_struct_size(which) == ctypes.sizeof(struct), struct.__name__
    assert lib.cb_struct_size(5) == 8          # cb_wlabel {float, int32}
    assert lib.cb_struct_size(6) == -1


def test_fused_column_bound(lib):
    # keys are (col << log2(8 G)) | t in 32 bits
    assert lib.cb_fused_max_cols(8) == (1 << 26) - 1
    assert lib.cb_fused_max_cols(16) == (1 << 25) - 1
    assert lib.cb_fused_max_cols(32) == (1 << 24) - 1
    assert lib.cb_fused_max_cols(7) == 0


def test_null_context_is_an_argument_error(lib):
    assert lib.cb_spgemm_ex(None, 1, None, None, None, None) == 1
    assert lib.cb_merge(None, 1, 1, None, None, None) == 1
    assert lib.cb_spmspv(None, 1, None, None, None, None) == 1
    assert lib.cb_spgemm_batched(None, 0, None, None, None, None) == 1
    t = cb.cb_tune()
    assert lib.cb_ctx_set_tune(None, ctypes.byref(t)) == 1
    assert lib.cb_ctx_get_tune(None, ctypes.byref(t)) == 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="a GPU is present")
def test_context_without_a_gpu_is_a_cuda_error(lib):
    h = ctypes.c_void_p()
    assert lib.cb_ctx_create(ctypes.byref(h), None) == 8
    assert not h.value
