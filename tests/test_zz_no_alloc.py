"""The allocation-free scan entry point, called through the C ABI.

cb_exclusive_scan_noalloc serves callers that cannot allocate device memory
(their GPU memory is owned by another allocator, or cudaMalloc's implicit
synchronisation is not acceptable where they call it).  Its scratch is a
fixed device array inside the library, shared by every call.  This test
checks it against the allocating entry point cb_exclusive_scan on two calls
in a row (the second one sees the first call's leftovers in the shared
scratch), against torch.cumsum up to the last tile of the array's capacity,
and that sizes beyond that capacity are rejected before anything is
launched.  It runs last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CB_OK = 0
CB_ERR_SCRATCH = 10
TILE = 4096
MAX_N = 65536 * TILE


def _noalloc(lib, x, n):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    got = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    rc = lib.cb_exclusive_scan_noalloc(ctypes.c_void_p(x.data_ptr()), n,
                                       ctypes.c_void_p(got.data_ptr()), stream)
    return rc, got


def _cumsum(x):
    want = torch.zeros(x.numel() + 1, dtype=torch.int64, device=x.device)
    torch.cumsum(x, 0, out=want[1:])
    return want


def test_noalloc_scan_matches_allocating_scan_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb
    lib = cb.load()
    gen = torch.Generator(device="cuda").manual_seed(1234)
    # 5,000,011 entries span 1,221 tiles, so the scan of tile sums carries
    # across two chunks of 1,024 tiles; 777,777 then reuses the scratch
    for n in (5_000_011, 777_777):
        x = torch.randint(0, 1 << 24, (n,), dtype=torch.int64, device="cuda", generator=gen)
        want = cb.exclusive_scan(x)                      # allocating entry point
        rc, got = _noalloc(lib, x, n)
        assert rc == CB_OK
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert torch.equal(got, _cumsum(x))


def test_noalloc_scan_last_tile_of_its_capacity():
    """n one below the 65,536-tile capacity (the last tile holds 4,095
    entries), then exactly the capacity: every scratch slot is used."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb
    lib = cb.load()
    gen = torch.Generator(device="cuda").manual_seed(99)
    x = torch.randint(0, 1 << 20, (MAX_N,), dtype=torch.int64, device="cuda", generator=gen)
    for n in (MAX_N - 1, MAX_N):
        xs = x[:n]
        rc, got = _noalloc(lib, xs, n)
        assert rc == CB_OK
        torch.cuda.synchronize()
        want = _cumsum(xs)
        assert torch.equal(got, want)
        del got, want
    torch.cuda.empty_cache()


def test_noalloc_scan_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb
    lib = cb.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.zeros(8, dtype=torch.int64, device="cuda")
    out = torch.zeros(9, dtype=torch.int64, device="cuda")
    # The size check happens on the host before any launch, so the small
    # buffers are never touched.
    rc = lib.cb_exclusive_scan_noalloc(ctypes.c_void_p(x.data_ptr()), MAX_N + 1,
                                       ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == CB_ERR_SCRATCH
    assert lib.cb_status_str(rc) == b"size beyond the static scratch capacity"
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
