"""Device-side generation of the batched workload (libcbgen.so).

Input generation only: the counter-based exact-degree ER definition is the
one in gen.py (er_counter, counter_values_*), so any generated product can be
regenerated on the host for the oracle.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build
from . import gen

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(_build.GENLIB):
            _build.build()
        lib = ctypes.CDLL(_build.GENLIB)
        P, I64 = ctypes.c_void_p, ctypes.c_int64
        lib.cbgen_er.argtypes = [ctypes.c_uint64, I64, I64, ctypes.c_int, P, P, P, P]
        lib.cbgen_values_u32.argtypes = [ctypes.c_uint64, I64, ctypes.c_uint32, ctypes.c_uint32, P, P]
        lib.cbgen_values_f64.argtypes = [ctypes.c_uint64, I64, ctypes.c_double, ctypes.c_double, P, P]
        for f in (lib.cbgen_er, lib.cbgen_values_u32, lib.cbgen_values_f64):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def er(seed: int, n: int, deg: int, semiring: str, vseed: int, device="cuda"):
    """One n x n exact-degree ER matrix with values, on the device."""
    from .cb import DeviceCSR
    lib = load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rp = torch.empty(n + 1, dtype=torch.int64, device=device)
    col = torch.empty(max(n * deg, 1), dtype=torch.int32, device=device)
    err = torch.zeros(1, dtype=torch.int32, device=device)
    rc = lib.cbgen_er(seed & ((1 << 64) - 1), n, n, deg, ctypes.c_void_p(rp.data_ptr()),
                      ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(err.data_ptr()), s)
    if rc:
        raise RuntimeError(f"cbgen_er failed ({rc})")
    nnz = n * deg
    if semiring == "min_plus_u32":
        val = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)
        rc = lib.cbgen_values_u32(vseed & ((1 << 64) - 1), nnz, 1, 1000, ctypes.c_void_p(val.data_ptr()), s)
        val = val.view(torch.uint32)
    else:
        val = torch.empty(max(nnz, 1), dtype=torch.float64, device=device)
        rc = lib.cbgen_values_f64(vseed & ((1 << 64) - 1), nnz, -1.0, 1.0, ctypes.c_void_p(val.data_ptr()), s)
    if rc:
        raise RuntimeError(f"cbgen_values failed ({rc})")
    return DeviceCSR(n, n, rp, col[:nnz], val[:nnz])


def batched_workload(count: int = 4096, device="cuda"):
    """The batched workload's products (A_i, B_i) generated on the device."""
    plan = gen.batched_plan(count)
    As, Bs = [], []
    for p in plan:
        As.append(er(p["seed_a"], p["n"], p["deg"], p["semiring"], p["seed_va"], device))
        Bs.append(er(p["seed_b"], p["n"], p["deg"], p["semiring"], p["seed_vb"], device))
    return plan, As, Bs
