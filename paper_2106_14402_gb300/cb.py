"""Python binding of libcb.so (include/cb.h): argument marshalling only.

Every step of the SpGEMM runs in the library's CUDA kernels; PyTorch only
provides device memory for the inputs and the current CUDA stream.  There is
no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

c_int64 = ctypes.c_int64
c_void_p = ctypes.c_void_p

# name -> (cb_semiring code, dtype of C's values)
SEMIRING = {
    "plus_times_i64": (1, torch.int64),
    "plus_times_f64": (2, torch.float64),
    "min_plus_u32": (3, torch.uint32),
    "or_and_bool": (4, torch.uint8),
    "sel2nd_min_i32": (5, torch.int32),
    # heterogeneous: A float32 weights, B int32 labels, C cb_wlabel records
    # {float w; int32 label} held as one int64 each (see wlabel_split)
    "maxw_label": (6, torch.int64),
}

# name -> dtypes of A's, B's and C's values
OPERAND_DTYPES = {name: (dt, dt, dt) for name, (_, dt) in SEMIRING.items()}
OPERAND_DTYPES["maxw_label"] = (torch.float32, torch.int32, torch.int64)


def wlabel_split(val: torch.Tensor):
    """(w float32, label int32) views of maxw_label values (int64 records)."""
    pairs = val.view(torch.int32).view(-1, 2)
    return pairs[:, 0].view(torch.float32), pairs[:, 1]

SIZING = {"exact": 0, "learned": 1, "upper_bound": 2}

STATUS = {0: "CB_OK", 1: "CB_ERR_ARG", 2: "CB_ERR_SHAPE", 3: "CB_ERR_SEMIRING", 4: "CB_ERR_INDEX",
          5: "CB_ERR_OOM", 6: "CB_ERR_BUDGET", 7: "CB_ERR_TIMEOUT", 8: "CB_ERR_CUDA",
          9: "CB_ERR_CAPACITY", 10: "CB_ERR_SCRATCH"}


class cb_csr(ctypes.Structure):
    _fields_ = [("nrows", c_int64), ("ncols", c_int64), ("nnz", c_int64),
                ("row_ptr", c_void_p), ("col", c_void_p), ("val", c_void_p)]


BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, c_int64, c_int64, ctypes.POINTER(cb_csr),
                            c_void_p)


class cb_opts(ctypes.Structure):
    _fields_ = [("sizing", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("out_capacity", c_int64), ("budget_bytes", c_int64),
                ("on_batch", BATCH_FN), ("user", c_void_p), ("mlp", c_void_p),
                ("margin", ctypes.c_float), ("flags", ctypes.c_int32),
                ("digests", c_void_p), ("resume_col", c_int64), ("resume_batch", ctypes.c_int32)]


class cb_tune(ctypes.Structure):
    _fields_ = [("sym_hash_max", ctypes.c_int32), ("num_hash_max", ctypes.c_int32),
                ("learn_max", ctypes.c_int32), ("cf_esc", ctypes.c_float),
                ("cf_prereduce", ctypes.c_float)]


class cb_stats(ctypes.Structure):
    _fields_ = [("flops", c_int64), ("nnz", c_int64), ("heavy_rows", c_int64),
                ("heavy_units", c_int64), ("overflow_rows", c_int64), ("batches", ctypes.c_int32),
                ("kernels", ctypes.c_int32), ("ms_stats", ctypes.c_float),
                ("ms_symbolic", ctypes.c_float), ("ms_scan", ctypes.c_float),
                ("ms_numeric", ctypes.c_float)]


class cb_spvec(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nnz", c_int64), ("idx", c_void_p), ("val", c_void_p)]


class CBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

# exported symbol -> (argtypes, restype)
_SIGS = {
    "cb_opts_default": ([ctypes.POINTER(cb_opts)], None),
    "cb_ctx_create": ([ctypes.POINTER(c_void_p), c_void_p], ctypes.c_int),
    "cb_ctx_destroy": ([c_void_p], None),
    "cb_ctx_set_stream": ([c_void_p, c_void_p], ctypes.c_int),
    "cb_last_error": ([c_void_p], ctypes.c_char_p),
    "cb_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "cb_spgemm": ([ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                   ctypes.POINTER(cb_csr)], ctypes.c_int),
    "cb_spgemm_ex": ([c_void_p, ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                      ctypes.POINTER(cb_csr), ctypes.POINTER(cb_opts)], ctypes.c_int),
    "cb_csr_free": ([ctypes.POINTER(cb_csr)], None),
    "cb_csr_free_async": ([c_void_p, ctypes.POINTER(cb_csr)], ctypes.c_int),
    "cb_row_stats": ([c_void_p, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr), c_void_p, c_void_p],
                     ctypes.c_int),
    "cb_row_nnz": ([c_void_p, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr), c_void_p], ctypes.c_int),
    "cb_exclusive_scan": ([c_void_p, c_void_p, c_int64, c_void_p], ctypes.c_int),
    "cb_exclusive_scan_noalloc": ([c_void_p, c_int64, c_void_p, c_void_p], ctypes.c_int),
    "cb_last_stats": ([c_void_p, ctypes.POINTER(cb_stats)], ctypes.c_int),
    "cb_ctx_set_fault": ([c_void_p, ctypes.c_int, c_int64, c_int64], ctypes.c_int),
    "cb_spgemm_batched": ([c_void_p, ctypes.c_int, c_void_p, c_void_p, c_void_p,
                           ctypes.POINTER(cb_opts)], ctypes.c_int),
    "cb_ctx_set_tune": ([c_void_p, ctypes.POINTER(cb_tune)], ctypes.c_int),
    "cb_ctx_get_tune": ([c_void_p, ctypes.POINTER(cb_tune)], ctypes.c_int),
    "cb_autotune": ([c_void_p, ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                     ctypes.POINTER(cb_opts), ctypes.POINTER(cb_tune), ctypes.POINTER(ctypes.c_float)],
                    ctypes.c_int),
    "cb_autotune_cached": ([c_void_p, ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                            ctypes.POINTER(cb_opts), ctypes.c_char_p, ctypes.POINTER(cb_tune),
                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cb_tune_key": ([ctypes.c_char_p, ctypes.c_int, ctypes.c_int32, c_int64, c_int64, c_int64,
                     ctypes.c_char_p, c_int64], ctypes.c_int),
    "cb_tune_cache_get": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(cb_tune),
                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cb_tune_cache_put": ([ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(cb_tune), ctypes.c_float],
                          ctypes.c_int),
    "cb_struct_size": ([ctypes.c_int], c_int64),
    "cb_spmspv": ([c_void_p, ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_spvec),
                   ctypes.POINTER(cb_spvec), ctypes.POINTER(cb_opts)], ctypes.c_int),
    "cb_spvec_free_async": ([c_void_p, ctypes.POINTER(cb_spvec)], ctypes.c_int),
    "cb_merge": ([c_void_p, ctypes.c_int, ctypes.c_int, c_void_p, ctypes.POINTER(cb_csr),
                  ctypes.POINTER(cb_opts)], ctypes.c_int),
    "cb_spgemm_fused": ([c_void_p, ctypes.c_int, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                         ctypes.POINTER(cb_csr), c_int64, ctypes.c_int, c_void_p], ctypes.c_int),
    "cb_fused_max_cols": ([ctypes.c_int], c_int64),
    "cb_fused_lanes": ([c_void_p, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr),
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(c_int64)], ctypes.c_int),
    "cb_mlp_create": ([ctypes.POINTER(c_void_p), c_void_p, c_void_p], ctypes.c_int),
    "cb_mlp_destroy": ([c_void_p], None),
    "cb_mlp_get": ([c_void_p, c_void_p, c_void_p, c_void_p], ctypes.c_int),
    "cb_row_features": ([c_void_p, ctypes.POINTER(cb_csr), ctypes.POINTER(cb_csr), c_void_p],
                        ctypes.c_int),
    "cb_mlp_predict": ([c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p],
                       ctypes.c_int),
    "cb_mlp_grad": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int64, ctypes.c_float, c_void_p,
                     c_void_p], ctypes.c_int),
    "cb_mlp_train": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int64, ctypes.c_int, c_int64,
                      ctypes.c_float, ctypes.c_float, c_void_p], ctypes.c_int),
}


def library_path() -> str:
    """libcb.so, or the bounds-checking debug build libcb_check.so when the
    environment variable CB_LIBRARY is "check" (debugging and tests only)."""
    return _build.LIB_CHECK if os.environ.get("CB_LIBRARY", "") == "check" else _build.LIB


def load(build_if_missing: bool = True):
    """Load the library (building it first if allowed); raises if it is unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"{os.path.basename(path)} not built at {path}")
                _build.build(check=path == _build.LIB_CHECK)
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return tuple(_SIGS)


# ---------------------------------------------------------------------------
# device matrices
# ---------------------------------------------------------------------------

@dataclass
class DeviceCSR:
    nrows: int
    ncols: int
    row_ptr: torch.Tensor   # int64 [nrows + 1]
    col: torch.Tensor       # int32 [nnz]
    val: torch.Tensor       # typed [nnz]
    _owner: object = None   # keeps library-allocated memory alive

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @staticmethod
    def from_host(M, semiring: str, device="cuda", operand: str = "A") -> "DeviceCSR":
        """Copy a host CSR to the device with the value dtype of `operand`
        ("A", "B" or "C") under the semiring."""
        dt = OPERAND_DTYPES[semiring]["ABC".index(operand)]
        val = torch.from_numpy(np.ascontiguousarray(M.val).view(_np_view(dt)))
        return DeviceCSR(M.nrows, M.ncols,
                         torch.from_numpy(np.ascontiguousarray(M.row_ptr, dtype=np.int64)).to(device),
                         torch.from_numpy(np.ascontiguousarray(M.col, dtype=np.int32)).to(device),
                         val.to(device).view(dt))

    def to_host(self):
        v = self.val
        if v.dtype == torch.uint32:
            v = v.view(torch.int32)
        val = v.cpu().numpy()
        if self.val.dtype == torch.uint32:
            val = val.view(np.uint32)
        return self.row_ptr.cpu().numpy(), self.col.cpu().numpy(), val

    @staticmethod
    def from_scipy(M, semiring: str, device="cuda", operand: str = "A") -> "DeviceCSR":
        """Copy a scipy.sparse matrix (any format; converted to CSR, its
        entries kept as stored: duplicates and unsorted rows are allowed by
        the ABI) with the value dtype of `operand` under the semiring."""
        csr = M.tocsr()
        dt = OPERAND_DTYPES[semiring]["ABC".index(operand)]
        host = type("HostCSR", (), {})()
        host.nrows, host.ncols = csr.shape
        host.row_ptr = csr.indptr.astype(np.int64)
        host.col = csr.indices.astype(np.int32)
        host.val = np.ascontiguousarray(csr.data).astype(_np_dtype(dt))
        return DeviceCSR.from_host(host, semiring, device, operand)

    def to_scipy(self):
        """This matrix as a scipy.sparse.csr_matrix on the host (one-type
        semirings; cb_wlabel records have no scipy dtype)."""
        import scipy.sparse as sp
        rp, col, val = self.to_host()
        return sp.csr_matrix((val, col, rp), shape=(self.nrows, self.ncols))

    def as_struct(self) -> cb_csr:
        return cb_csr(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                      self.col.data_ptr() if self.nnz else None,
                      self.val.data_ptr() if self.nnz else None)


def _np_dtype(dt):
    return {torch.int64: np.int64, torch.float64: np.float64, torch.uint32: np.uint32,
            torch.uint8: np.uint8, torch.int32: np.int32, torch.float32: np.float32}[dt]


def _np_view(dt):
    return {torch.int64: np.int64, torch.float64: np.float64, torch.uint32: np.int32,
            torch.uint8: np.uint8, torch.int32: np.int32, torch.float32: np.float32}[dt]


_TYPESTR = {torch.int64: "<i8", torch.float64: "<f8", torch.uint32: "<u4", torch.uint8: "|u1",
            torch.int32: "<i4", torch.float32: "<f4"}


class _Owner:
    """Frees library-allocated C arrays when the last tensor viewing them dies,
    in stream order on the context's stream (after the kernels writing them)."""

    def __init__(self, ctx, csr: cb_csr):
        self.ctx = ctx
        self.csr = csr

    def __del__(self):
        try:
            self.ctx.lib.cb_csr_free_async(self.ctx.handle, ctypes.byref(self.csr))
        except Exception:
            pass


class _Buf:
    def __init__(self, ptr: int, n: int, dtype, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": _TYPESTR[dtype],
                                         "data": (ptr, False), "version": 3, "strides": None}
        self.owner = owner


def _wrap(ptr, n, dtype, owner, device):
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device=device)
    if dtype == torch.uint32:
        t = torch.as_tensor(_Buf(ptr, n, torch.int32, owner), device=device)
        return t.view(torch.uint32)
    return torch.as_tensor(_Buf(ptr, n, dtype, owner), device=device)


# ---------------------------------------------------------------------------
# contexts (one per device and stream)
# ---------------------------------------------------------------------------

class Context:
    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.lib = load()
        self.stream = stream or torch.cuda.current_stream()
        self.handle = c_void_p()
        rc = self.lib.cb_ctx_create(ctypes.byref(self.handle), c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise CBError(rc, "cb_ctx_create failed")

    def __del__(self):
        try:
            if self.handle:
                self.lib.cb_ctx_destroy(self.handle)
                self.handle = c_void_p()
        except Exception:
            pass

    def error(self) -> str:
        msg = self.lib.cb_last_error(self.handle)
        return msg.decode() if msg else ""

    def check(self, rc: int):
        if rc != 0:
            raise CBError(rc, self.error())

    def set_tune(self, sym_hash_max=512, num_hash_max=512, learn_max=512, cf_esc=1.25,
                 cf_prereduce=4.0) -> dict:
        t = cb_tune(sym_hash_max, num_hash_max, learn_max, cf_esc, cf_prereduce)
        self.check(self.lib.cb_ctx_set_tune(self.handle, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in cb_tune._fields_}

    def get_tune(self) -> dict:
        t = cb_tune()
        self.check(self.lib.cb_ctx_get_tune(self.handle, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in cb_tune._fields_}

    def set_fault(self, kind: int, arg: int, arg2: int = 0) -> None:
        """Fault injection (cb_ctx_set_fault): FAULT_ALLOC fails the arg-th device
        allocation; FAULT_SILENT_TILE keeps tile arg of the one-launch kernel
        from publishing, waits giving up after arg2 polls (arg < 0: defaults);
        FAULT_SHORT_ROW makes row arg's exact size one short after the
        symbolic phase (arg < 0: off)."""
        self.check(self.lib.cb_ctx_set_fault(self.handle, int(kind), int(arg), int(arg2)))

    def stats(self) -> dict:
        s = cb_stats()
        self.check(self.lib.cb_last_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in cb_stats._fields_}


_ctx_cache: dict = {}


def context(stream: torch.cuda.Stream | None = None) -> Context:
    stream = stream or torch.cuda.current_stream()
    key = (stream.device.index, stream.cuda_stream)
    ctx = _ctx_cache.get(key)
    if ctx is None:
        ctx = Context(stream)
        _ctx_cache[key] = ctx
    return ctx


def make_opts(sizing="exact", validate=True, out_capacity=0, budget_bytes=0, on_batch=None,
              margin=0.25, flags=0, mlp=None) -> cb_opts:
    lib = load()
    o = cb_opts()
    lib.cb_opts_default(ctypes.byref(o))
    o.sizing = SIZING[sizing]
    o.validate = 1 if validate else 0
    o.out_capacity = int(out_capacity)
    o.budget_bytes = int(budget_bytes)
    if on_batch is not None:
        o.on_batch = on_batch
    o.margin = float(margin)
    o.flags = int(flags)
    if mlp is not None:
        o.mlp = mlp.handle.value
    return o


# ---------------------------------------------------------------------------
# the calls
# ---------------------------------------------------------------------------

FLAG_CHECK = 1
FLAG_TIMING = 2
FLAG_LEARNED_ROWS = 4
FLAG_NO_FUSED = 8
FLAG_GRAPH = 16
FLAG_SYNC_FREE = 32
FLAG_SPMSPV_BUCKET = 64

# fault injection kinds (cb_ctx_set_fault)
FAULT_ALLOC = 1
FAULT_SILENT_TILE = 2
FAULT_SHORT_ROW = 3

# device status bits of cb_spgemm_fused
FUSED_CAPACITY = 1
FUSED_ROW_TOO_LARGE = 2
FUSED_STALLED = 4


def spgemm(semiring: str, A: DeviceCSR, B: DeviceCSR, *, validate: bool = True, check: bool = False,
           ctx: Context | None = None, out: DeviceCSR | None = None, sizing: str = "exact",
           timing: bool = False, mlp=None, margin: float = 0.25, fused: bool = True) -> DeviceCSR:
    """C = A (+).(x) B on the GPU (cb_spgemm_ex).

    With `out` (a DeviceCSR whose col/val tensors are large enough), C is
    written into those buffers and a DeviceCSR viewing the first nnz(C)
    entries is returned; otherwise the library allocates C.
    `check` adds a synchronising self-consistency check of the kernels.
    `fused=False` keeps products whose rows are all small on the two-phase
    path instead of the one-launch kernel.
    """
    code, dt = SEMIRING[semiring]
    ctx = ctx or context()
    sa, sb = A.as_struct(), B.as_struct()
    opts = make_opts(sizing=sizing, validate=validate, mlp=mlp, margin=margin,
                     flags=(FLAG_CHECK if check else 0) | (FLAG_TIMING if timing else 0) |
                     (0 if fused else FLAG_NO_FUSED))
    if out is not None:
        opts.out_capacity = max(1, min(out.col.numel(), out.val.numel()))
        sc = cb_csr(0, 0, 0, out.row_ptr.data_ptr(), out.col.data_ptr(), out.val.data_ptr())
        ctx.check(ctx.lib.cb_spgemm_ex(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb),
                                       ctypes.byref(sc), ctypes.byref(opts)))
        n = sc.nnz
        return DeviceCSR(sc.nrows, sc.ncols, out.row_ptr[:sc.nrows + 1], out.col[:n], out.val[:n])
    sc = cb_csr()
    ctx.check(ctx.lib.cb_spgemm_ex(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb),
                                   ctypes.byref(sc), ctypes.byref(opts)))
    owner = _Owner(ctx, cb_csr(sc.nrows, sc.ncols, sc.nnz, sc.row_ptr, sc.col, sc.val))
    dev = A.row_ptr.device
    return DeviceCSR(sc.nrows, sc.ncols, _wrap(sc.row_ptr, sc.nrows + 1, torch.int64, owner, dev),
                     _wrap(sc.col, sc.nnz, torch.int32, owner, dev),
                     _wrap(sc.val, sc.nnz, dt, owner, dev), owner)


class _SpvOwner:
    """Frees a library-allocated sparse vector in stream order on the context's stream."""

    def __init__(self, ctx, v: cb_spvec):
        self.ctx = ctx
        self.v = v

    def __del__(self):
        try:
            self.ctx.lib.cb_spvec_free_async(self.ctx.handle, ctypes.byref(self.v))
        except Exception:
            pass


def spmspv(semiring: str, A: DeviceCSR, x_idx: torch.Tensor, x_val: torch.Tensor, *,
           validate: bool = True, ctx: Context | None = None, bucket: bool = False,
           timing: bool = False):
    """y^T = x^T A over the semiring (cb_spmspv): x is a sparse vector of length
    A.nrows given by int32 indices and values of the semiring's A type.  Returns
    (y_idx int32, y_val) device tensors, indices strictly increasing.
    `bucket=True` runs the bucket (propagation-blocking) form."""
    code, dt = SEMIRING[semiring]
    ctx = ctx or context()
    if x_idx.dtype != torch.int32 or x_val.dtype != OPERAND_DTYPES[semiring][0] or \
            x_idx.numel() != x_val.numel():
        raise ValueError("x needs int32 indices and values of the semiring's A dtype, equally many")
    sa = A.as_struct()
    nx = x_idx.numel()
    sx = cb_spvec(A.nrows, nx, x_idx.data_ptr() if nx else None, x_val.data_ptr() if nx else None)
    sy = cb_spvec()
    opts = make_opts(validate=validate, flags=(FLAG_SPMSPV_BUCKET if bucket else 0) |
                     (FLAG_TIMING if timing else 0))
    ctx.check(ctx.lib.cb_spmspv(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sx), ctypes.byref(sy),
                                ctypes.byref(opts)))
    owner = _SpvOwner(ctx, cb_spvec(sy.n, sy.nnz, sy.idx, sy.val))
    dev = A.row_ptr.device
    return (_wrap(sy.idx, sy.nnz, torch.int32, owner, dev), _wrap(sy.val, sy.nnz, dt, owner, dev))


def merge(semiring: str, parts, *, validate: bool = True, ctx: Context | None = None,
          timing: bool = False, fused: bool = True) -> DeviceCSR:
    """C = parts[0] (+) ... (+) parts[k-1] on the GPU (cb_merge); the parts are
    DeviceCSR of one shape holding C-type values.  The library allocates C."""
    code, dt = SEMIRING[semiring]
    ctx = ctx or context()
    arr = (cb_csr * len(parts))(*[p.as_struct() for p in parts])
    opts = make_opts(validate=validate,
                     flags=(FLAG_TIMING if timing else 0) | (0 if fused else FLAG_NO_FUSED))
    sc = cb_csr()
    ctx.check(ctx.lib.cb_merge(ctx.handle, code, len(parts), ctypes.cast(arr, c_void_p),
                               ctypes.byref(sc), ctypes.byref(opts)))
    owner = _Owner(ctx, cb_csr(sc.nrows, sc.ncols, sc.nnz, sc.row_ptr, sc.col, sc.val))
    dev = parts[0].row_ptr.device
    return DeviceCSR(sc.nrows, sc.ncols, _wrap(sc.row_ptr, sc.nrows + 1, torch.int64, owner, dev),
                     _wrap(sc.col, sc.nnz, torch.int32, owner, dev),
                     _wrap(sc.val, sc.nnz, dt, owner, dev), owner)


def fused_lanes(A: DeviceCSR, B: DeviceCSR, ctx: Context | None = None):
    """(lanes, flops): the smallest lanes per row (8, 16, 32) whose bounds
    every row of A.B meets (0 if none) and the total product count
    (cb_fused_lanes; synchronises)."""
    ctx = ctx or context()
    sa, sb = A.as_struct(), B.as_struct()
    lanes, flops = ctypes.c_int(0), c_int64(0)
    ctx.check(ctx.lib.cb_fused_lanes(ctx.handle, ctypes.byref(sa), ctypes.byref(sb),
                                     ctypes.byref(lanes), ctypes.byref(flops)))
    return lanes.value, flops.value


def fused_max_cols(lanes: int) -> int:
    return int(load().cb_fused_max_cols(int(lanes)))


def spgemm_fused(semiring: str, A: DeviceCSR, B: DeviceCSR, out: DeviceCSR, status: torch.Tensor,
                 lanes: int = 8, ctx: Context | None = None) -> None:
    """One-launch C = A (+).(x) B into `out` (cb_spgemm_fused): out.row_ptr
    gets nrows + 1 entries, out.col / out.val hold the capacity; `status`
    (int32 device tensor, zeroed by the caller) receives FUSED_* bits.
    Nothing is synchronised: nnz(C) is out.row_ptr[nrows] on the device."""
    code, dt = SEMIRING[semiring]
    ctx = ctx or context()
    if status.dtype != torch.int32 or not status.is_cuda:
        raise ValueError("status must be an int32 CUDA tensor")
    if out.val.dtype != dt:
        raise ValueError("out.val has the wrong dtype for this semiring")
    sa, sb = A.as_struct(), B.as_struct()
    cap = min(out.col.numel(), out.val.numel())
    sc = cb_csr(0, 0, 0, out.row_ptr.data_ptr(), out.col.data_ptr() if cap else None,
                out.val.data_ptr() if cap else None)
    ctx.check(ctx.lib.cb_spgemm_fused(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb),
                                      ctypes.byref(sc), cap, int(lanes), status.data_ptr()))


def row_stats(A: DeviceCSR, B: DeviceCSR, ctx: Context | None = None):
    """(flops[m] int64, maxb[m] int32) on the device (cb_row_stats)."""
    ctx = ctx or context()
    dev = A.row_ptr.device
    flops = torch.empty(A.nrows, dtype=torch.int64, device=dev)
    maxb = torch.empty(A.nrows, dtype=torch.int32, device=dev)
    sa, sb = A.as_struct(), B.as_struct()
    ctx.check(ctx.lib.cb_row_stats(ctx.handle, ctypes.byref(sa), ctypes.byref(sb),
                                   c_void_p(flops.data_ptr()), c_void_p(maxb.data_ptr())))
    return flops, maxb


def row_nnz(A: DeviceCSR, B: DeviceCSR, ctx: Context | None = None) -> torch.Tensor:
    """Exact nnz of every row of A.B on the device (cb_row_nnz, the symbolic phase)."""
    ctx = ctx or context()
    out = torch.empty(A.nrows, dtype=torch.int64, device=A.row_ptr.device)
    sa, sb = A.as_struct(), B.as_struct()
    ctx.check(ctx.lib.cb_row_nnz(ctx.handle, ctypes.byref(sa), ctypes.byref(sb),
                                 c_void_p(out.data_ptr())))
    return out


def exclusive_scan(x: torch.Tensor, ctx: Context | None = None) -> torch.Tensor:
    ctx = ctx or context()
    assert x.dtype == torch.int64 and x.is_contiguous()
    out = torch.empty(x.numel() + 1, dtype=torch.int64, device=x.device)
    ctx.check(ctx.lib.cb_exclusive_scan(ctx.handle, c_void_p(x.data_ptr()), x.numel(),
                                        c_void_p(out.data_ptr())))
    return out


def _view(ptr, n, dtype, device):
    """Tensor view of library memory that stays valid only while the callback runs."""
    return _wrap(ptr, n, dtype, None, device)


def spgemm_column_batches(semiring: str, A: DeviceCSR, B: DeviceCSR, budget_bytes: int, on_batch,
                          *, validate: bool = True, ctx: Context | None = None,
                          sizing: str = "exact", timing: bool = False, mlp=None,
                          margin: float = 0.25, resume_col: int = 0, resume_batch: int = 0) -> dict:
    """Column-batched C = A (+).(x) B (cb_spgemm_ex with budget_bytes > 0).

    on_batch(batch, col_lo, col_hi, Cb) is called for each batch with a
    DeviceCSR view of C[:, col_lo:col_hi) (global column indices) that is
    valid only during the call; return True to stop early.  Returns the
    call's statistics (batches, flops, nnz, ...).  resume_col / resume_batch
    restart a stopped call at the col_lo and index of its first unconsumed
    batch (only columns [resume_col, B.ncols) are formed).
    """
    code, dt = SEMIRING[semiring]
    ctx = ctx or context()
    dev = A.row_ptr.device
    errors = []

    def _cb(batch, lo, hi, cptr, user):
        try:
            c = cptr.contents
            view = DeviceCSR(c.nrows, c.ncols, _view(c.row_ptr, c.nrows + 1, torch.int64, dev),
                             _view(c.col, c.nnz, torch.int32, dev), _view(c.val, c.nnz, dt, dev))
            return 1 if on_batch(batch, lo, hi, view) else 0
        except Exception as e:  # never raise through the C ABI
            errors.append(e)
            return 1

    fn = BATCH_FN(_cb)
    sa, sb = A.as_struct(), B.as_struct()
    opts = make_opts(sizing=sizing, validate=validate, budget_bytes=budget_bytes, on_batch=fn,
                     flags=FLAG_TIMING if timing else 0, mlp=mlp, margin=margin)
    opts.resume_col = int(resume_col)
    opts.resume_batch = int(resume_batch)
    sc = cb_csr()
    ctx.check(ctx.lib.cb_spgemm_ex(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb),
                                   ctypes.byref(sc), ctypes.byref(opts)))
    if errors:
        raise errors[0]
    st = ctx.stats()
    st["nnz_total"] = sc.nnz
    return st


# ---------------------------------------------------------------------------
# learned row-size predictor
# ---------------------------------------------------------------------------

MLP_NPARAM = 4481
MLP_NFEAT = 4


def _ptr_or_none(t):
    return c_void_p(t.data_ptr()) if t is not None else None


class MLP:
    """Device-resident predictor (cb_mlp): fp32 master weights, bf16 copies, Adam state."""

    def __init__(self, params, norm):
        self.lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        nrm = np.ascontiguousarray(norm, dtype=np.float32)
        assert p.shape == (MLP_NPARAM,) and nrm.shape == (6,)
        self.handle = c_void_p()
        rc = self.lib.cb_mlp_create(ctypes.byref(self.handle), p.ctypes.data, nrm.ctypes.data)
        if rc != 0:
            raise CBError(rc, "cb_mlp_create failed")

    def __del__(self):
        try:
            if self.handle:
                self.lib.cb_mlp_destroy(self.handle)
                self.handle = c_void_p()
        except Exception:
            pass

    def get(self):
        p = np.zeros(MLP_NPARAM, np.float32)
        nrm = np.zeros(6, np.float32)
        step = ctypes.c_int64()
        rc = self.lib.cb_mlp_get(self.handle, p.ctypes.data, nrm.ctypes.data, ctypes.byref(step))
        if rc != 0:
            raise CBError(rc, "cb_mlp_get failed")
        return p, nrm, step.value

    @staticmethod
    def _check_feat(feat):
        if feat.dim() != 2 or feat.shape[1] != MLP_NFEAT or feat.dtype != torch.float32 \
                or not feat.is_contiguous():
            raise ValueError(f"features must be a contiguous float32 [m, {MLP_NFEAT}] tensor")

    def predict(self, feat: torch.Tensor, ncols: int, ctx: Context | None = None):
        self._check_feat(feat)
        ctx = ctx or context()
        m = feat.shape[0]
        z = torch.empty(m, dtype=torch.float32, device=feat.device)
        pred = torch.empty(m, dtype=torch.int64, device=feat.device)
        ctx.check(self.lib.cb_mlp_predict(ctx.handle, self.handle, c_void_p(feat.data_ptr()), m,
                                          int(ncols), c_void_p(z.data_ptr()),
                                          c_void_p(pred.data_ptr())))
        return z, pred

    def grad(self, feat: torch.Tensor, nnz: torch.Tensor, tau: float = 0.9,
             ctx: Context | None = None):
        self._check_feat(feat)
        ctx = ctx or context()
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        ctx.check(self.lib.cb_mlp_grad(ctx.handle, self.handle, c_void_p(feat.data_ptr()),
                                       c_void_p(nnz.data_ptr()), feat.shape[0], float(tau),
                                       c_void_p(g.data_ptr()), c_void_p(loss.data_ptr())))
        return g, loss

    def train(self, feat: torch.Tensor, nnz: torch.Tensor, epochs: int, batch: int, lr: float,
              tau: float = 0.9, ctx: Context | None = None):
        self._check_feat(feat)
        ctx = ctx or context()
        losses = np.zeros(max(epochs, 1), np.float32)
        ctx.check(self.lib.cb_mlp_train(ctx.handle, self.handle, c_void_p(feat.data_ptr()),
                                        c_void_p(nnz.data_ptr()), feat.shape[0], int(epochs),
                                        int(batch), float(lr), float(tau), losses.ctypes.data))
        return losses[:epochs]


def row_features(A: DeviceCSR, B: DeviceCSR, ctx: Context | None = None) -> torch.Tensor:
    """Raw per-row features (nnz(A_i), flops_i, maxB_i, output width) as a
    float32 [m, 4] device tensor."""
    ctx = ctx or context()
    feat = torch.empty((A.nrows, 4), dtype=torch.float32, device=A.row_ptr.device)
    sa, sb = A.as_struct(), B.as_struct()
    ctx.check(ctx.lib.cb_row_features(ctx.handle, ctypes.byref(sa), ctypes.byref(sb),
                                      c_void_p(feat.data_ptr())))
    return feat


def spgemm_batched(semirings, As, Bs, on_wave, *, budget_bytes: int = 0, validate: bool = True,
                   sizing: str = "exact", mlp=None, margin: float = 0.25,
                   ctx: Context | None = None, mode: str = "host",
                   digests: torch.Tensor | None = None, fused: bool = True) -> dict:
    """Batched products C_i = A_i (+).(x) B_i (cb_spgemm_batched).

    on_wave(wave, first, end, Cw) receives a DeviceCSR that stacks
    C_first..C_{end-1} by rows (each product's own column indices), valid
    only during the call; return True to stop.  Returns the statistics.
    mode "sync_free" runs each wave without host synchronisation inside it;
    mode "graph" also captures all waves into one CUDA graph, and on_wave is
    then called as on_wave(wave, first, end, nrows, nnz) from a graph host
    node (no tensors: CUDA may not be used there; the return value is
    ignored).  Both cut waves by the flop bound; a group with a product whose
    bound alone exceeds the budget runs as mode "host".
    `digests` (optional, an int64 CUDA tensor of 2 * len(As) entries) receives
    each product's two digest words (cb.h, cb_spgemm_batched), as raw 64-bit
    patterns.  `fused=False` keeps every wave on the two-phase path (no
    one-launch or work-queue kernel).
    """
    flags = {"host": 0, "sync_free": FLAG_SYNC_FREE, "graph": FLAG_GRAPH}[mode] | \
        (0 if fused else FLAG_NO_FUSED)
    ctx = ctx or context()
    n = len(As)
    assert len(Bs) == n and len(semirings) == n
    codes = (ctypes.c_int * max(n, 1))(*[SEMIRING[s][0] for s in semirings])
    sa = (cb_csr * max(n, 1))(*[a.as_struct() for a in As])
    sb = (cb_csr * max(n, 1))(*[b.as_struct() for b in Bs])
    dev = As[0].row_ptr.device if n else torch.device("cuda")
    errors = []

    def _cb(wave, first, end, cptr, user):
        try:
            c = cptr.contents
            if mode == "graph":
                on_wave(wave, first, end, c.nrows, c.nnz)
                return 0
            dt = SEMIRING[semirings[first]][1]
            view = DeviceCSR(c.nrows, c.ncols, _view(c.row_ptr, c.nrows + 1, torch.int64, dev),
                             _view(c.col, c.nnz, torch.int32, dev), _view(c.val, c.nnz, dt, dev))
            return 1 if on_wave(wave, first, end, view) else 0
        except Exception as e:  # never raise through the C ABI
            errors.append(e)
            return 1

    fn = BATCH_FN(_cb)
    opts = make_opts(sizing=sizing, validate=validate, budget_bytes=budget_bytes, on_batch=fn,
                     mlp=mlp, margin=margin, flags=flags)
    if digests is not None:
        if digests.dtype != torch.int64 or not digests.is_cuda or digests.numel() < 2 * n \
                or not digests.is_contiguous():
            raise ValueError("digests must be a contiguous int64 CUDA tensor of 2 * count entries")
        opts.digests = digests.data_ptr()
    ctx.check(ctx.lib.cb_spgemm_batched(ctx.handle, n, ctypes.cast(codes, c_void_p),
                                        ctypes.cast(sa, c_void_p), ctypes.cast(sb, c_void_p),
                                        ctypes.byref(opts)))
    if errors:
        raise errors[0]
    return ctx.stats()


def autotune(semiring: str, A: DeviceCSR, B: DeviceCSR, *, sizing: str = "exact", mlp=None,
             margin: float = 0.25, ctx: Context | None = None):
    """Time A.B under a grid of tier bounds (cb_autotune); the context keeps the
    fastest.  Returns (bounds dict, milliseconds)."""
    ctx = ctx or context()
    code, _ = SEMIRING[semiring]
    sa, sb = A.as_struct(), B.as_struct()
    opts = make_opts(sizing=sizing, mlp=mlp, margin=margin)
    t = cb_tune()
    ms = ctypes.c_float()
    ctx.check(ctx.lib.cb_autotune(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(opts),
                                  ctypes.byref(t), ctypes.byref(ms)))
    return {k: getattr(t, k) for k, _ in cb_tune._fields_}, ms.value


def autotune_cached(semiring: str, A: DeviceCSR, B: DeviceCSR, cache_path: str, *,
                    sizing: str = "exact", mlp=None, margin: float = 0.25,
                    ctx: Context | None = None):
    """cb_autotune through the JSON cache at cache_path (keyed by device name,
    semiring, sizing and size class): a hit sets the cached bounds with no GPU
    work.  Returns (bounds dict, milliseconds, hit)."""
    ctx = ctx or context()
    code, _ = SEMIRING[semiring]
    sa, sb = A.as_struct(), B.as_struct()
    opts = make_opts(sizing=sizing, mlp=mlp, margin=margin)
    t = cb_tune()
    ms = ctypes.c_float()
    hit = ctypes.c_int()
    ctx.check(ctx.lib.cb_autotune_cached(ctx.handle, code, ctypes.byref(sa), ctypes.byref(sb),
                                         ctypes.byref(opts), os.fsencode(cache_path), ctypes.byref(t),
                                         ctypes.byref(ms), ctypes.byref(hit)))
    return {k: getattr(t, k) for k, _ in cb_tune._fields_}, ms.value, bool(hit.value)


def tune_key(device_name: str, semiring: str, nrows: int, nnz_a: int, nnz_b: int,
             sizing: str = "exact") -> str:
    """The autotune cache key (cb_tune_key); host only."""
    lib = load()
    buf = ctypes.create_string_buffer(512)
    rc = lib.cb_tune_key(device_name.encode(), SEMIRING[semiring][0], SIZING[sizing], nrows, nnz_a,
                         nnz_b, buf, len(buf))
    if rc:
        raise CBError(rc, "cb_tune_key: bad argument")
    return buf.value.decode()


def tune_cache_get(path: str, key: str):
    """(bounds dict, ms) for key from the cache file, or None; host only."""
    lib = load()
    t, ms, found = cb_tune(), ctypes.c_float(), ctypes.c_int()
    rc = lib.cb_tune_cache_get(os.fsencode(path), key.encode(), ctypes.byref(t), ctypes.byref(ms),
                               ctypes.byref(found))
    if rc:
        raise CBError(rc, f"tune cache {path} unreadable or not a tune cache")
    if not found.value:
        return None
    return {k: getattr(t, k) for k, _ in cb_tune._fields_}, ms.value


def tune_cache_put(path: str, key: str, bounds: dict, ms: float) -> None:
    """Insert or replace key's entry in the cache file; host only."""
    lib = load()
    t = cb_tune(**bounds)
    rc = lib.cb_tune_cache_put(os.fsencode(path), key.encode(), ctypes.byref(t), float(ms))
    if rc:
        raise CBError(rc, f"tune cache {path} unreadable or not writable")
