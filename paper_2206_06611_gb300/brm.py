"""Python binding of libbrm (BRMerge SpGEMM for sm_103a) -- argument
marshalling only.

Every function here forwards to the extern "C" entry point of the same name in
``libbrm.so`` (declared in ``include/brm.h``).  PyTorch supplies device memory
(its caching allocator is handed to the library as the brm_allocator callbacks)
and the stream (the current torch stream); all computation runs in the
library's CUDA kernels.  There is no fallback: if the library cannot be built
or loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import re

import numpy as np

from . import build as _build

# ---------------------------------------------------------------------------
# C structures (mirror include/brm.h)
# ---------------------------------------------------------------------------
BRM_OK = 0
BRM_ERR = {-1: "BRM_ERR_INVALID", -2: "BRM_ERR_SHAPE", -3: "BRM_ERR_DTYPE", -4: "BRM_ERR_OOM",
           -5: "BRM_ERR_OVERFLOW", -6: "BRM_ERR_CUDA", -7: "BRM_ERR_TIMEOUT"}
BRM_F32, BRM_F64 = 0, 1


class brm_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


class brm_csr_out(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class brm_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


class brm_options(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int32), ("compensated", ctypes.c_int32),
                ("warp_max_nprod", ctypes.c_int32), ("block_max_nprod", ctypes.c_int32),
                ("reg_max_nprod", ctypes.c_int32), ("reg_keys", ctypes.c_int32), ("reg_warps", ctypes.c_int32),
                ("symbolic_hash", ctypes.c_int32), ("reg_top", ctypes.c_int32), ("reg_perm", ctypes.c_int32),
                ("reg_num_half", ctypes.c_int32), ("reg_num_direct", ctypes.c_int32),
                ("long_bucket", ctypes.c_int32),
                ("arena_bytes", ctypes.c_size_t),
                ("upper_chunk_bytes", ctypes.c_size_t),
                ("long_window", ctypes.c_int32)]


class BrmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{BRM_ERR.get(code, code)}: {msg}")
        self.code = code


# ---------------------------------------------------------------------------
# library loading
# ---------------------------------------------------------------------------
_lib = None
HEADER = os.path.join(_build.INCLUDE, "brm.h")


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libbrm.so (building it first when stale and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbrm.so is not built ({_build.LIB}); run paper_2206_06611_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    pcsr, pout = ctypes.POINTER(brm_csr), ctypes.POINTER(brm_csr_out)
    popt, pal = ctypes.POINTER(brm_options), ctypes.POINTER(brm_allocator)
    lib.brm_options_default.argtypes = [popt]
    lib.brm_options_default.restype = None
    lib.brm_last_error.restype = ctypes.c_char_p
    lib.brm_version.restype = ctypes.c_char_p
    lib.brm_spgemm_symbolic.argtypes = [pcsr, pcsr, P, ctypes.POINTER(I64), popt, pal, P]
    lib.brm_spgemm_precise.argtypes = [pcsr, pcsr, pout, popt, pal, P]
    lib.brm_spgemm_upper.argtypes = [pcsr, pcsr, pout, popt, pal, P]
    lib.brm_csr_out_free.argtypes = [pout, pal, P]
    lib.brm_csr_out_free.restype = None
    lib.brm_row_nprod.argtypes = [pcsr, pcsr, P, P, P, P, P]
    lib.brm_row_split.argtypes = [pcsr, pcsr, ctypes.c_int32, P, pal, P]
    lib.brm_row_split.restype = ctypes.c_int
    lib.brm_spgemm_numeric_noalloc.argtypes = [pcsr, pcsr, P, P, P, popt, P]
    lib.brm_spgemm_backward.argtypes = [pcsr, pcsr, P, P, P, P, P, popt, pal, P]
    lib.brm_spgemm_backward.restype = ctypes.c_int
    I32 = ctypes.c_int32
    lib.brm_spgemm_batched.argtypes = [I32, pcsr, pcsr, pout, P, popt, pal, P]
    lib.brm_batch_create.argtypes = [I32, pcsr, pcsr, popt, pal, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.brm_batch_numeric.argtypes = [P, P]
    lib.brm_batch_graph_launch.argtypes = [P, P]
    lib.brm_batch_check.argtypes = [P, P]
    lib.brm_batch_result.argtypes = [P, pout, P]
    lib.brm_batch_take.argtypes = [P, pout, P]
    lib.brm_batch_destroy.argtypes = [P]
    lib.brm_batch_destroy.restype = None
    lib.brm_autotune.argtypes = [I32, pcsr, pcsr, popt, popt, ctypes.POINTER(ctypes.c_double), pal, P]
    for f in (lib.brm_spgemm_batched, lib.brm_batch_create, lib.brm_batch_numeric, lib.brm_batch_graph_launch,
              lib.brm_batch_check, lib.brm_batch_result, lib.brm_batch_take, lib.brm_autotune):
        f.restype = ctypes.c_int
    for f in (lib.brm_spgemm_symbolic, lib.brm_spgemm_precise, lib.brm_spgemm_upper, lib.brm_row_nprod,
              lib.brm_spgemm_numeric_noalloc):
        f.restype = ctypes.c_int
    lib.brm_trace_enable.argtypes = [ctypes.c_int]
    lib.brm_trace_enable.restype = ctypes.c_int
    lib.brm_trace_reset.argtypes = []
    lib.brm_trace_reset.restype = None
    lib.brm_trace_read.argtypes = [P, P, ctypes.c_int]
    lib.brm_trace_read.restype = ctypes.c_int
    lib.brm_trace_phase_name.argtypes = [ctypes.c_int]
    lib.brm_trace_phase_name.restype = ctypes.c_char_p
    lib.brm_kernel_launches.argtypes = []
    lib.brm_kernel_launches.restype = ctypes.c_int64
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    """Function names declared in include/brm.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(brm_[a-z_0-9]+)\s*\(", text, re.M)))


def _check(rc: int):
    if rc != BRM_OK:
        raise BrmError(rc, load().brm_last_error().decode())


# ---------------------------------------------------------------------------
# device CSR and marshalling
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class DeviceCSR:
    """CSR on the GPU: rp (int32 for inputs, int64 for results), col int32, val."""
    rows: int
    cols: int
    rp: "torch.Tensor"
    col: "torch.Tensor"
    val: "torch.Tensor | None"

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def to_host(self):
        from .inputs import CSR
        val = None if self.val is None else self.val.cpu().numpy()
        return CSR(self.rows, self.cols, self.rp.cpu().numpy(), self.col.cpu().numpy(), val)


def to_device(A, device="cuda", dtype=None) -> DeviceCSR:
    """Copy a host CSR (paper_2206_06611_gb300.inputs.CSR) to the GPU."""
    import torch
    val = A.val if dtype is None else A.val.astype(dtype)
    return DeviceCSR(A.rows, A.cols,
                     torch.from_numpy(np.ascontiguousarray(A.rp, dtype=np.int32)).to(device),
                     torch.from_numpy(np.ascontiguousarray(A.col, dtype=np.int32)).to(device),
                     torch.from_numpy(np.ascontiguousarray(val)).to(device))


def _dtype_code(t) -> int:
    import torch
    if t is None:
        return BRM_F64
    if t.dtype == torch.float64:
        return BRM_F64
    if t.dtype == torch.float32:
        return BRM_F32
    raise TypeError(f"unsupported value dtype {t.dtype}")


def _csr_struct(A: DeviceCSR) -> brm_csr:
    import torch
    for t, want in ((A.rp, torch.int32), (A.col, torch.int32)):
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise TypeError("row_ptr and col_idx must be contiguous int32 CUDA tensors")
    if A.val is not None and (not A.val.is_cuda or not A.val.is_contiguous()):
        raise TypeError("values must be a contiguous CUDA tensor")
    return brm_csr(A.rows, A.cols, A.nnz, A.rp.data_ptr(), A.col.data_ptr() if A.nnz else None,
                   None if A.val is None or A.nnz == 0 else A.val.data_ptr(), _dtype_code(A.val))


class TorchAllocator:
    """brm_allocator backed by torch's caching allocator (current device/stream)."""

    def __init__(self, device=None):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.live = {}
        self._alloc_cb = ALLOC_FN(self._alloc)
        self._release_cb = RELEASE_FN(self._release)
        self.struct = brm_allocator(self._alloc_cb, self._release_cb, None)

    def _alloc(self, nbytes, ctx):
        import torch
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except torch.OutOfMemoryError:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _release(self, p, ctx):
        self.live.pop(p, None)

    def take(self, p, dtype, count):
        """Hand the allocation at p over to Python as a typed tensor."""
        t = self.live.pop(p)
        return t.view(dtype)[:count]


_alloc_cache = {}


def _allocator():
    import torch
    dev = torch.cuda.current_device()
    if dev not in _alloc_cache:
        _alloc_cache[dev] = TorchAllocator(dev)
    return _alloc_cache[dev]


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def options(validate=False, compensated=False, warp_max_nprod=0, block_max_nprod=0, reg_max_nprod=0,
            reg_keys=0, reg_warps=0, symbolic_hash=False, reg_top=True, reg_perm=True, reg_num_half=True,
            reg_num_direct=True, long_bucket=False, arena_bytes=0, upper_chunk_bytes=0,
            long_window=None) -> brm_options:
    o = brm_options()
    load().brm_options_default(ctypes.byref(o))
    o.validate = int(bool(validate))
    o.compensated = int(bool(compensated))
    if warp_max_nprod:
        o.warp_max_nprod = warp_max_nprod
    if block_max_nprod:
        o.block_max_nprod = block_max_nprod
    if reg_max_nprod:
        o.reg_max_nprod = reg_max_nprod
    if reg_keys:
        o.reg_keys = reg_keys
    if reg_warps:
        o.reg_warps = reg_warps
    o.symbolic_hash = int(bool(symbolic_hash))
    o.reg_top = int(bool(reg_top))
    o.reg_perm = int(bool(reg_perm))
    o.reg_num_half = int(bool(reg_num_half))
    o.reg_num_direct = int(bool(reg_num_direct))
    o.long_bucket = int(bool(long_bucket))
    o.arena_bytes = arena_bytes
    o.upper_chunk_bytes = upper_chunk_bytes
    if long_window is not None:
        # True: every long row of at most 2048 lists takes the column tiles
        o.long_window = (2 if long_window else 0) if isinstance(long_window, bool) else int(long_window)
    return o


def _result(al: TorchAllocator, C: brm_csr_out, val_dtype) -> DeviceCSR:
    import torch
    rp = al.take(C.row_ptr, torch.int64, C.rows + 1)
    col = al.take(C.col_idx, torch.int32, C.nnz)
    val = al.take(C.val, val_dtype, C.nnz)
    return DeviceCSR(C.rows, C.cols, rp, col, val)


def brm_spgemm_precise(A: DeviceCSR, B: DeviceCSR, *, compensated=False, validate=False, stream=None,
                       **opts) -> DeviceCSR:
    """C = A*B by BRMerge-Precise (symbolic pass, exact allocation, numeric pass)."""
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    o = options(validate=validate, compensated=compensated, **opts)
    al = _allocator()
    C = brm_csr_out()
    _check(lib.brm_spgemm_precise(ctypes.byref(a), ctypes.byref(b), ctypes.byref(C), ctypes.byref(o),
                                  ctypes.byref(al.struct), _stream(stream)))
    return _result(al, C, A.val.dtype)


def brm_spgemm_upper(A: DeviceCSR, B: DeviceCSR, *, compensated=False, validate=False, stream=None,
                     **opts) -> DeviceCSR:
    """C = A*B by BRMerge-Upper (upper-bound C_bar, numeric pass, compaction)."""
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    o = options(validate=validate, compensated=compensated, **opts)
    al = _allocator()
    C = brm_csr_out()
    _check(lib.brm_spgemm_upper(ctypes.byref(a), ctypes.byref(b), ctypes.byref(C), ctypes.byref(o),
                                ctypes.byref(al.struct), _stream(stream)))
    return _result(al, C, A.val.dtype)


def brm_spgemm_symbolic(A: DeviceCSR, B: DeviceCSR, *, validate=False, stream=None, **opts):
    """(C.row_ptr as an int64 CUDA tensor, nnz(C))."""
    import torch
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    o = options(validate=validate, **opts)
    rp = torch.empty(A.rows + 1, dtype=torch.int64, device=A.rp.device)
    nnz = ctypes.c_int64(0)
    _check(lib.brm_spgemm_symbolic(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(rp.data_ptr()),
                                   ctypes.byref(nnz), ctypes.byref(o), ctypes.byref(_allocator().struct),
                                   _stream(stream)))
    return rp, int(nnz.value)


def brm_spgemm_numeric_noalloc(A: DeviceCSR, B: DeviceCSR, C_rp, C_col, C_val, *, compensated=False,
                               validate=False, stream=None, **opts) -> DeviceCSR:
    """Numeric pass into caller-provided C arrays; the library allocates
    nothing (its workspace is a fixed array inside libbrm).  C_rp is the int64
    row pointer of A*B (e.g. from brm_spgemm_symbolic); C_col (int32) and C_val
    (A's dtype) hold C_rp[-1] entries and are overwritten."""
    import torch
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    if C_rp.dtype != torch.int64 or C_col.dtype != torch.int32 or C_val.dtype != A.val.dtype:
        raise TypeError("C_rp must be int64, C_col int32 and C_val of A's value dtype")
    for t in (C_rp, C_col, C_val):
        if not t.is_cuda or not t.is_contiguous():
            raise TypeError("C arrays must be contiguous CUDA tensors")
    o = options(validate=validate, compensated=compensated, **opts)
    _check(lib.brm_spgemm_numeric_noalloc(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(C_rp.data_ptr()),
                                          ctypes.c_void_p(C_col.data_ptr()), ctypes.c_void_p(C_val.data_ptr()),
                                          ctypes.byref(o), _stream(stream)))
    return DeviceCSR(A.rows, B.cols, C_rp, C_col, C_val)


def brm_spgemm_backward(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, dC, want_da=True, want_db=True, stream=None):
    """(dA on A's pattern, dB on B's pattern) of a loss with dLoss/dC = dC on
    C's pattern; either is None when not wanted."""
    import torch
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    if dC.dtype != A.val.dtype or not dC.is_cuda or not dC.is_contiguous() or dC.numel() != C.nnz:
        raise TypeError("dC must be a contiguous CUDA tensor of C's nnz values in A's dtype")
    dA = torch.empty_like(A.val) if want_da else None
    dB = torch.empty_like(B.val) if want_db else None
    _check(lib.brm_spgemm_backward(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(C.rp.data_ptr()),
                                   ctypes.c_void_p(C.col.data_ptr() if C.nnz else None),
                                   ctypes.c_void_p(dC.data_ptr() if C.nnz else None),
                                   ctypes.c_void_p(dA.data_ptr() if dA is not None and A.nnz else None),
                                   ctypes.c_void_p(dB.data_ptr() if dB is not None and B.nnz else None),
                                   None, ctypes.byref(_allocator().struct), _stream(stream)))
    return dA, dB


# ---------------------------------------------------------------------------
# batched products
# ---------------------------------------------------------------------------
def _csr_array(Ms):
    arr = (brm_csr * max(len(Ms), 1))()
    for i, M in enumerate(Ms):
        arr[i] = _csr_struct(M)
    return arr


def _options_from(o: brm_options) -> dict:
    return {f: getattr(o, f) for f, _ in brm_options._fields_}


def _stacked(al, C: brm_csr_out, dtype, take: bool) -> DeviceCSR:
    import torch
    if take:
        return _result(al, C, dtype)
    rp = al.live[C.row_ptr].view(torch.int64)[:C.rows + 1]
    col = al.live[C.col_idx].view(torch.int32)[:C.nnz]
    val = al.live[C.val].view(dtype)[:C.nnz]
    return DeviceCSR(C.rows, C.cols, rp, col, val)


def brm_spgemm_batched(As, Bs, *, stream=None, **opts):
    """C_p = A_p * B_p for all p in one batched BRMerge-Precise call.
    Returns (the stacked C as a DeviceCSR, row offsets: a list of count + 1)."""
    if len(As) != len(Bs):
        raise ValueError("As and Bs differ in length")
    lib = load()
    a, b = _csr_array(As), _csr_array(Bs)
    o = options(**opts)
    al = _allocator()
    C = brm_csr_out()
    off = (ctypes.c_int64 * (len(As) + 1))()
    _check(lib.brm_spgemm_batched(len(As), a, b, ctypes.byref(C), ctypes.cast(off, ctypes.c_void_p), ctypes.byref(o),
                                  ctypes.byref(al.struct), _stream(stream)))
    return _result(al, C, As[0].val.dtype), list(off)


def split(C: DeviceCSR, offsets, cols=None):
    """The products of a stacked result as DeviceCSRs (views of C's arrays;
    each row pointer rebased to start at 0)."""
    out = []
    for p in range(len(offsets) - 1):
        r0, r1 = offsets[p], offsets[p + 1]
        rp = C.rp[r0:r1 + 1]
        base = int(rp[0].item()) if r1 >= r0 else 0
        lo, hi = base, int(rp[-1].item())
        out.append(DeviceCSR(r1 - r0, C.cols if cols is None else cols[p], rp - base, C.col[lo:hi], C.val[lo:hi]))
    return out


class Batch:
    """A prepared batch (brm_batch_*): symbolic pass done and C allocated;
    numeric() / graph_launch() recompute C's values from the current values
    of the same input arrays."""

    def __init__(self, As, Bs, *, stream=None, **opts):
        if len(As) != len(Bs):
            raise ValueError("As and Bs differ in length")
        self.lib = load()
        self.As, self.Bs = list(As), list(Bs)          # keep the inputs alive
        a, b = _csr_array(self.As), _csr_array(self.Bs)
        o = options(**opts)
        self.al = _allocator()
        h = ctypes.c_void_p()
        _check(self.lib.brm_batch_create(len(As), a, b, ctypes.byref(o), ctypes.byref(self.al.struct),
                                         _stream(stream), ctypes.byref(h)))
        self.h = h
        self.dtype = As[0].val.dtype if As else None

    def numeric(self, stream=None):
        _check(self.lib.brm_batch_numeric(self.h, _stream(stream)))

    def graph_launch(self, stream=None):
        _check(self.lib.brm_batch_graph_launch(self.h, _stream(stream)))

    def check(self, stream=None):
        _check(self.lib.brm_batch_check(self.h, _stream(stream)))

    def result(self):
        """(stacked C as views of the batch's arrays, row offsets)."""
        C = brm_csr_out()
        off = (ctypes.c_int64 * (len(self.As) + 1))()
        _check(self.lib.brm_batch_result(self.h, ctypes.byref(C), ctypes.cast(off, ctypes.c_void_p)))
        return _stacked(self.al, C, self.dtype, take=False), list(off)

    def close(self):
        if self.h:
            self.lib.brm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def brm_autotune(As, Bs, *, stream=None, **base):
    """(the fastest options as a dict, its milliseconds) for these products."""
    lib = load()
    a, b = _csr_array(As), _csr_array(Bs)
    o = options(**base)
    best = brm_options()
    ms = ctypes.c_double(0)
    _check(lib.brm_autotune(len(As), a, b, ctypes.byref(o), ctypes.byref(best), ctypes.byref(ms),
                            ctypes.byref(_allocator().struct), _stream(stream)))
    return _options_from(best), float(ms.value)


def _spgemm_fn():
    import torch

    class _SpGEMM(torch.autograd.Function):
        """C.val = (A * B).val with the hand-written masked backward."""

        @staticmethod
        def forward(ctx, a_val, b_val, A, B, method, opts):
            dA = DeviceCSR(A.rows, A.cols, A.rp, A.col, a_val.detach())
            dB = DeviceCSR(B.rows, B.cols, B.rp, B.col, b_val.detach())
            f = brm_spgemm_precise if method == "precise" else brm_spgemm_upper
            C = f(dA, dB, **opts)
            ctx.save_for_backward(a_val.detach(), b_val.detach(), C.rp, C.col)
            ctx.shapes = (A, B)
            ctx.mark_non_differentiable(C.rp, C.col)
            return C.val, C.rp, C.col

        @staticmethod
        def backward(ctx, g_val, g_rp, g_col):
            a_val, b_val, crp, ccol = ctx.saved_tensors
            A, B = ctx.shapes
            dA = DeviceCSR(A.rows, A.cols, A.rp, A.col, a_val)
            dB = DeviceCSR(B.rows, B.cols, B.rp, B.col, b_val)
            C = DeviceCSR(A.rows, B.cols, crp, ccol, None)
            ga, gb = brm_spgemm_backward(dA, dB, C, g_val.contiguous(), want_da=ctx.needs_input_grad[0],
                                         want_db=ctx.needs_input_grad[1])
            return ga, gb, None, None, None, None

    return _SpGEMM


_SPGEMM = None


def spgemm(A: DeviceCSR, B: DeviceCSR, method: str = "precise", **opts) -> DeviceCSR:
    """C = A*B whose values are differentiable with respect to A.val and
    B.val (torch autograd); the backward pass is brm_spgemm_backward."""
    global _SPGEMM
    if _SPGEMM is None:
        _SPGEMM = _spgemm_fn()
    val, rp, col = _SPGEMM.apply(A.val, B.val, A, B, method, opts)
    return DeviceCSR(A.rows, B.cols, rp, col, val)


def brm_row_nprod(A: DeviceCSR, B: DeviceCSR, *, stream=None):
    """(per-row product counts int64 tensor, total, max row nprod, max row nnz of A)."""
    import torch
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    out = torch.empty(max(A.rows, 1), dtype=torch.int64, device=A.rp.device)
    tot, mx, ml = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.brm_row_nprod(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(out.data_ptr()), ctypes.byref(tot),
                             ctypes.byref(mx), ctypes.byref(ml), _stream(stream)))
    return out[:A.rows], int(tot.value), int(mx.value), int(ml.value)


# ---------------------------------------------------------------------------
# one product over several GPUs: the static row split
# ---------------------------------------------------------------------------
def brm_row_split(A: DeviceCSR, B: DeviceCSR, parts: int, *, stream=None) -> list:
    """Row bounds (parts + 1 ints) of the nprod-balanced static split."""
    lib = load()
    a, b = _csr_struct(A), _csr_struct(B)
    out = (ctypes.c_int64 * (parts + 1))()
    _check(lib.brm_row_split(ctypes.byref(a), ctypes.byref(b), int(parts), ctypes.cast(out, ctypes.c_void_p),
                             ctypes.byref(_allocator().struct), _stream(stream)))
    return list(out)


def row_slice(A: DeviceCSR, r0: int, r1: int) -> DeviceCSR:
    """Rows r0 .. r1-1 of A as a CSR of their own (row pointer rebased to 0;
    columns and values are views of A's)."""
    s, e = int(A.rp[r0].item()), int(A.rp[r1].item())
    rp = (A.rp[r0:r1 + 1] - s).to(A.rp.dtype)
    return DeviceCSR(r1 - r0, A.cols, rp, A.col[s:e], None if A.val is None else A.val[s:e])


def global_row_offset(nnz_local: int, group=None, device=None) -> tuple:
    """(offset of this rank's rows in C's global arrays, global nnz): one
    all-gather of every rank's nnz (int64) over torch.distributed."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    t = torch.tensor([int(nnz_local)], dtype=torch.int64, device=device)
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    counts = [int(x.item()) for x in parts]
    return sum(counts[:rank]), sum(counts)


def spgemm_sharded(A: DeviceCSR, B: DeviceCSR, group=None, **opts):
    """This rank's share of C = A * B over the ranks of a process group: the
    rows (r0, r1) of the static split, computed by BRMerge-Precise on that
    slice of A (B whole on every rank), and their place in the global C.
    Returns (C rows as a DeviceCSR with a local row pointer, r0, r1, offset
    of the rows' entries in the global C, global nnz)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    bounds = brm_row_split(A, B, world)
    r0, r1 = bounds[rank], bounds[rank + 1]
    C = brm_spgemm_precise(row_slice(A, r0, r1), B, **opts)
    dev = C.rp.device if dist.get_backend(group) == "nccl" else "cpu"
    off, total = global_row_offset(C.nnz, group, dev)
    return C, r0, r1, off, total


def spgemm_sharded_backward(A: DeviceCSR, B: DeviceCSR, C: DeviceCSR, dC, r0: int, r1: int, group=None):
    """The backward of spgemm_sharded on this rank: for its rows r0 .. r1-1
    (C and dC: this rank's rows, local row pointer), dA of those rows' entries
    of A (A's values A.rp[r0] .. A.rp[r1]-1, local to the rank) and dB of the
    whole product -- every rank's dB of its rows (the library's backward on
    the row slice, summed over those rows in increasing order) added up over
    the group by one all-reduce, the exchange step of the row split.  The
    ranks' partial sums are added in the collective's order, so dB may differ
    from a single device's ordered sum in the last bits."""
    import torch.distributed as dist
    dA, dB = brm_spgemm_backward(row_slice(A, r0, r1), B, C, dC)
    if dist.get_backend(group) == "nccl":
        dist.all_reduce(dB, op=dist.ReduceOp.SUM, group=group)
        return dA, dB
    host = dB.cpu()
    dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
    return dA, host.to(dB.device)


# ---------------------------------------------------------------------------
# tracing
# ---------------------------------------------------------------------------
def brm_trace_enable(on: bool = True) -> bool:
    return bool(load().brm_trace_enable(int(bool(on))))


def brm_trace_reset() -> None:
    load().brm_trace_reset()


def brm_trace_read() -> dict:
    """{phase name: (device milliseconds, kernel launches)} accumulated so far."""
    lib = load()
    n = 16
    ms = (ctypes.c_double * n)()
    nl = (ctypes.c_int64 * n)()
    k = lib.brm_trace_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(nl, ctypes.c_void_p), n)
    return {lib.brm_trace_phase_name(i).decode(): (ms[i], nl[i]) for i in range(k)}


def brm_kernel_launches() -> int:
    return int(load().brm_kernel_launches())
