"""Out-of-memory handling through the caller's allocator (include/brm.h: on
error every allocation made by the call is released and *C is zeroed).

The fault is injected on the host: an allocator that counts its calls and
returns NULL at call k.  A call runs once to count its allocations, then once
for every k.  Each run must end with BRM_OK (an allocation the library can do
without, e.g. the workspace slab or the whole C_bar of BRMerge-Upper, which
then runs in row chunks) and the oracle's result, or with BRM_ERR_OOM and a
zeroed C; either way every allocation not handed to the caller is released.
Covered: BRMerge-Precise (with long rows), BRMerge-Upper in row chunks,
batched products, the symbolic pass and the backward pass.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_rows_exact, bins_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402


class FailingAllocator:
    """brm_allocator over torch memory that returns NULL on call number fail_at."""

    def __init__(self, fail_at=0):
        self.fail_at, self.calls, self.live = fail_at, 0, {}
        self._a = brm.ALLOC_FN(self._alloc)
        self._r = brm.RELEASE_FN(self._release)
        self.struct = brm.brm_allocator(self._a, self._r, None)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _release(self, p, ctx):
        if p:
            assert p in self.live, "released a pointer the allocator did not hand out"
            del self.live[p]


def _zeroed(C):
    return C.rows == 0 and C.nnz == 0 and not C.row_ptr and not C.col_idx and not C.val


def _sweep(call, check, owned):
    """call(al) -> (rc, C or None); check(C, al) verifies a result (its arrays
    are tensors of al); owned(C) lists the pointers a successful call hands
    over.  Returns the allocations of a successful call."""
    al = FailingAllocator()
    rc, C = call(al)
    torch.cuda.synchronize()
    assert rc == 0, brm.load().brm_last_error()
    n = al.calls
    check(C, al)
    assert set(al.live) == set(owned(C))
    outcomes = set()
    for k in range(1, n + 1):
        al = FailingAllocator(k)
        rc, C = call(al)
        torch.cuda.synchronize()
        assert rc in (0, -4), (k, rc, brm.load().brm_last_error())
        outcomes.add(rc)
        if rc == 0:
            check(C, al)
            assert set(al.live) == set(owned(C))
        else:
            assert not al.live, f"allocation {k} failed and {len(al.live)} allocations were not released"
            if C is not None:
                assert _zeroed(C)
    assert -4 in outcomes
    return n


def _product_call(fn, A, B, **kw):
    lib = brm.load()
    a, b = brm._csr_struct(A), brm._csr_struct(B)
    o = brm.options(**kw)

    def call(al):
        C = brm.brm_csr_out()
        rc = getattr(lib, fn)(ctypes.byref(a), ctypes.byref(b), ctypes.byref(C), ctypes.byref(o),
                              ctypes.byref(al.struct), brm._stream())
        return rc, C
    return call


def _result(C, al):
    """The result's arrays as views of the allocator's tensors."""
    rp = al.live[C.row_ptr].view(torch.int64)[:C.rows + 1]
    col = al.live[C.col_idx].view(torch.int32)[:C.nnz]
    val = al.live[C.val].view(torch.float64)[:C.nnz]
    return brm.DeviceCSR(C.rows, C.cols, rp, col, val)


def _check_with(A, B):
    ref = oracle.alg1(A, B)

    def check(C, al):
        assert C.rows == A.rows and C.nnz == ref.nnz
        assert_rows_exact(_result(C, al), ref)
    return check


def _owned(C):
    return [p for p in (C.row_ptr, C.col_idx, C.val) if p]


def test_precise_every_allocation_fails_once():
    A, B = bins_matrix(seed=11)          # rows in every bin, long rows among them
    dA, dB = brm.to_device(A), brm.to_device(B)
    n = _sweep(_product_call("brm_spgemm_precise", dA, dB), _check_with(A, B), _owned)
    assert n >= 5


def test_upper_in_chunks_every_allocation_fails_once():
    A, B = bins_matrix(seed=12)
    dA, dB = brm.to_device(A), brm.to_device(B)
    _sweep(_product_call("brm_spgemm_upper", dA, dB, upper_chunk_bytes=200000), _check_with(A, B), _owned)


def test_batched_every_allocation_fails_once():
    mats = I.batched_mix(6, nmin=100, nmax=2000)
    dev = [brm.to_device(M) for M in mats]
    lib = brm.load()
    arr = brm._csr_array(dev)
    o = brm.options()
    refs = [oracle.alg1(M, M) for M in mats]

    def call(al):
        C = brm.brm_csr_out()
        off = (ctypes.c_int64 * (len(dev) + 1))()
        rc = lib.brm_spgemm_batched(len(dev), arr, arr, ctypes.byref(C), ctypes.cast(off, ctypes.c_void_p),
                                    ctypes.byref(o), ctypes.byref(al.struct), brm._stream())
        return rc, C

    def check(C, al):
        assert C.nnz == sum(r.nnz for r in refs)
        R = _result(C, al)
        off = np.cumsum([0] + [M.rows for M in mats])
        for p, ref in enumerate(refs):
            assert_rows_exact(brm.split(R, list(off), [M.cols for M in mats])[p], ref)
    _sweep(call, check, _owned)


def test_symbolic_and_backward_fail_cleanly():
    A, B = bins_matrix(seed=13)
    dA, dB = brm.to_device(A), brm.to_device(B)
    lib = brm.load()
    a, b = brm._csr_struct(dA), brm._csr_struct(dB)
    want = np.concatenate(([0], np.cumsum(oracle.symbolic(A, B))))
    rp = torch.empty(A.rows + 1, dtype=torch.int64, device="cuda")

    def sym(al):
        nnz = ctypes.c_int64(0)
        rc = lib.brm_spgemm_symbolic(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(rp.data_ptr()),
                                     ctypes.byref(nnz), ctypes.byref(brm.options()), ctypes.byref(al.struct),
                                     brm._stream())
        return rc, None

    def sym_check(_, al):
        assert np.array_equal(rp.cpu().numpy(), want)
    _sweep(sym, sym_check, lambda _: [])

    C = brm.brm_spgemm_precise(dA, dB)
    G = torch.ones(C.nnz, dtype=torch.float64, device="cuda")
    ga = torch.empty_like(dA.val)
    gb = torch.empty_like(dB.val)
    ra, rb = oracle.backward(A, B, C.rp.cpu().numpy(), C.col.cpu().numpy(), G.cpu().numpy())

    def bwd(al):
        rc = lib.brm_spgemm_backward(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(C.rp.data_ptr()),
                                     ctypes.c_void_p(C.col.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                     ctypes.c_void_p(ga.data_ptr()), ctypes.c_void_p(gb.data_ptr()), None,
                                     ctypes.byref(al.struct), brm._stream())
        return rc, None

    def bwd_check(_, al):
        assert np.array_equal(ga.cpu().numpy(), ra) and np.array_equal(gb.cpu().numpy(), rb)
    _sweep(bwd, bwd_check, lambda _: [])
