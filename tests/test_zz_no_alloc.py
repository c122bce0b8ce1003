"""The numeric pass that allocates no device memory (brm_spgemm_numeric_noalloc).

That entry point serves callers that cannot allocate device memory at all:
an application whose own pool owns the whole GPU, a latency-bound loop that
must not take an allocation's implicit synchronisation, or a plug-in that may
only write the buffers it is given.  Its workspace is a fixed array inside
libbrm, shared by every call, so these checks call it twice in a row on
different products -- a result that leaked state from the previous call
would show -- and compare each result bit for bit with the CPU oracle's
BRMerge rounds (Algorithm 1 in the same precision) and with
brm_spgemm_precise (the same kernels with allocated workspace).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_rows_exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402


def _noalloc_like_precise(A, B, dtype=np.float64, compensated=False):
    prec = "f64" if dtype == np.float64 else ("f32c" if compensated else "f32")
    ref = oracle.alg1(A, B, prec=prec)
    dA, dB = brm.to_device(A, dtype=dtype), brm.to_device(B, dtype=dtype)
    want = brm.brm_spgemm_precise(dA, dB, compensated=compensated)
    torch.cuda.synchronize()
    # caller-owned outputs, filled with garbage that must all be overwritten
    rp = want.rp.clone()
    col = torch.full_like(want.col, -7)
    val = torch.full_like(want.val, float("nan"))
    got = brm.brm_spgemm_numeric_noalloc(dA, dB, rp, col, val, compensated=compensated)
    torch.cuda.synchronize()
    assert torch.equal(got.rp, want.rp)
    assert torch.equal(got.col, want.col)
    assert torch.equal(got.val, want.val)
    assert_rows_exact(got, ref)
    return got


def test_noalloc_matches_precise_on_two_calls_in_a_row():
    # call 1: Erdos-Renyi rows (all in the warp bin); call 2: a product with
    # rows in both shared-memory bins and empty rows, so the second call's
    # row lists and counts differ from what the array still holds
    A = I.erdos_renyi(20000, 16, seed=21)
    _noalloc_like_precise(A, A)
    B = I.erdos_renyi(500, 60, seed=23, ncols=4000)
    _noalloc_like_precise(_stack([I.erdos_renyi(1500, 40, seed=22, ncols=500),     # block bin
                                  I.CSR(300, 500, np.zeros(301, np.int32), np.zeros(0, np.int32),
                                        np.zeros(0)),                               # empty rows
                                  I.erdos_renyi(1500, 3, seed=24, ncols=500)]), B)  # warp bin


def _stack(parts):
    """Rows of the parts one after the other (same column count)."""
    rp = [np.zeros(1, np.int64)]
    for P in parts:
        rp.append(P.rp[1:].astype(np.int64) + rp[-1][-1])
    return I.CSR(sum(P.rows for P in parts), parts[0].cols, np.concatenate(rp).astype(np.int32),
                 np.concatenate([P.col for P in parts]), np.concatenate([P.val for P in parts]))


def test_noalloc_float_modes():
    A = I.erdos_renyi(5000, 12, seed=24)
    _noalloc_like_precise(A, A, np.float32, False)
    _noalloc_like_precise(A, A, np.float32, True)


def test_noalloc_rejects_rows_beyond_its_limits():
    # more rows than the fixed workspace holds: refused before any GPU work
    dA = brm.to_device(I.identity(4))
    big, small = brm._csr_struct(dA), brm._csr_struct(dA)
    big.rows = (1 << 20) + 1          # A: too many rows; B: the 4 x 4 identity
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    lib = brm.load()
    rc = lib.brm_spgemm_numeric_noalloc(ctypes.byref(big), ctypes.byref(small), ctypes.c_void_p(one.data_ptr()),
                                        ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()), None,
                                        brm._stream())
    assert rc == -5 and b"at most" in lib.brm_last_error()
    # a row too long for the shared-memory bins: refused, C left untouched
    A = I.erdos_renyi(8, 200, seed=25, ncols=400)
    B = I.erdos_renyi(400, 100, seed=26, ncols=5000)
    dA, dB = brm.to_device(A), brm.to_device(B)
    rp, nnz = brm.brm_spgemm_symbolic(dA, dB)
    col = torch.full((nnz,), -7, dtype=torch.int32, device="cuda")
    val = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(brm.BrmError) as e:
        brm.brm_spgemm_numeric_noalloc(dA, dB, rp, col, val)
    assert e.value.code == -5
    assert bool((col == -7).all())


def test_noalloc_rejects_a_slot_for_an_empty_row():
    """A row pointer that gives a row without products a slot of one entry
    (every later row shifted by one): the call fails with BRM_ERR_INVALID."""
    A = I.erdos_renyi(300, 5, seed=27, ncols=200)
    Z = I.CSR(5, 200, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    A = _stack([A, Z, I.erdos_renyi(40, 5, seed=28, ncols=200)])
    B = I.erdos_renyi(200, 6, seed=29, ncols=700)
    dA, dB = brm.to_device(A), brm.to_device(B)
    rp, nnz = brm.brm_spgemm_symbolic(dA, dB)
    empty_row = 302
    assert int(rp[empty_row + 1] - rp[empty_row]) == 0
    bad = rp.clone()
    bad[empty_row + 1:] += 1
    col = torch.zeros(nnz + 1, dtype=torch.int32, device="cuda")
    val = torch.zeros(nnz + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(brm.BrmError) as e:
        brm.brm_spgemm_numeric_noalloc(dA, dB, bad, col, val)
    assert e.value.code == -1
    # the same arrays with the right row pointer: accepted, the oracle's result
    got = brm.brm_spgemm_numeric_noalloc(dA, dB, rp, col[:nnz], val[:nnz])
    torch.cuda.synchronize()
    assert_rows_exact(got, oracle.alg1(A, B))
