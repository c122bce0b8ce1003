"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/brm.h declares, and its host-side argument checks answer
without touching a GPU (no compute call is made here)."""
import ctypes

import pytest

from paper_2206_06611_gb300 import brm


@pytest.fixture(scope="module")
def lib():
    return brm.load()


def test_header_declares_the_entry_points():
    names = brm.declared_symbols()
    for want in ("brm_spgemm_symbolic", "brm_spgemm_precise", "brm_spgemm_upper", "brm_row_nprod",
                 "brm_csr_out_free", "brm_options_default", "brm_last_error", "brm_version",
                 "brm_trace_enable", "brm_trace_read", "brm_kernel_launches", "brm_spgemm_backward",
                 "brm_spgemm_numeric_noalloc"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in brm.declared_symbols():
        assert hasattr(lib, name), name


def test_options_default(lib):
    o = brm.brm_options()
    lib.brm_options_default(ctypes.byref(o))
    assert o.validate == 0 and o.compensated == 0
    assert o.warp_max_nprod == 256 and o.block_max_nprod == 4096 and o.arena_bytes == 0
    assert b"sm_103a" in lib.brm_version()


def _csr(rows, cols, nnz=0, dtype=brm.BRM_F64, rp=1, col=1, val=1):
    # non-NULL dummy pointers: the checks below fail before anything is read
    return brm.brm_csr(rows, cols, nnz, rp and 0x1000, col and 0x1000, val and 0x1000, dtype)


def _precise(lib, A, B):
    C = brm.brm_csr_out()
    rc = lib.brm_spgemm_precise(ctypes.byref(A) if A is not None else None, ctypes.byref(B), ctypes.byref(C),
                                None, None, None)
    return rc, lib.brm_last_error().decode(), C


def test_host_argument_checks(lib):
    rc, msg, C = _precise(lib, None, _csr(3, 3))
    assert rc == -1 and "A is NULL" in msg and C.row_ptr is None
    rc, msg, _ = _precise(lib, _csr(3, 4), _csr(5, 3))
    assert rc == -2 and "4" in msg and "5" in msg
    rc, msg, _ = _precise(lib, _csr(3, 3, dtype=7), _csr(3, 3))
    assert rc == -3
    rc, msg, _ = _precise(lib, _csr(3, 3, dtype=brm.BRM_F32), _csr(3, 3, dtype=brm.BRM_F64))
    assert rc == -3 and "different" in msg
    rc, msg, _ = _precise(lib, _csr(-1, 3), _csr(3, 3))
    assert rc == -1
    rc, msg, _ = _precise(lib, _csr(3, 3, nnz=5, val=0), _csr(3, 3))
    assert rc == -1 and "val" in msg
    rc, msg, _ = _precise(lib, _csr(3, 1 << 31), _csr(1 << 31, 3))
    assert rc == -5
    # the symbolic pass does not need values
    nnz = ctypes.c_int64(0)
    rc = lib.brm_spgemm_symbolic(ctypes.byref(_csr(3, 4, val=0)), ctypes.byref(_csr(5, 3, val=0)),
                                 ctypes.c_void_p(0x1000), ctypes.byref(nnz), None, None, None)
    assert rc == -2
    rc = lib.brm_spgemm_symbolic(ctypes.byref(_csr(3, 3, val=0)), ctypes.byref(_csr(3, 3, val=0)),
                                 None, ctypes.byref(nnz), None, None, None)
    assert rc == -1


def test_trace_api_without_gpu(lib):
    n = lib.brm_trace_read(None, None, 0)
    names = [lib.brm_trace_phase_name(i).decode() for i in range(n)]
    assert names[0] == "validate" and "numeric_reg" in names and "numeric_warp" in names
    assert names[-4:] == ["compact", "backward", "symbolic_tile", "numeric_tile"]
    assert lib.brm_trace_phase_name(99) == b""
    was = lib.brm_trace_enable(1)
    assert lib.brm_trace_enable(was) == 1
    assert lib.brm_kernel_launches() >= 0
