"""CPU oracle for BRMerge SpGEMM -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library under ``paper_2206_06611_gb300``
never does, and shares no code with it: the one module both sides use is
``paper_2206_06611_gb300.inputs``, which only draws matrices.

The arithmetic lives in ``brm_oracle.c`` (plain C, single-threaded, built with
``-O2 -ffp-contract=off``); this file loads it with ctypes and hands it numpy
arrays.  Functions and what pins them (tests/test_oracle_*.py):

* ``gustavson``  Eq. (2), the plain row-wise definition, in double.  Pinned by
  dense brute force on integer matrices, the closed-form square of the 2-D and
  3-D Laplacians, identity/permutation products and the transpose identity.
* ``symbolic``   Section II-B's structural row counts.  Pinned by brute force
  and the Laplacian closed form.
* ``alg1``       the BRMerge accumulation (Section III-A/B, Algorithm 1,
  Figs. 2-3): rounds that merge neighbouring lists until one is left, in
  double / float / float with TwoSum.  Pinned by the Fig. 2 round count, a hand-derived case in
  which the tree order changes the double result, equality with Gustavson on
  integer inputs and the summation error bound elsewhere.
* ``backward``   the gradients of sum(C * G).  Pinned by exact finite
  differences (the loss is linear in each operand) and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_row_nprod.argtypes = [I64, P, P, P, P, P]
        lib.orc_row_nprod.restype = None
        lib.orc_symbolic.argtypes = [I64, P, P, P, ctypes.c_int32, P, P, P]
        lib.orc_gustavson.argtypes = [I64, P, P, P, P, ctypes.c_int32, P, P, P, P, P, P, P]
        lib.orc_alg1.argtypes = [I64, P, ctypes.c_int, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_backward.argtypes = [I64, P, P, P, P, ctypes.c_int32, P, P, P, P, P, P, P, P]
        for f in (lib.orc_symbolic, lib.orc_gustavson, lib.orc_alg1, lib.orc_backward):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _rows(A, rows):
    if rows is None:
        return np.arange(A.rows, dtype=np.int64)
    return _c(rows, np.int64)


class Result:
    """Rows ``rows`` of C: crp (int64, len(rows)+1), col (int32), val (float64)."""

    def __init__(self, rows, crp, col, val, abs_=None, rounds=None):
        self.rows, self.crp, self.col, self.val, self.abs, self.rounds = rows, crp, col, val, abs_, rounds

    @property
    def nnz(self) -> int:
        return int(self.crp[-1])

    def row(self, t: int):
        a, b = int(self.crp[t]), int(self.crp[t + 1])
        return self.col[a:b], self.val[a:b]


def row_nprod(A, B, rows=None) -> np.ndarray:
    rows = _rows(A, rows)
    out = np.zeros(len(rows), dtype=np.int64)
    arp, acol, brp = _c(A.rp, np.int32), _c(A.col, np.int32), _c(B.rp, np.int32)
    _load().orc_row_nprod(len(rows), _p(rows), _p(arp), _p(acol), _p(brp), _p(out))
    return out


def symbolic(A, B, rows=None) -> np.ndarray:
    """nnz of each requested row of C = A*B (structure only)."""
    assert A.cols == B.rows
    rows = _rows(A, rows)
    out = np.zeros(len(rows), dtype=np.int64)
    arp, acol = _c(A.rp, np.int32), _c(A.col, np.int32)
    brp, bcol = _c(B.rp, np.int32), _c(B.col, np.int32)
    rc = _load().orc_symbolic(len(rows), _p(rows), _p(arp), _p(acol), B.cols, _p(brp), _p(bcol), _p(out))
    assert rc == 0, rc
    return out


def _crp(A, B, rows):
    nnz = symbolic(A, B, rows)
    crp = np.zeros(len(rows) + 1, dtype=np.int64)
    crp[1:] = np.cumsum(nnz)
    return crp


def gustavson(A, B, rows=None, with_abs: bool = False) -> Result:
    """Rows of C = A*B by Eq. (2) in double (float inputs are widened)."""
    assert A.cols == B.rows
    rows = _rows(A, rows)
    crp = _crp(A, B, rows)
    col = np.zeros(int(crp[-1]), dtype=np.int32)
    val = np.zeros(int(crp[-1]), dtype=np.float64)
    cab = np.zeros(int(crp[-1]), dtype=np.float64) if with_abs else None
    arp, acol, av = _c(A.rp, np.int32), _c(A.col, np.int32), _c(A.val, np.float64)
    brp, bcol, bv = _c(B.rp, np.int32), _c(B.col, np.int32), _c(B.val, np.float64)
    rc = _load().orc_gustavson(len(rows), _p(rows), _p(arp), _p(acol), _p(av), B.cols,
                               _p(brp), _p(bcol), _p(bv), _p(crp), _p(col), _p(val), _p(cab))
    assert rc == 0, rc
    return Result(rows, crp, col, val, cab)


PREC = {"f64": 0, "f32": 1, "f32c": 2}


def alg1(A, B, rows=None, prec: str = "f64") -> Result:
    """Rows of C by Algorithm 1.  prec: 'f64', 'f32' or 'f32c' (TwoSum)."""
    assert A.cols == B.rows
    rows = _rows(A, rows)
    crp = _crp(A, B, rows)
    col = np.zeros(int(crp[-1]), dtype=np.int32)
    val = np.zeros(int(crp[-1]), dtype=np.float64)
    rounds = np.zeros(len(rows), dtype=np.int32)
    arp, acol = _c(A.rp, np.int32), _c(A.col, np.int32)
    brp, bcol = _c(B.rp, np.int32), _c(B.col, np.int32)
    if prec == "f64":
        avd, bvd, avf, bvf = _c(A.val, np.float64), _c(B.val, np.float64), None, None
    else:
        avd, bvd, avf, bvf = None, None, _c(A.val, np.float32), _c(B.val, np.float32)
    rc = _load().orc_alg1(len(rows), _p(rows), PREC[prec], _p(arp), _p(acol), _p(avd), _p(avf),
                          _p(brp), _p(bcol), _p(bvd), _p(bvf), _p(crp), _p(col), _p(val), _p(rounds))
    assert rc == 0, rc
    return Result(rows, crp, col, val, rounds=rounds)


def backward(A, B, crp, ccol, g, rows=None, want_da=True, want_db=True):
    """(dA values on A's pattern, dB values on B's pattern) of sum(C * G), double.

    ``crp``/``ccol``/``g``: C's pattern and G for the listed rows (all rows by
    default; dB is complete only then).  dA entries of unlisted rows stay 0.
    """
    rows = _rows(A, rows)
    arp, acol, av = _c(A.rp, np.int32), _c(A.col, np.int32), _c(A.val, np.float64)
    brp, bcol, bv = _c(B.rp, np.int32), _c(B.col, np.int32), _c(B.val, np.float64)
    crp, ccol, g = _c(crp, np.int64), _c(ccol, np.int32), _c(g, np.float64)
    da = np.zeros(A.nnz, dtype=np.float64) if want_da else None
    db = np.zeros(B.nnz, dtype=np.float64) if want_db else None
    rc = _load().orc_backward(len(rows), _p(rows), _p(arp), _p(acol), _p(av), B.cols, _p(brp),
                              _p(bcol), _p(bv), _p(crp), _p(ccol), _p(g), _p(da), _p(db))
    assert rc == 0, rc
    return da, db


def balanced_row_groups(nprod: np.ndarray, p: int):
    """The paper's static split (Section III-D): p contiguous row groups of
    about equal total nprod.  Returns p+1 row boundaries."""
    cum = np.concatenate(([0], np.cumsum(nprod, dtype=np.int64)))
    total = int(cum[-1])
    bounds = [0]
    for g in range(1, p):
        bounds.append(int(np.searchsorted(cum, total * g // p, side="left")))
    bounds.append(len(nprod))
    return np.maximum.accumulate(np.array(bounds, dtype=np.int64))


def _split_rows(A, B, rows, threads):
    rows = _rows(A, rows)
    threads = max(1, min(int(threads or os.cpu_count() or 1), max(len(rows), 1)))
    bounds = balanced_row_groups(row_nprod(A, B, rows), threads)
    return rows, bounds, [rows[bounds[t]:bounds[t + 1]] for t in range(threads)]


def _join(rows, bounds, res) -> Result:
    crp = np.zeros(len(rows) + 1, dtype=np.int64)
    off = 0
    for t, r in enumerate(res):
        crp[bounds[t]:bounds[t + 1] + 1] = r.crp + off
        off += r.nnz
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)  # noqa: E731
    abs_ = cat([r.abs for r in res]) if all(r.abs is not None for r in res) else None
    rounds = cat([r.rounds for r in res]).astype(np.int32) if all(r.rounds is not None for r in res) else None
    return Result(rows, crp, cat([r.col for r in res]).astype(np.int32), cat([r.val for r in res]), abs_, rounds)


def _pool_map(fn, parts):
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(parts)) as ex:
        return list(ex.map(fn, parts))


def gustavson_parallel(A, B, threads: int, rows=None, with_abs: bool = False) -> Result:
    """Gustavson on ``threads`` host threads over nprod-balanced row groups
    (ctypes drops the GIL during each C call).  Same results as gustavson()."""
    rows, bounds, parts = _split_rows(A, B, rows, threads)
    return _join(rows, bounds, _pool_map(lambda r: gustavson(A, B, r, with_abs), parts))


def alg1_parallel(A, B, rows=None, prec: str = "f64", threads: int | None = None) -> Result:
    """alg1() with the rows spread over host threads (each row is computed
    by one call of the same single-threaded code; only the rows are split)."""
    rows, bounds, parts = _split_rows(A, B, rows, threads)
    return _join(rows, bounds, _pool_map(lambda r: alg1(A, B, r, prec), parts))


def symbolic_parallel(A, B, rows=None, threads: int | None = None) -> np.ndarray:
    """symbolic() with the rows spread over host threads."""
    rows, bounds, parts = _split_rows(A, B, rows, threads)
    res = _pool_map(lambda r: symbolic(A, B, r), parts)
    return np.concatenate(res) if res else np.zeros(0, np.int64)
