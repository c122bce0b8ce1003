"""Long rows by column tiles (option long_window).

By default (long_window 1) the long rows of at least 65536 products and at
most 2048 lists take the tiles and the others the merge rounds; with
long_window 2 (the tests' default here) every long row of at most 65535
lists takes them.  A long row is cut into column tiles of at most 2048
products planned from the symbolic pass's bitmap and per-cell product
histogram; every tile's products are sorted by column in shared memory (a
stable radix sort that keeps list order) and Algorithm 1's merge rounds run
on the sorted positions; a single crowded cell of more than 2048 products is
taken in chunks of aligned list blocks, every column's chunk sums carried
between them.  Lists are searched in blocks of 2048 (rows of more lists keep
their cursors in device memory).  Rows of more than 65535 lists keep the
merge rounds in the same pass.  The result must be the merge rounds' bits and
the oracle's Algorithm 1 in every precision.  The cases reach: tiles of many
cells and of one cell, hot cells of several crowded columns (many chunks,
several list blocks), a single run of 2048 products, rows of up to 20000
lists, spans of several tiles, B wider than one bitmap window of 2^20
columns, rows past the 65535-list limit (merge rounds instead, alone and
mixed with tiled rows), BRMerge-Upper (the plan made in the numeric pass),
batched products and a prepared batch replayed from a CUDA graph.
"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_close_to_gustavson, assert_rows_exact, bins_matrix
from test_gpu_long_rows import csr_from_rows, hot_b, rows_of_a

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402

MODES = [("f64", np.float64, False), ("f32", np.float32, False), ("f32c", np.float32, True)]


def run(A, B, method="precise", dtype=np.float64, compensated=False, **kw):
    kw.setdefault("long_window", True)
    dA, dB = brm.to_device(A, dtype=dtype), brm.to_device(B, dtype=dtype)
    f = brm.brm_spgemm_precise if method == "precise" else brm.brm_spgemm_upper
    C = f(dA, dB, compensated=compensated, **kw)
    torch.cuda.synchronize()
    return C


def same(C1, C2):
    assert torch.equal(C1.rp, C2.rp)
    assert torch.equal(C1.col, C2.col)
    assert torch.equal(C1.val, C2.val)


def long_trace(A, B, **kw):
    """Launches of the long rows' symbolic and numeric passes (tiles and merge
    rounds) in one Precise call."""
    brm.brm_trace_reset()
    was = brm.brm_trace_enable(True)
    run(A, B, **kw)
    t = brm.brm_trace_read()
    brm.brm_trace_enable(was)
    return (t["symbolic_long"][1] + t["symbolic_tile"][1], t["numeric_long"][1] + t["numeric_tile"][1])


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_tiles_match_rounds_and_oracle(mode, dtype, comp):
    A, B = bins_matrix(seed=7)
    ref = oracle.alg1(A, B, prec=mode)
    Cw = run(A, B, "precise", dtype, comp)
    assert_rows_exact(Cw, ref)
    same(Cw, run(A, B, "precise", dtype, comp, long_window=False))
    same(Cw, run(A, B, "upper", dtype, comp))
    R = I.rmat(15, 16, seed=84)
    Cr = run(R, R, "precise", dtype, comp)
    same(Cr, run(R, R, "precise", dtype, comp, long_window=False))
    same(Cr, run(R, R, "upper", dtype, comp))
    nprod = oracle.row_nprod(R, R)
    rows = np.sort(np.argsort(-nprod, kind="stable")[:50])
    assert_rows_exact(Cr, oracle.alg1(R, R, rows, prec=mode), rows)
    if mode == "f64":
        assert_close_to_gustavson(Cr, R, R, rows)


def test_tiles_are_taken():
    """With long_window the long rows run as the plan (symbolic pass) and one
    tile launch (numeric pass)."""
    R = I.rmat(12, 16, seed=85)
    assert long_trace(R, R) == (1, 1)
    sym, num = long_trace(R, R, long_window=False)
    assert sym == 1 and num >= 1


def test_default_split():
    """The default options (long_window 1) send the long rows of at least
    65536 products and at most 2048 lists to the tiles and the others to the
    merge rounds, in the same passes, with the merge rounds' bits."""
    R = I.rmat(16, 16, seed=86)
    nprod = oracle.row_nprod(R, R)
    L = np.diff(R.rp)
    long = (nprod > 4096) | (L > 1024)
    assert (long & (nprod >= 65536) & (L <= 2048)).any() and (long & (nprod < 65536)).any()
    dR = brm.to_device(R)
    brm.brm_trace_reset()
    was = brm.brm_trace_enable(True)
    C = brm.brm_spgemm_precise(dR, dR)
    torch.cuda.synchronize()
    t = brm.brm_trace_read()
    brm.brm_trace_enable(was)
    assert t["symbolic_tile"][1] == 1 and t["numeric_tile"][1] == 1
    assert t["symbolic_long"][1] == 1 and t["numeric_long"][1] >= 1
    same(C, run(R, R, long_window=False))
    rows = np.sort(np.argsort(-nprod, kind="stable")[:20])
    assert_rows_exact(C, oracle.alg1(R, R, rows), rows)


@pytest.mark.parametrize("mode,dtype,comp", MODES)
@pytest.mark.parametrize("ncols", [4096, 1 << 20])
def test_hot_cells(mode, dtype, comp, ncols):
    """Columns 0..3 in most of up to 20000 lists: with 2^20 columns (cells of
    128) they share one cell of up to ~63000 products, taken in chunks of
    aligned list blocks, block after block of 2048 lists; with 4096 columns
    every cell is one column wide, a tile of up to 2048 products or, past 2048
    lists, a hot one.  A cell of warm columns, cold columns spread wide."""
    k = 70000
    hot_cols = [0, 1, 2, 3] + list(range(16, 200, 3))
    hot_p = [0.97, 0.9, 0.8, 0.5] + [0.01] * (len(hot_cols) - 4)
    B = hot_b(k, ncols, 91, hot_cols, hot_p, 3)
    A = rows_of_a([20000, 5000, 2048, 2047, 1025, 600, 1], k, 92)
    ref = oracle.alg1(A, B, prec=mode)
    C = run(A, B, "precise", dtype, comp)
    assert_rows_exact(C, ref)
    same(C, run(A, B, "upper", dtype, comp))
    if mode == "f64":
        same(C, run(A, B, "precise", dtype, comp, long_window=False))
        assert_close_to_gustavson(C, A, B)


def test_tiles_degenerate_rows():
    """Every list the same one column (one run of 2048 products), 1096 of
    them and 949 lists of five columns of the same cell (a hot tile of 5841
    products), one list of 10000 products, two identical lists, a row of
    2000 lists of which only one is not empty, and a row of 2049 lists (two
    list blocks)."""
    k, ncols = 6000, 300000
    one = [np.array([777])] * 2048
    wide = [np.arange(0, 300000, 30)]
    pair = [np.arange(5, 300000, 50)] * 2
    B = csr_from_rows(one + wide + pair + [np.arange(775, 780)] * 949 + [np.zeros(0, np.int64)] * 3000, ncols, 93, 1)
    assert B.rows == k
    A = csr_from_rows([np.arange(2048), np.concatenate([np.arange(1096), np.arange(2051, 3000)]), np.array([2048]),
                       np.array([2049, 2050]), np.arange(2040, 2051),
                       np.concatenate([np.arange(2048, 2049), np.arange(k - 1999, k)]), np.arange(1000, 3049)],
                      k, 94, 2)
    ref = oracle.alg1(A, B)
    for kw in ({}, {"long_window": False}):
        assert_rows_exact(run(A, B, **kw), ref)
    assert_rows_exact(run(A, B, "upper"), ref)


def test_tiles_wide_B_several_bitmap_windows():
    """B with 3 * 2^20 + 5 columns: the plan takes four bitmap windows (cells
    of 128 columns), some rows have no product in some of them."""
    k, ncols = 3000, 3 * (1 << 20) + 5
    B = hot_b(k, ncols, 95, [0, ncols - 1, 1 << 20, (1 << 21) + 3], [0.9, 0.9, 0.5, 0.2], 20)
    Bl = csr_from_rows([np.array([5, 1 << 21, ncols - 2])] * 40 + [np.zeros(0, np.int64)] * (k - 40), ncols, 106, 1)
    A = rows_of_a([2999, 1500, 700, 300], k, 96)
    ref = oracle.alg1(A, B)
    C = run(A, B)
    assert_rows_exact(C, ref)
    same(C, run(A, B, long_window=False))
    A2 = csr_from_rows([np.arange(40)] * 3 + [np.arange(2000)], k, 107, 2)
    assert_rows_exact(run(A2, Bl), oracle.alg1(A2, Bl))


def test_tiles_list_limit_uses_merge_rounds():
    """Rows of more than 65535 lists keep the merge rounds: alone (one
    symbolic launch, the column bitmap), and mixed with tiled rows in the
    same passes (the plan and the bitmap, the tiles and the rounds)."""
    k, ncols = 70000, 50000
    B = hot_b(k, ncols, 97, [10, 11], [0.3, 0.3], 2)
    A = rows_of_a([70000, 69999, 10], k, 98)
    assert_rows_exact(run(A, B), oracle.alg1(A, B))
    sym, num = long_trace(A, B)
    assert sym == 1 and num >= 1
    A2 = rows_of_a([70000, 2049, 2048, 4000, 1500, 300], k, 108)
    ref = oracle.alg1(A2, B)
    C = run(A2, B)
    assert_rows_exact(C, ref)
    same(C, run(A2, B, long_window=False))
    assert_rows_exact(run(A2, B, "upper"), ref)
    sym, num = long_trace(A2, B)
    assert sym == 2 and num >= 2


def test_tiles_batched_and_graph_replay():
    """Long rows of two products in one batched call, and a prepared batch
    whose numeric pass (the window kernel among its launches) is replayed
    from a CUDA graph on new values."""
    k = 20000
    B1 = hot_b(k, 1 << 18, 99, [0, 7], [0.9, 0.4], 4)
    A1 = rows_of_a([15000, 4000, 100, 0, 2], k, 100)
    B2 = hot_b(k, 5000, 101, [3], [0.8], 6)
    A2 = rows_of_a([3, 19999, 8000], k, 102)
    dev = [brm.to_device(M) for M in (A1, A2, B1, B2)]
    C, off = brm.brm_spgemm_batched(dev[:2], dev[2:], long_window=True)
    torch.cuda.synchronize()
    for Cp, (A, B) in zip(brm.split(C, off, [B1.cols, B2.cols]), [(A1, B1), (A2, B2)]):
        assert_rows_exact(Cp, oracle.alg1(A, B))
    b = brm.Batch(dev[:2], dev[2:], long_window=True)
    for round_ in range(3):
        new = []
        for i, (M, D) in enumerate(zip((A1, A2), dev[:2])):
            v = I.rand_sym(120 + round_, i, np.arange(M.nnz))
            D.val.copy_(torch.from_numpy(v))
            new.append(I.CSR(M.rows, M.cols, M.rp, M.col, v))
        if round_ == 0:
            b.numeric()
        else:
            b.graph_launch()
        b.check()
        Cb, offb = b.result()
        for Cp, (A, B) in zip(brm.split(Cb, offb, [B1.cols, B2.cols]), [(new[0], B1), (new[1], B2)]):
            assert_rows_exact(Cp, oracle.alg1(A, B))
    b.close()
