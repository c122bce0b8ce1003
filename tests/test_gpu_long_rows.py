"""Long rows (more products than a thread block merges in shared memory).

The symbolic pass counts a long row's columns in a shared-memory bitmap; the
numeric pass merges it by rounds through the device-memory arena (default) or,
with option long_bucket, by column buckets: the row's products are scattered
to column cells and every column is reduced in the merge tree's order.  Both
numeric kernels must give the same bits as each other and as the oracle's
Algorithm 1.
The cases reach every branch of the bucket kernels: units of several cells,
runs reduced by one lane and by a whole warp, cells of more than 256 products
split again by column (the work list), and columns of more than 256 products
reduced over one slot per list, at both levels; also B wider than one bitmap
window and rows beyond the 65535-list limit (merge rounds).
"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

from helpers import assert_close_to_gustavson, assert_rows_exact, bins_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_06611_gb300 import brm  # noqa: E402

MODES = [("f64", np.float64, False), ("f32", np.float32, False), ("f32c", np.float32, True)]


def run(A, B, method="precise", dtype=np.float64, compensated=False, **kw):
    kw.setdefault("long_bucket", True)
    dA, dB = brm.to_device(A, dtype=dtype), brm.to_device(B, dtype=dtype)
    f = brm.brm_spgemm_precise if method == "precise" else brm.brm_spgemm_upper
    C = f(dA, dB, compensated=compensated, **kw)
    torch.cuda.synchronize()
    return C


def same(C1, C2):
    assert torch.equal(C1.rp, C2.rp)
    assert torch.equal(C1.col, C2.col)
    assert torch.equal(C1.val, C2.val)


def csr_from_rows(rows, ncols, seed, stream):
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    assert rp[-1] < 2 ** 31
    col = np.concatenate([np.asarray(r, np.int64) for r in rows]).astype(np.int32) if rp[-1] else \
        np.zeros(0, np.int32)
    return I.CSR(len(rows), ncols, rp.astype(np.int32), col, I.rand_sym(seed, stream, np.arange(len(col))))


def hot_b(k, ncols, seed, hot_cols, hot_p, spread):
    """k rows of B: each holds column hot_cols[i] with probability hot_p[i]
    and `spread` random columns over [0, ncols)."""
    hc = np.asarray(hot_cols, np.int64)
    take = np.stack([I.rand_unit(seed, 40 + i, np.arange(k)) < p for i, p in enumerate(hot_p)], axis=1) \
        if len(hot_cols) else np.zeros((k, 0), bool)
    rnd = (I.rand_u64(seed, 60, np.arange(k * spread)) % np.uint64(ncols)).astype(np.int64).reshape(k, spread)
    rows = [np.unique(np.concatenate([hc[take[r]], rnd[r]])) for r in range(k)]
    return csr_from_rows(rows, ncols, seed, 61)


def rows_of_a(Ls, k, seed):
    rows = []
    for t, L in enumerate(Ls):
        if L >= k:
            rows.append(np.arange(k))
            continue
        u = I.rand_u64(seed, 70 + t, np.arange(4 * L + 64)) % np.uint64(k)
        _, idx = np.unique(u, return_index=True)
        rows.append(np.sort(u[np.sort(idx)][:L].astype(np.int64)))
    return csr_from_rows(rows, k, seed, 71)


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_bucket_matches_merge_rounds(mode, dtype, comp):
    """Rows of every bin and R-MAT scale 14: the bucket kernels give the bits
    of the merge rounds and of the oracle's Algorithm 1."""
    A, B = bins_matrix(seed=6)
    ref = oracle.alg1(A, B, prec=mode)
    Cb = run(A, B, "precise", dtype, comp)
    assert_rows_exact(Cb, ref)
    same(Cb, run(A, B, "precise", dtype, comp, long_bucket=False))
    same(Cb, run(A, B, "upper", dtype, comp))
    R = I.rmat(14, 16, seed=81)
    Cr = run(R, R, "precise", dtype, comp)
    same(Cr, run(R, R, "precise", dtype, comp, long_bucket=False))
    nprod = oracle.row_nprod(R, R)
    rows = np.argsort(-nprod, kind="stable")[:60]
    assert_rows_exact(Cr, oracle.alg1(R, R, np.sort(rows), prec=mode), np.sort(rows))


@pytest.mark.parametrize("mode,dtype,comp", MODES)
@pytest.mark.parametrize("ncols", [4096, 1 << 20])
def test_hot_cells_and_giant_columns(mode, dtype, comp, ncols):
    """Rows whose columns 0..3 sit in most lists (runs of up to 65535
    products), a cell of a few hundred warm columns, and a spread of cold
    ones.  With 4096 columns every cell is one column (giant columns at the
    first level); with 2^20 the cells hold 256 columns and the hot cell is
    split again by column."""
    k = 70000
    hot_cols = [0, 1, 2, 3] + list(range(16, 200, 3))
    hot_p = [0.97, 0.5, 0.08, 0.03] + [0.01] * (len(hot_cols) - 4)
    B = hot_b(k, ncols, 91, hot_cols, hot_p, 3)
    A = rows_of_a([65535, 20000, 5000, 4500, 3000, 600, 1], k, 92)
    ref = oracle.alg1(A, B, prec=mode)
    C = run(A, B, "precise", dtype, comp)
    assert_rows_exact(C, ref)
    same(C, run(A, B, "precise", dtype, comp, long_bucket=False))
    same(C, run(A, B, "upper", dtype, comp))
    if mode == "f64":
        assert_close_to_gustavson(C, A, B)


def test_single_column_and_single_list_rows():
    """Degenerate long rows: every list holds the same one column (a single
    giant run), one list of 10000 products (no duplicates), two lists that
    are identical (every run has two products)."""
    k, ncols = 12000, 300000
    one = [np.array([777])] * 9000
    wide = [np.arange(0, 300000, 30)]
    pair = [np.arange(5, 300000, 50)] * 2
    B = csr_from_rows(one + wide + pair + [np.array([1, 2])] * (k - 9003), ncols, 93, 1)
    A = csr_from_rows([np.arange(9000), np.array([9000]), np.array([9001, 9002]), np.arange(8990, 9003)],
                      k, 94, 2)
    ref = oracle.alg1(A, B)
    C = run(A, B)
    assert_rows_exact(C, ref)
    same(C, run(A, B, long_bucket=False))


def test_wide_B_several_bitmap_windows():
    """B with 3 * 2^20 + 5 columns: the symbolic bitmap takes four windows and
    the cells hold 1024 columns each."""
    k, ncols = 3000, 3 * (1 << 20) + 5
    B = hot_b(k, ncols, 95, [0, ncols - 1, 1 << 20, (1 << 21) + 3], [0.9, 0.9, 0.5, 0.2], 20)
    A = rows_of_a([2999, 1500, 700, 300], k, 96)
    ref = oracle.alg1(A, B)
    C = run(A, B)
    assert_rows_exact(C, ref)
    same(C, run(A, B, long_bucket=False))


def test_list_limit_uses_merge_rounds():
    """A row of 70000 lists is beyond the bucket kernel's 16-bit list index:
    the pass keeps the merge rounds, with the same result."""
    k, ncols = 70000, 50000
    B = hot_b(k, ncols, 97, [10, 11], [0.3, 0.3], 2)
    A = rows_of_a([70000, 5000, 10], k, 98)
    ref = oracle.alg1(A, B)
    C = run(A, B)
    assert_rows_exact(C, ref)
    same(C, run(A, B, long_bucket=False))


def test_batched_long_rows():
    """Two products with long rows in one batched call (the bucket kernel
    finds each row's A and B through the product table)."""
    k = 20000
    B1 = hot_b(k, 1 << 18, 99, [0, 7], [0.9, 0.4], 4)
    A1 = rows_of_a([15000, 4000, 100, 0, 2], k, 100)
    B2 = hot_b(k, 5000, 101, [3], [0.8], 6)
    A2 = rows_of_a([3, 19999, 8000], k, 102)
    C, off = brm.brm_spgemm_batched([brm.to_device(A1), brm.to_device(A2)], [brm.to_device(B1), brm.to_device(B2)],
                                    long_bucket=True)
    torch.cuda.synchronize()
    for Cp, (A, B) in zip(brm.split(C, off, [B1.cols, B2.cols]), [(A1, B1), (A2, B2)]):
        assert_rows_exact(Cp, oracle.alg1(A, B))


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_arena_rounds_many_tiles_and_empty_pairs(mode, dtype, comp):
    """The merge rounds in the arena, tile by tile: a row of 1.2 M products
    (more than 512 tiles in its first rounds, so the tile cuts are found in
    two chunks) and a row of 57000 lists, nearly all empty (a tile spans more
    pairs than it stages list offsets for)."""
    k, ncols = 60000, 50000
    rnd = (I.rand_u64(103, 1, np.arange(3000 * 400)) % np.uint64(ncols)).astype(np.int64).reshape(3000, 400)
    rows = [np.unique(r) for r in rnd]
    rows += [np.arange(t % 97, ncols, 1000) if t % 1000 == 0 else np.zeros(0, np.int64) for t in range(3000, k)]
    B = csr_from_rows(rows, ncols, 104, 1)
    A = csr_from_rows([np.arange(3000), np.arange(3000, k), np.array([5, 3000, 4000, 59000])], k, 105, 2)
    ref = oracle.alg1(A, B, prec=mode)
    C = run(A, B, "precise", dtype, comp, long_bucket=False, long_window=False)
    assert_rows_exact(C, ref)
    same(C, run(A, B, "upper", dtype, comp, long_bucket=False, long_window=False))


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_persistent_blocks_share_arena_slots(mode, dtype, comp):
    """R-MAT scale 14: thousands of long rows on fewer persistent blocks, each
    reusing its arena slot for row after row; with an arena budget of one
    byte a single block merges them all.  Same bits as the default run and as
    the oracle on the largest rows."""
    R = I.rmat(14, 16, seed=83)
    C = run(R, R, "precise", dtype, comp, long_bucket=False, long_window=False)
    same(C, run(R, R, "precise", dtype, comp, long_bucket=False, long_window=False, arena_bytes=1))
    same(C, run(R, R, "upper", dtype, comp, long_bucket=False, long_window=False, arena_bytes=1 << 20))
    nprod = oracle.row_nprod(R, R)
    rows = np.sort(np.argsort(-nprod, kind="stable")[:40])
    assert_rows_exact(C, oracle.alg1(R, R, rows, prec=mode), rows)
