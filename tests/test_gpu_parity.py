"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Criteria:
* structure (row_ptr, col_idx): bit-exact everywhere;
* FP64 values: bit-exact against the oracle's step-by-step Algorithm 1 (the
  kernels merge the same pairs in the same tree and never fuse a multiply-add)
  and within 1e-12 per row (normwise, scaled by |A||B|) of Gustavson's Eq. (2);
* integer-valued inputs: bit-exact against Gustavson as well;
* FP32 and FP32-with-TwoSum values: bit-exact against the oracle's Algorithm 1
  in the same precision;
* BRMerge-Upper and BRMerge-Precise: identical results.
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
    dA, dB = brm.to_device(A, dtype=dtype), brm.to_device(B, dtype=dtype)
    f = brm.brm_spgemm_precise if method == "precise" else brm.brm_spgemm_upper
    C = f(dA, dB, compensated=compensated, **kw)
    torch.cuda.synchronize()
    return C


def same(C1, C2):
    assert torch.equal(C1.rp, C2.rp)
    assert torch.equal(C1.col, C2.col)
    assert torch.equal(C1.val, C2.val)


# --------------------------------------------------------------------------
# the 64 x 64 Laplacian (integer values: any order gives the exact result)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["precise", "upper"])
def test_lap2d_exact(method):
    A = I.lap2d(64)
    C = run(A, A, method)
    assert C.nnz == 51972
    ref = oracle.gustavson(A, A)
    assert_rows_exact(C, ref)
    assert_rows_exact(C, oracle.alg1(A, A))


def test_lap3d_exact():
    A = I.lap3d(9)
    C = run(A, A)
    assert_rows_exact(C, oracle.gustavson(A, A))


# --------------------------------------------------------------------------
# small random matrices, several tiles and ragged tails, every precision mode
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,k,n,da,db,seed", [
    (1, 1, 1, 1.0, 1.0, 1), (7, 1, 5, 0.6, 0.6, 2), (5, 9, 1, 0.5, 0.7, 3), (40, 60, 50, 0.3, 0.2, 4),
    (64, 300, 200, 0.2, 0.1, 5), (33, 500, 400, 0.5, 0.05, 6), (20, 20, 20, 0.0, 0.5, 7), (20, 20, 20, 0.4, 0.0, 8),
])
def test_random_integer_exact(m, k, n, da, db, seed):
    A = I.random_int(m, k, da, seed, 0)
    B = I.random_int(k, n, db, seed, 1)
    ref = oracle.gustavson(A, B)
    for method in ("precise", "upper"):
        assert_rows_exact(run(A, B, method), ref)


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_bins_all_modes_exact(mode, dtype, comp):
    """Rows in every bin (empty, warp, block, long by products and by list
    count, many empty lists, duplicate-heavy) against Algorithm 1."""
    A, B = bins_matrix()
    ref = oracle.alg1(A, B, prec=mode)
    Cp = run(A, B, "precise", dtype, comp)
    assert_rows_exact(Cp, ref)
    Cu = run(A, B, "upper", dtype, comp)
    same(Cp, Cu)
    if mode == "f64":
        assert_close_to_gustavson(Cp, A, B)


def test_bins_small_thresholds():
    """The same rows through other bins: register bins limited or off, tiny
    warp / block capacities."""
    A, B = bins_matrix(seed=4)
    ref = oracle.alg1(A, B)
    for rcap, wcap, bcap in ((-1, 8, 64), (-1, 32, 32), (-1, 1, 2), (64, 0, 0), (256, 0, 0), (-1, 0, 0)):
        assert_rows_exact(run(A, B, reg_max_nprod=rcap, warp_max_nprod=wcap, block_max_nprod=bcap), ref)
    for keys in (8, 16, 32):
        for sym_hash in (False, True):
            assert_rows_exact(run(A, B, reg_keys=keys, symbolic_hash=sym_hash), ref)
        assert_rows_exact(run(A, B, reg_keys=keys, reg_top=False), ref)
        assert_rows_exact(run(A, B, reg_keys=keys, reg_perm=False), ref)
        assert_rows_exact(run(A, B, reg_keys=keys, reg_num_half=False), ref)


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_register_bins_every_size(mode, dtype, comp):
    """Rows of 1..1024 products and 1..256 lists (every register bin with 8,
    16 and 32 keys per thread, their capacity edges, duplicate-heavy and
    duplicate-free rows)."""
    k, n = 3000, 2500
    B = I.erdos_renyi(k, 4, seed=31, ncols=n)
    Bd = I.erdos_renyi(k, 4, seed=32, ncols=40)          # few columns: long runs of duplicates
    Ls = [1, 2, 7, 8, 9, 16, 17, 31, 32, 33, 63, 64, 65, 128, 129, 200, 255, 256]
    for Bm in (B, Bd):
        rows = []
        for t, L in enumerate(Ls):
            u = I.rand_u64(34, t, np.arange(8 * L + 64)) % np.uint64(k)
            _, idx = np.unique(u, return_index=True)
            rows.append(np.sort(u[np.sort(idx)][:L].astype(np.int64)))
        arp = np.zeros(len(rows) + 1, dtype=np.int64)
        arp[1:] = np.cumsum([len(r) for r in rows])
        acol = np.concatenate(rows).astype(np.int32)
        A = I.CSR(len(rows), k, arp.astype(np.int32), acol, I.rand_sym(35, 1, np.arange(len(acol))))
        ref = oracle.alg1(A, Bm, prec=mode)
        for keys in (8, 16, 32):
            assert_rows_exact(run(A, Bm, "precise", dtype, comp, reg_keys=keys), ref)
            assert_rows_exact(run(A, Bm, "precise", dtype, comp, reg_keys=keys, reg_perm=False), ref)
            assert_rows_exact(run(A, Bm, "precise", dtype, comp, reg_keys=keys, reg_num_direct=False), ref)
            assert_rows_exact(run(A, Bm, "upper", dtype, comp, reg_keys=keys), ref)


def test_register_bins_wide_B():
    """B with more columns than the register keys can pack for the larger
    bins: those rows take the shared-memory kernels, the result is the same."""
    k, n = 2000, (1 << 23) + 7
    B = I.erdos_renyi(k, 6, seed=36, ncols=n)
    for L, seed in ((100, 37), (40, 38), (3, 39)):   # block bin, register bins of 8 and 1 threads
        X = I.erdos_renyi(300, L, seed=seed, ncols=k)
        assert_rows_exact(run(X, B), oracle.alg1(X, B))


@pytest.mark.parametrize("chunk", [1, 4096, 200000])
def test_upper_in_row_chunks(chunk):
    """BRMerge-Upper with a C_bar budget smaller than the product: row chunks
    (down to one row each) give the same C as BRMerge-Precise."""
    A, B = bins_matrix(seed=9)
    ref = oracle.alg1(A, B)
    Cu = run(A, B, "upper", upper_chunk_bytes=chunk)
    assert_rows_exact(Cu, ref)
    same(Cu, run(A, B, "precise"))


def test_long_rows_small_arena_batches():
    """A tiny arena budget: one persistent block merges every long row, one
    after another, in one arena slot (merge rounds; the column windows need
    no arena)."""
    A, B = bins_matrix(seed=5)
    ref = oracle.alg1(A, B)
    assert_rows_exact(run(A, B, arena_bytes=1, long_window=False), ref)
    assert_rows_exact(run(A, B, arena_bytes=1, long_window=True), ref)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------
def _csr(rows, cols, rp, col, val):
    return I.CSR(rows, cols, np.asarray(rp, np.int32), np.asarray(col, np.int32), np.asarray(val, np.float64))


@pytest.mark.parametrize("case", ["zero_rows", "empty_A", "empty_B", "one", "col_vector", "identity", "perm"])
def test_edge_cases(case):
    if case == "zero_rows":
        A, B = _csr(0, 5, [0], [], []), I.random_int(5, 4, 0.5, 1, 1)
    elif case == "empty_A":
        A, B = _csr(4, 5, [0] * 5, [], []), I.random_int(5, 4, 0.5, 1, 1)
    elif case == "empty_B":
        A, B = I.random_int(4, 5, 0.5, 1, 0), _csr(5, 6, [0] * 6, [], [])
    elif case == "one":
        A, B = _csr(1, 1, [0, 1], [0], [3.0]), _csr(1, 1, [0, 1], [0], [-2.0])
    elif case == "col_vector":
        A, B = I.random_int(30, 7, 0.5, 2, 0), I.random_int(7, 1, 0.7, 2, 1)
    elif case == "identity":
        A, B = I.erdos_renyi(1000, 9, seed=7), I.identity(1000)
    else:
        A, B = I.permutation(1000, seed=8), I.erdos_renyi(1000, 9, seed=9)
    for method in ("precise", "upper"):
        C = run(A, B, method)
        assert C.rows == A.rows and C.cols == B.cols
        assert_rows_exact(C, oracle.gustavson(A, B))
    if case == "identity":
        C = run(A, B)
        assert np.array_equal(C.col.cpu().numpy(), A.col) and np.array_equal(C.val.cpu().numpy(), A.val)


def test_symbolic_and_row_nprod():
    A, B = bins_matrix(seed=6)
    dA, dB = brm.to_device(A), brm.to_device(B)
    rp, nnz = brm.brm_spgemm_symbolic(dA, dB)
    want = np.concatenate(([0], np.cumsum(oracle.symbolic(A, B))))
    assert nnz == want[-1]
    assert np.array_equal(rp.cpu().numpy(), want)
    npr, tot, mx, ml = brm.brm_row_nprod(dA, dB)
    ref = oracle.row_nprod(A, B)
    assert np.array_equal(npr.cpu().numpy(), ref)
    assert tot == ref.sum() and mx == ref.max() and ml == np.diff(A.rp).max()


def test_hash_symbolic_every_bin():
    """The paper's hashing symbolic pass (register, warp and block bins by
    shared-memory hash tables, long rows by the column bitmap) gives the
    oracle's row counts, and BRMerge-Precise on them the oracle's C."""
    R = I.rmat(14, 16, seed=87)
    dR = brm.to_device(R)
    want = np.concatenate(([0], np.cumsum(oracle.symbolic(R, R))))
    brm.brm_trace_reset()
    was = brm.brm_trace_enable(True)
    rp, nnz = brm.brm_spgemm_symbolic(dR, dR, symbolic_hash=True)
    assert nnz == want[-1] and np.array_equal(rp.cpu().numpy(), want)
    # without the register bins, the short rows take the warp bin's table
    rp, nnz = brm.brm_spgemm_symbolic(dR, dR, symbolic_hash=True, reg_max_nprod=-1)
    t = brm.brm_trace_read()
    brm.brm_trace_enable(was)
    assert nnz == want[-1] and np.array_equal(rp.cpu().numpy(), want)
    assert t["symbolic_warp"][1] >= 1 and t["symbolic_block"][1] >= 1
    assert t["symbolic_long"][1] + t["symbolic_tile"][1] >= 1
    C = run(R, R, symbolic_hash=True)
    nprod = oracle.row_nprod(R, R)
    rows = np.sort(np.concatenate([np.argsort(-nprod, kind="stable")[:30],
                                   np.nonzero((nprod > 256) & (nprod <= 4096))[0][:200]]))
    assert_rows_exact(C, oracle.alg1(R, R, rows), rows)


def test_validate_rejects_malformed():
    A = I.random_int(10, 10, 0.5, 3, 0)
    bad_col = A.col.copy()
    r = int(np.nonzero(np.diff(A.rp) >= 2)[0][0])
    s = A.rp[r]
    bad_col[s], bad_col[s + 1] = bad_col[s + 1], bad_col[s]        # unsorted row
    Abad = I.CSR(A.rows, A.cols, A.rp, bad_col, A.val)
    with pytest.raises(brm.BrmError) as e:
        run(Abad, A, validate=True)
    assert e.value.code == -1
    bad_col2 = A.col.copy()
    bad_col2[-1] = 10                                               # out of range
    with pytest.raises(brm.BrmError):
        run(I.CSR(A.rows, A.cols, A.rp, bad_col2, A.val), A, validate=True)
    C = run(A, A, validate=True)                                    # well-formed passes
    assert_rows_exact(C, oracle.gustavson(A, A))


def test_trace_counts_launches():
    A = I.lap2d(32)
    brm.brm_trace_reset()
    was = brm.brm_trace_enable(True)
    n0 = brm.brm_kernel_launches()
    run(A, A)
    t = brm.brm_trace_read()
    brm.brm_trace_enable(was)
    assert brm.brm_kernel_launches() > n0
    # every row of the 32 x 32 Laplacian squared has <= 25 products and <= 5
    # lists: all in the register bins of one or two threads per row
    assert 1 <= t["numeric_reg"][1] <= 2 and t["numeric_reg"][0] > 0
    assert t["bin"][1] == 2 and t["symbolic_reg"][1] == t["numeric_reg"][1]
    assert t["numeric_warp"][1] == 0 and t["numeric_block"][1] == 0 and t["numeric_long"][1] == 0


# --------------------------------------------------------------------------
# workload-sized cases
# --------------------------------------------------------------------------
def _sample_rows(m, nprod, count, seed):
    top = np.argsort(-nprod, kind="stable")[: count // 4]
    rnd = np.sort(I.rand_below(seed, 30, np.arange(count), m))
    return np.unique(np.concatenate([top, rnd, [0, m - 1]]))


def test_er_full_size_sampled():
    """Erdos-Renyi n = 2^20, 16 per row, A*A in FP64 (the benchmark workload,
    the same launch configuration): full structure against the oracle's
    symbolic pass, values of sampled rows bit-exact against Algorithm 1 and
    within 1e-12 of Gustavson."""
    A = I.erdos_renyi(1 << 20, 16)
    C = run(A, A)
    want_nnz = oracle.symbolic(A, A)
    rp = C.rp.cpu().numpy()
    assert np.array_equal(np.diff(rp), want_nnz)
    rows = _sample_rows(A.rows, oracle.row_nprod(A, A), 4000, 11)
    assert_rows_exact(C, oracle.alg1(A, A, rows), rows)
    assert_close_to_gustavson(C, A, A, rows)
    col = C.col.cpu().numpy().astype(np.int64)
    starts = np.zeros(len(col), dtype=bool)
    starts[rp[:-1][rp[:-1] < len(col)]] = True       # first entry of each row
    assert np.all((np.diff(col) > 0) | starts[1:]), "columns not strictly ascending inside rows"


@pytest.mark.parametrize("mode,dtype,comp", MODES)
def test_rmat_sampled(mode, dtype, comp):
    """R-MAT scale 16 (power-law rows in every bin): sampled rows, including
    the longest, bit-exact against Algorithm 1 in the same precision."""
    A = I.rmat(16, 16)
    C = run(A, A, "precise", dtype, comp)
    rows = _sample_rows(A.rows, oracle.row_nprod(A, A), 600, 12)
    assert_rows_exact(C, oracle.alg1(A, A, rows, prec=mode), rows)
    want_nnz = oracle.symbolic(A, A)
    assert np.array_equal(np.diff(C.rp.cpu().numpy()), want_nnz)


def test_float32_error_report_against_f64_oracle():
    """The FP32 paths against the FP64 oracle (inputs rounded to float, their
    exact products summed in double): entrywise within the summation bounds
    of plain float addition over the merge tree's depth, and of TwoSum; the
    compensated path is at least as accurate in the median."""
    A = I.rmat(14, 16, seed=71).astype(np.float32)
    rows = _sample_rows(A.rows, oracle.row_nprod(A, A), 800, 72)
    Ap = I.CSR(A.rows, A.cols, A.rp, A.col, A.val.astype(np.float64))
    ref = oracle.gustavson(Ap, Ap, rows, with_abs=True)
    u32 = 2.0 ** -24
    depth = int(np.ceil(np.log2(max(2, np.diff(A.rp.astype(np.int64)).max()))))
    errs = {}
    for comp in (False, True):
        C = run(A, A, "precise", np.float32, comp)
        rp, col, val = C.rp.cpu().numpy(), C.col.cpu().numpy(), C.val.cpu().numpy().astype(np.float64)
        from helpers import rows_of
        crp, c, v = rows_of(rp, col, val, rows)
        assert np.array_equal(c, ref.col)
        errs[comp] = np.abs(v - ref.val)
    assert np.all(errs[False] <= (depth + 1) * u32 * ref.abs * 1.0001)
    assert np.all(errs[True] <= u32 * np.abs(ref.val) + u32 * ref.abs + 3 * depth * u32 ** 2 * ref.abs)
    assert np.median(errs[True]) <= np.median(errs[False])
