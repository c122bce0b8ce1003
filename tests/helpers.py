"""Shared helpers of the GPU parity tests (comparisons against the oracle)."""
import numpy as np

import oracle
from paper_2206_06611_gb300 import inputs as I

# FP64 tolerance of the spec criterion: per row,
#   ||c_gpu - c_ref||_2 <= 1e-12 * ||(|A| |B|)_i*||_2
# (the scale of the standard summation error bound, Higham, Accuracy and
# Stability of Numerical Algorithms, 2nd ed., Sec. 4.2: every entry's error is
# at most gamma_{L-1} times its sum of absolute products).
RTOL_F64 = 1e-12


def host_result(C):
    """(rp int64, col int32, val float64) of a DeviceCSR result."""
    return (C.rp.cpu().numpy().astype(np.int64), C.col.cpu().numpy(), C.val.cpu().numpy().astype(np.float64))


def rows_of(rp, col, val, rows):
    """Concatenate the given rows of a CSR (for comparison with oracle samples)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = rp[rows + 1] - rp[rows]
    crp = np.zeros(len(rows) + 1, dtype=np.int64)
    crp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if len(rows) else np.zeros(0, np.int64)
    return crp, col[idx], val[idx]


def assert_rows_exact(C, ref, rows=None):
    """Structure and values equal, row by row (values with ==, so -0 == +0)."""
    rp, col, val = host_result(C)
    if rows is None:
        assert np.array_equal(rp, ref.crp), "row_ptr differs"
        crp, c, v = rp, col, val
    else:
        crp, c, v = rows_of(rp, col, val, rows)
        assert np.array_equal(crp, ref.crp), "row lengths differ"
    assert np.array_equal(c, ref.col), "column indices differ"
    bad = np.nonzero(~(v == ref.val))[0]
    assert len(bad) == 0, f"{len(bad)} values differ, first at {bad[:5]}: {v[bad[:5]]} vs {ref.val[bad[:5]]}"


def rowwise_rel_err(crp, v, ref_val, ref_abs):
    """Per row ||v - ref||_2 / ||abs||_2 (0 for rows whose scale is 0)."""
    d = (v - ref_val) ** 2
    s = ref_abs ** 2
    cs = np.concatenate(([0.0], np.cumsum(d)))
    ca = np.concatenate(([0.0], np.cumsum(s)))
    num = np.sqrt(np.maximum(cs[crp[1:]] - cs[crp[:-1]], 0))
    den = np.sqrt(np.maximum(ca[crp[1:]] - ca[crp[:-1]], 0))
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def assert_close_to_gustavson(C, A, B, rows=None, rtol=RTOL_F64):
    ref = oracle.gustavson(A, B, rows, with_abs=True)
    rp, col, val = host_result(C)
    if rows is None:
        crp, c, v = rp, col, val
    else:
        crp, c, v = rows_of(rp, col, val, rows)
    assert np.array_equal(crp, ref.crp)
    assert np.array_equal(c, ref.col)
    err = rowwise_rel_err(crp, v, ref.val, ref.abs)
    assert err.max(initial=0.0) <= rtol, f"max row error {err.max()}"
    return err


def _first_unique(u, count):
    """The first `count` distinct values of u in draw order."""
    _, idx = np.unique(u, return_index=True)
    return u[np.sort(idx)][:count]


def bins_matrix(seed=3):
    """A and B whose rows of A*B fall in every bin: empty rows, tiny rows,
    warp rows (nprod <= 256), block rows (<= 4096 products, <= 1024 lists),
    long rows (more products, or more than 1024 lists with few products),
    rows with many empty lists, duplicate-heavy rows.  Values U[-1,1)."""
    k, n = 6000, 3000
    # B: row lengths 0..60 (a third empty), some long rows
    blen = I.rand_below(seed, 20, np.arange(k), 61)
    blen[I.rand_unit(seed, 21, np.arange(k)) < 0.33] = 0
    blen[::997] = 400
    rows_b = []
    for r in range(k):
        u = I.rand_u64(seed, 22, np.arange(r * 512, r * 512 + 512)) % np.uint64(n)
        rows_b.append(np.sort(_first_unique(u.astype(np.int64), blen[r])))
    brp = np.zeros(k + 1, dtype=np.int64)
    brp[1:] = np.cumsum([len(c) for c in rows_b])
    bcol = np.concatenate(rows_b).astype(np.int32)
    B = I.CSR(k, n, brp.astype(np.int32), bcol, I.rand_sym(seed, 23, np.arange(len(bcol))))
    # A: row list counts covering all bins
    Ls = [0, 1, 2, 3, 5, 7, 8, 16, 17, 31, 33, 64, 100, 150, 255, 256, 257, 300, 500, 1000, 1023, 1024,
          1025, 1500, 2047, 2500, 4000, 5999]
    rows_a = []
    for t, L in enumerate(Ls):
        u = I.rand_u64(seed, 24, np.arange(t * 8192, t * 8192 + 8192)) % np.uint64(k)
        rows_a.append(np.sort(_first_unique(u.astype(np.int64), L)))
    # a row that points only at empty B rows (many empty lists, no products)
    empty_b = np.nonzero(blen == 0)[0]
    rows_a.append(np.sort(empty_b[:700]))
    # a row with many empty lists and a few products (long bin by list count)
    mixed = np.sort(np.concatenate([empty_b[700:2000], np.nonzero(blen > 0)[0][:5]]))
    rows_a.append(mixed)
    # a duplicate-heavy row: many lists over few columns
    rows_a.append(np.nonzero((blen > 0) & (blen < 4))[0][:900])
    arp = np.zeros(len(rows_a) + 1, dtype=np.int64)
    arp[1:] = np.cumsum([len(c) for c in rows_a])
    acol = np.concatenate(rows_a).astype(np.int32)
    A = I.CSR(len(rows_a), k, arp.astype(np.int32), acol, I.rand_sym(seed, 25, np.arange(len(acol))))
    return A, B


def device_rows(C, rows):
    """(row_ptr, col, val as float64) of the given rows of a device result,
    gathered on the device (for results too large to copy to the host)."""
    import torch
    rows = np.asarray(rows, dtype=np.int64)
    rp = C.rp.cpu().numpy()
    starts, ends = rp[rows], rp[rows + 1]
    idx = np.concatenate([np.arange(a, b, dtype=np.int64) for a, b in zip(starts, ends)]) if len(rows) else \
        np.zeros(0, np.int64)
    it = torch.from_numpy(idx).to(C.col.device)
    crp = np.zeros(len(rows) + 1, dtype=np.int64)
    crp[1:] = np.cumsum(ends - starts)
    return crp, C.col[it].cpu().numpy(), C.val[it].cpu().numpy().astype(np.float64)


def assert_sample_exact(crp, col, val, ref):
    """Sampled rows (crp, col, val) equal to an oracle Result of the same rows."""
    assert np.array_equal(crp, ref.crp), "row lengths differ"
    assert np.array_equal(col, ref.col), "column indices differ"
    bad = np.nonzero(~(val == ref.val))[0]
    assert len(bad) == 0, f"{len(bad)} values differ, first at {bad[:5]}: {val[bad[:5]]} vs {ref.val[bad[:5]]}"


def straddling_rows(rp, marks):
    """Rows whose slice of C contains one of the offsets in `marks` (and the
    rows right before and after them)."""
    out = []
    m = len(rp) - 1
    for x in marks:
        if x < rp[-1]:
            i = int(np.searchsorted(rp, x, side="right")) - 1
            out += [j for j in (i - 1, i, i + 1) if 0 <= j < m]
    return np.array(sorted(set(out)), dtype=np.int64)
