"""Pins for the CPU oracle: each check compares it with something fixed by the
paper or by mathematics, never with itself.

* brute force: dense products of small integer matrices (Eq. 1), exhaustive
  over every 2x2 and 3x3 sparsity pattern;
* closed forms: the squares of the 2-D 5-point and 3-D 7-point Laplacians,
  derived from grid geometry;
* special cases: identity and permutation products, (AB)^T = B^T A^T;
* Fig. 2: six lists take three merging rounds; ceil(log2 L) in general;
* hand-derived double-precision cases in which the merge tree of Algorithm 1
  (pairs (0,1),(2,3),..., empty lists keeping their slot) gives a result that
  a sequential sum does not;
* the summation error bound (Higham, Accuracy and Stability of Numerical
  Algorithms, 2nd ed., Sec. 4.2) between Algorithm 1 and Gustavson;
* exact finite differences for the backward (the loss is linear in A and B).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def pattern(A):
    P = np.zeros((A.rows, A.cols), dtype=np.int64)
    for i in range(A.rows):
        P[i, A.row(i)[0]] = 1
    return P


def dense_of(res, m, n):
    D = np.zeros((m, n))
    S = np.zeros((m, n), dtype=np.int64)
    for t in range(m):
        c, v = res.row(t)
        D[t, c] = v
        S[t, c] = 1
    return D, S


def csr_from_dense_pattern(P, V):
    m, n = P.shape
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(P.sum(axis=1))
    r, c = np.nonzero(P)
    return I.CSR(m, n, rp.astype(np.int32), c.astype(np.int32), V[r, c].astype(np.float64))


def transpose(A):
    P = pattern(A).T.copy()
    V = I.to_dense(A).T.copy()
    return csr_from_dense_pattern(P, V)


def check_sorted_unique(res):
    for t in range(len(res.rows)):
        c, _ = res.row(t)
        assert np.all(np.diff(c) > 0)


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,k,n,da,db,seed", [
    (1, 1, 1, 1.0, 1.0, 1), (7, 1, 5, 0.6, 0.6, 2), (5, 9, 1, 0.5, 0.7, 3),
    (17, 23, 19, 0.3, 0.2, 4), (48, 40, 44, 0.1, 0.15, 5), (33, 48, 29, 0.6, 0.5, 6),
    (20, 20, 20, 0.0, 0.5, 7), (20, 20, 20, 0.4, 0.0, 8), (31, 17, 45, 0.05, 0.05, 9),
])
def test_dense_brute_force(m, k, n, da, db, seed):
    A = I.random_int(m, k, da, seed, 0)
    B = I.random_int(k, n, db, seed, 1)
    DA, DB = I.to_dense(A), I.to_dense(B)
    want = DA @ DB                                   # integers: exact in double
    want_pat = (pattern(A) @ pattern(B)) > 0         # structural pattern
    for res in (oracle.gustavson(A, B), oracle.alg1(A, B, prec="f64"),
                oracle.alg1(A, B, prec="f32"), oracle.alg1(A, B, prec="f32c")):
        D, S = dense_of(res, m, n)
        check_sorted_unique(res)
        assert np.array_equal(S.astype(bool), want_pat)
        assert np.array_equal(D, want)
    nnz = oracle.symbolic(A, B)
    assert np.array_equal(nnz, want_pat.sum(axis=1))
    nprod = oracle.row_nprod(A, B)
    assert np.array_equal(nprod, pattern(A) @ pattern(B).sum(axis=1))


def _all_patterns(r, c):
    for bits in range(1 << (r * c)):
        yield np.array([(bits >> s) & 1 for s in range(r * c)], dtype=np.int64).reshape(r, c)


@pytest.mark.parametrize("size", [2, 3])
def test_exhaustive_small_patterns(size):
    """Every sparsity pattern of A (2x2: all 16 x 16 pairs; 3x3: all 512
    patterns of A against 8 fixed patterns of B), integer values."""
    rng_vals = np.arange(1, size * size + 1, dtype=np.float64).reshape(size, size)
    pats = list(_all_patterns(size, size))
    bpats = pats if size == 2 else [pats[i] for i in (0, 1, 7, 73, 146, 273, 438, 511)]
    for PA in pats:
        A = csr_from_dense_pattern(PA, rng_vals - 3.0)
        for PB in bpats:
            B = csr_from_dense_pattern(PB, 2.0 - rng_vals.T)
            want = I.to_dense(A) @ I.to_dense(B)
            for res in (oracle.gustavson(A, B), oracle.alg1(A, B)):
                D, S = dense_of(res, size, size)
                assert np.array_equal(S, ((PA @ PB) > 0).astype(np.int64))
                assert np.array_equal(D, want)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
def lap2d_square_closed_form(g):
    """Entries of L^2 for the 5-point Laplacian (4 / -1) from grid geometry:
    (L^2)_pp = 16 + deg(p); at an axis neighbour -8; at a diagonal neighbour
    (+-1,+-1) 2 (two paths of (-1)(-1)); at axis distance 2: 1."""
    n = g * g
    out = {}
    for y in range(g):
        for x in range(g):
            p = x + g * y
            deg = sum(1 for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)) if 0 <= x + dx < g and 0 <= y + dy < g)
            out[(p, p)] = 16.0 + deg
            for dx, dy, v in ((1, 0, -8.0), (-1, 0, -8.0), (0, 1, -8.0), (0, -1, -8.0),
                              (1, 1, 2.0), (1, -1, 2.0), (-1, 1, 2.0), (-1, -1, 2.0),
                              (2, 0, 1.0), (-2, 0, 1.0), (0, 2, 1.0), (0, -2, 1.0)):
                if 0 <= x + dx < g and 0 <= y + dy < g:
                    out[(p, x + dx + g * (y + dy))] = v
    return n, out


def test_lap2d_square_closed_form():
    g = 64
    A = I.lap2d(g)
    assert A.nnz == 20224
    n, want = lap2d_square_closed_form(g)
    assert int(oracle.row_nprod(A, A).sum()) == 4 * 3 ** 2 + 248 * 4 ** 2 + 3844 * 5 ** 2 == 100104
    for res in (oracle.gustavson(A, A), oracle.alg1(A, A)):
        assert res.nnz == len(want) == 51972
        for t in range(n):
            c, v = res.row(t)
            got = {(t, int(j)): float(x) for j, x in zip(c, v)}
            exp = {key: val for key, val in want.items() if key[0] == t}
            assert got == exp


def test_lap3d_square_closed_form():
    """7-point Laplacian (6 / -1): diagonal 36 + deg, axis neighbour -12,
    planar diagonal 2, axis distance 2: 1."""
    s = 6
    A = I.lap3d(s)
    res = oracle.gustavson(A, A)
    res1 = oracle.alg1(A, A)
    assert np.array_equal(res.col, res1.col) and np.array_equal(res.val, res1.val)
    inside = lambda x, y, z: 0 <= x < s and 0 <= y < s and 0 <= z < s
    axes = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    nnz = 0
    for z in range(s):
        for y in range(s):
            for x in range(s):
                p = x + s * (y + s * z)
                exp = {p: 36.0 + sum(1 for d in axes if inside(x + d[0], y + d[1], z + d[2]))}
                for d in axes:
                    if inside(x + d[0], y + d[1], z + d[2]):
                        exp[x + d[0] + s * (y + d[1] + s * (z + d[2]))] = -12.0
                    if inside(x + 2 * d[0], y + 2 * d[1], z + 2 * d[2]):
                        exp[x + 2 * d[0] + s * (y + 2 * d[1] + s * (z + 2 * d[2]))] = 1.0
                for a in range(6):
                    for b in range(6):
                        da, db = axes[a], axes[b]
                        if a // 2 < b // 2:
                            q = (x + da[0] + db[0], y + da[1] + db[1], z + da[2] + db[2])
                            if inside(*q):
                                exp[q[0] + s * (q[1] + s * q[2])] = 2.0
                c, v = res.row(p)
                assert dict(zip(c.tolist(), v.tolist())) == exp
                nnz += len(exp)
    assert res.nnz == nnz


# --------------------------------------------------------------------------
# special cases
# --------------------------------------------------------------------------
def test_identity_and_permutation():
    A = I.erdos_renyi(300, 7, seed=11)
    Id = I.identity(300)
    res = oracle.gustavson(A, Id)
    assert np.array_equal(res.crp, A.rp) and np.array_equal(res.col, A.col) and np.array_equal(res.val, A.val)
    res = oracle.alg1(Id, A)
    assert np.array_equal(res.col, A.col) and np.array_equal(res.val, A.val)
    P = I.permutation(300, seed=5)
    res = oracle.alg1(P, A)
    for i in range(300):
        c, v = res.row(i)
        c0, v0 = A.row(int(P.col[i]))
        assert np.array_equal(c, c0) and np.array_equal(v, v0)


def test_transpose_identity():
    """Eq. (2) vs Eq. (3): (A B)^T and B^T A^T have the same entries."""
    A = I.random_int(30, 25, 0.2, 21, 0)
    B = I.random_int(25, 35, 0.15, 21, 1)
    C = oracle.gustavson(A, B)
    Ct = oracle.gustavson(transpose(B), transpose(A))
    D, S = dense_of(C, 30, 35)
    Dt, St = dense_of(Ct, 35, 30)
    assert np.array_equal(S.T, St) and np.array_equal(D.T, Dt)


def test_invariants_rmat_er():
    A = I.rmat(10, 8, seed=3)
    E = I.erdos_renyi(1024, 16, seed=4)
    for X, Y in ((A, A), (E, E), (A, E)):
        nprod = oracle.row_nprod(X, Y)
        res = oracle.gustavson(X, Y)
        check_sorted_unique(res)
        nnz = np.diff(res.crp)
        assert np.all(nnz <= np.minimum(nprod, Y.cols))
        assert np.array_equal(nnz, oracle.symbolic(X, Y))
        assert res.nnz <= nprod.sum()
    assert int(oracle.row_nprod(E, E).sum()) == 256 * 1024


# --------------------------------------------------------------------------
# Algorithm 1: round count and tree shape
# --------------------------------------------------------------------------
def lists_row(values_per_list):
    """A 1 x L row times an L x 1 B: list k is [A_0k * B_k0] at column 0, or
    empty when values_per_list[k] is None (B row k empty)."""
    L = len(values_per_list)
    A = I.CSR(1, L, np.array([0, L], dtype=np.int32), np.arange(L, dtype=np.int32), np.ones(L))
    brp = [0]
    for v in values_per_list:
        brp.append(brp[-1] + (0 if v is None else 1))
    vals = np.array([v for v in values_per_list if v is not None], dtype=np.float64)
    B = I.CSR(L, 1, np.array(brp, dtype=np.int32), np.zeros(len(vals), dtype=np.int32), vals)
    return A, B


def test_fig2_round_count_golden():
    path = os.path.join(HERE, "golden", "fig2_rounds.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for L, rounds in rows:
        A, B = lists_row([1.0] * int(L))
        assert int(oracle.alg1(A, B).rounds[0]) == int(rounds)


@pytest.mark.parametrize("L", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 16, 17, 33, 100])
def test_round_count_ceil_log2(L):
    A, B = lists_row([float(k + 1) for k in range(L)])
    res = oracle.alg1(A, B)
    assert int(res.rounds[0]) == (0 if L <= 1 else math.ceil(math.log2(L)))
    if L:
        assert res.val[0] == L * (L + 1) / 2


T53 = 2.0 ** 53


def test_tree_order_pairs():
    """Lists [2^53], [1], [1], [-2^53].  Tree: (2^53 + 1) rounds to 2^53 (tie to
    even), (1 + -2^53) = -(2^53 - 1) exactly, total 1.  A left-to-right sum
    gives 0, which Gustavson (dense accumulator, stored order) returns."""
    A, B = lists_row([T53, 1.0, 1.0, -T53])
    assert oracle.alg1(A, B).val[0] == 1.0
    assert oracle.gustavson(A, B).val[0] == 0.0


def test_tree_order_empty_lists_keep_slot():
    """Lists [1], [], [2^53], [-2^53]: empty list 1 keeps its slot, so round 0
    pairs (1, empty) and (2^53, -2^53); total 1 + 0 = 1.  Dropping the empty
    list would pair (1, 2^53) -> 2^53, then 2^53 - 2^53 = 0."""
    A, B = lists_row([1.0, None, T53, -T53])
    assert oracle.alg1(A, B).val[0] == 1.0


def test_tree_order_odd_list_copied():
    """Lists [2^53], [1], [1], [1], [-2^53].  Round 0: 2^53, 2, [-2^53] copied;
    round 1: 2^53 + 2 = 2^53 + 2 (representable), [-2^53] copied; round 2: 2."""
    A, B = lists_row([T53, 1.0, 1.0, 1.0, -T53])
    res = oracle.alg1(A, B)
    assert res.val[0] == 2.0 and int(res.rounds[0]) == 3


def test_tree_order_float_modes():
    """Single precision, lists [2^24], [1], [1], [-2^24]: plain float gives 1 as
    in double with 2^53; TwoSum keeps the lost 1 of (2^24 + 1) and gives 2,
    the exact sum."""
    A, B = lists_row([2.0 ** 24, 1.0, 1.0, -(2.0 ** 24)])
    assert oracle.alg1(A, B, prec="f32").val[0] == 1.0
    assert oracle.alg1(A, B, prec="f32c").val[0] == 2.0


# --------------------------------------------------------------------------
# error bounds
# --------------------------------------------------------------------------
def per_row_err(res_a, res_b, absres):
    d = res_a.val - res_b.val
    out = []
    for t in range(len(res_a.rows)):
        a, b = int(res_a.crp[t]), int(res_a.crp[t + 1])
        out.append((np.linalg.norm(d[a:b]), np.linalg.norm(absres.abs[a:b])))
    return np.array(out)


@pytest.mark.parametrize("which", ["er", "rmat"])
def test_alg1_vs_gustavson_error_bound(which):
    """Any summation order of s terms has error <= (s-1) u sum|x_i| per entry;
    two orders differ by at most twice that.  Per row in 2-norm:
    ||c_alg1 - c_gus|| <= 2 (Lmax) u || |A||B| ||."""
    A = I.erdos_renyi(2048, 16, seed=9) if which == "er" else I.rmat(11, 16, seed=9)
    g = oracle.gustavson(A, A, with_abs=True)
    a1 = oracle.alg1(A, A)
    assert np.array_equal(g.crp, a1.crp) and np.array_equal(g.col, a1.col)
    Lmax = int(np.diff(A.rp).max())
    u = 2.0 ** -53
    e = per_row_err(a1, g, g)
    assert np.all(e[:, 0] <= 2 * Lmax * u * e[:, 1])
    # and the two orders really differ somewhere on random data
    assert np.any(a1.val != g.val)


def test_float_modes_error_bounds():
    """f32: each entry of C is a sum of float-rounded products; plain float
    summation errs by <= depth * u32 * sum|p|; TwoSum-compensated by
    <= u32 |s| + 3 depth u32^2 sum|p| (Ogita, Rump, Oishi, SISC 2005, Prop. 4.5
    style bound for cascaded TwoSum)."""
    A = I.rmat(11, 16, seed=13).astype(np.float32)
    res = oracle.alg1(A, A, prec="f32")
    resc = oracle.alg1(A, A, prec="f32c")
    # exact sums of the float-rounded products, from double (a*b of two floats
    # is exact in double; rounding that to float gives the float product)
    Ap = I.CSR(A.rows, A.cols, A.rp, A.col, A.val.astype(np.float64))
    ref = oracle.gustavson(Ap, Ap, with_abs=True)   # double sums of exact products
    u32 = 2.0 ** -24
    L = np.diff(A.rp.astype(np.int64))
    depth = int(np.ceil(np.log2(max(2, L.max()))))
    # products rounded to float: |p - ab| <= u32 |ab| adds u32 * sum|ab|
    err = np.abs(res.val - ref.val)
    errc = np.abs(resc.val - ref.val)
    assert np.all(err <= (depth + 1) * u32 * ref.abs * 1.0001)
    assert np.all(errc <= u32 * np.abs(ref.val) + u32 * ref.abs + 3 * depth * u32 ** 2 * ref.abs)
    assert np.median(errc) <= np.median(err)


# --------------------------------------------------------------------------
# backward
# --------------------------------------------------------------------------
def test_backward_exact_finite_differences():
    """loss(A, B) = sum(C * G) is linear in A and in B, so with integer data
    loss(A + E_ik) - loss(A) equals dA_ik exactly (h = 1), likewise for B."""
    A = I.random_int(12, 10, 0.35, 31, 0)
    B = I.random_int(10, 14, 0.35, 31, 1)
    C = oracle.gustavson(A, B)
    G = (I.rand_below(77, I.S_GRAD, np.arange(C.nnz), 7) - 3).astype(np.float64)

    def loss(X, Y):
        Cx = oracle.gustavson(X, Y)
        D, _ = dense_of(Cx, X.rows, Y.cols)
        Gd, _ = dense_of(oracle.Result(C.rows, C.crp, C.col, G), X.rows, Y.cols)
        return float((D * Gd).sum())

    da, db = oracle.backward(A, B, C.crp, C.col, G)
    base = loss(A, B)
    for p in range(A.nnz):
        Ap = I.CSR(A.rows, A.cols, A.rp, A.col, A.val.copy())
        Ap.val[p] += 1.0
        assert loss(Ap, B) - base == da[p]
    for q in range(B.nnz):
        Bp = I.CSR(B.rows, B.cols, B.rp, B.col, B.val.copy())
        Bp.val[q] += 1.0
        assert loss(A, Bp) - base == db[q]
    # and against dense matrix algebra: dA = (G B^T) on A's pattern
    Gd, _ = dense_of(oracle.Result(C.rows, C.crp, C.col, G), A.rows, B.cols)
    dA = Gd @ I.to_dense(B).T
    dB = I.to_dense(A).T @ Gd
    for i in range(A.rows):
        c, _ = A.row(i)
        assert np.array_equal(da[A.rp[i]:A.rp[i + 1]], dA[i, c])
    for k in range(B.rows):
        c, _ = B.row(k)
        assert np.array_equal(db[B.rp[k]:B.rp[k + 1]], dB[k, c])


def test_parallel_gustavson_matches():
    A = I.rmat(10, 8, seed=5)
    r1 = oracle.gustavson(A, A)
    r2 = oracle.gustavson_parallel(A, A, 4)
    assert np.array_equal(r1.crp, r2.crp) and np.array_equal(r1.col, r2.col) and np.array_equal(r1.val, r2.val)


def test_parallel_alg1_and_symbolic_match():
    """Spreading rows over threads changes nothing: same rows, same values,
    in the requested row order (also for an unsorted sample)."""
    A = I.rmat(10, 8, seed=5)
    rows = np.array([1000, 3, 3, 0, 511, 17, 1023], dtype=np.int64)
    for prec in ("f64", "f32c"):
        r1, r2 = oracle.alg1(A, A, rows, prec), oracle.alg1_parallel(A, A, rows, prec, threads=3)
        assert np.array_equal(r1.crp, r2.crp) and np.array_equal(r1.col, r2.col)
        assert np.array_equal(r1.val, r2.val) and np.array_equal(r1.rounds, r2.rounds)
    assert np.array_equal(oracle.symbolic(A, A), oracle.symbolic_parallel(A, A, threads=4))


def test_sampled_rows_match_full():
    A = I.rmat(10, 8, seed=6)
    full = oracle.alg1(A, A)
    rows = np.array([0, 5, 17, 1000, 1023, 3], dtype=np.int64)
    samp = oracle.alg1(A, A, rows=rows)
    for t, i in enumerate(rows):
        c, v = samp.row(t)
        c0, v0 = full.row(int(i))
        assert np.array_equal(c, c0) and np.array_equal(v, v0)


def test_balanced_row_groups_brute_force():
    """Section III-D's static split (reading: group g starts at the first row
    whose exclusive nprod prefix reaches floor(g * total / p)) against a
    direct search, and its balance: no group holds more than total / p plus
    its largest row."""
    rng = np.random.default_rng(1406)
    cases = [np.array([5, 5, 5, 5]), np.array([1, 100, 1, 1]), np.zeros(6, np.int64), np.array([7])]
    cases += [rng.integers(0, 50, size=n) * (rng.random(n) < 0.7) for n in (1, 2, 9, 40, 300)]
    for nprod in cases:
        nprod = np.asarray(nprod, np.int64)
        total = int(nprod.sum())
        for p in (1, 2, 3, 7, 16):
            b = oracle.balanced_row_groups(nprod, p)
            want = [0]
            for g in range(1, p):
                target = total * g // p
                i = 0
                while i < len(nprod) and int(nprod[:i].sum()) < target:
                    i += 1
                want.append(max(i, want[-1]))
            want.append(len(nprod))
            assert [int(x) for x in b] == want
            assert all(x <= y for x, y in zip(b, b[1:]))
            for g in range(p):
                part = nprod[b[g]:b[g + 1]]
                if len(part):
                    assert int(part.sum()) <= total / p + int(part.max())
    assert [int(x) for x in oracle.balanced_row_groups(np.array([5, 5, 5, 5]), 2)] == [0, 2, 4]
