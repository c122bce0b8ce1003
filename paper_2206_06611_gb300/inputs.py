"""Seeded synthetic CSR inputs for the BRMerge SpGEMM workloads.

This module is the one piece shared by the CUDA path's tests/bench and the
CPU oracle's tests.  It draws matrices and nothing else: it holds none of the
SpGEMM arithmetic (no products, no merging, no accumulation).

Every random draw goes through one counter-based generator, SplitMix64's
output function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``seed + stream*G2 + (idx+1)*G``.  A draw
therefore depends only on (seed, stream, idx) and never on call order, which
lets tests regenerate any row on its own.

Workloads (the paper evaluates C = A*A over 26 SuiteSparse matrices, Table II;
those matrices are not available here, so synthetic stand-ins with the same
kinds of structure are drawn instead):

* ``lap2d``   2-D 5-point Laplacian, values 4 / -1 (integer valued).
* ``lap3d``   3-D 7-point Laplacian, values 6 / -1 (integer valued).
* ``erdos_renyi``  exactly k distinct uniform columns per row (Floyd's
  sampling without replacement), values U[-1, 1).
* ``rmat``    R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004) with quadrant
  probabilities (a, b, c, d), no noise, no vertex permutation, self loops
  kept, duplicate edges removed, values U[-1, 1).
* ``batched_mix``  512 uneven products (log-uniform sizes, half Lap3D, half
  ER with 4..32 nonzeros per row).
* ``random_int``  small random matrices with integer values in [-4, 4] for
  exact brute-force checks.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_G2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_SEED = 0x220606611

# stream ids: one per kind of draw, so that draws never collide
S_ER_COL, S_ER_VAL, S_RMAT_QUAD, S_RMAT_VAL, S_SIZE, S_KIND, S_NORM, S_RAND_PAT, S_RAND_VAL, S_GRAD = range(1, 11)


@dataclasses.dataclass
class CSR:
    """Host CSR matrix: int32 row pointer and column indices, float values.

    Columns are strictly ascending inside every row.
    """
    rows: int
    cols: int
    rp: np.ndarray   # int32 [rows+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.rows, self.cols, self.rp, self.col, self.val.astype(dtype))

    def row(self, i: int):
        a, b = int(self.rp[i]), int(self.rp[i + 1])
        return self.col[a:b], self.val[a:b]


# ----------------------------------------------------------------------------
# counter-based generator
# ----------------------------------------------------------------------------
def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def rand_u64(seed: int, stream: int, idx) -> np.ndarray:
    """64-bit draws for counters ``idx`` (any integer array) of one stream."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(stream) * _G2
        z = base + (idx + np.uint64(1)) * _G
    return _mix(z)


def rand_unit(seed: int, stream: int, idx) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (rand_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rand_sym(seed: int, stream: int, idx) -> np.ndarray:
    """Doubles in [-1, 1) (exact: 2*u - 1 with u on a 2^-53 grid)."""
    return 2.0 * rand_unit(seed, stream, idx) - 1.0


def rand_below(seed: int, stream: int, idx, bound) -> np.ndarray:
    """Integers in [0, bound) by the 32x32 multiply-shift map (no rejection)."""
    hi = rand_u64(seed, stream, idx) >> np.uint64(32)
    return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def rand_normal(seed: int, stream: int, idx) -> np.ndarray:
    """N(0,1) by Box-Muller on two draws per index (cosine branch)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = rand_unit(seed, stream, idx * np.uint64(2))
    u2 = rand_unit(seed, stream, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# structured matrices
# ----------------------------------------------------------------------------
def _from_coo(rows: int, cols: int, r: np.ndarray, c: np.ndarray, v: np.ndarray) -> CSR:
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(rows + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(r, minlength=rows))
    return CSR(rows, cols, rp.astype(np.int32), c.astype(np.int32), np.ascontiguousarray(v))


def lap2d(g: int = 64) -> CSR:
    """5-point Laplacian on a g x g grid, node id x + g*y, 4 on the diagonal, -1 off it."""
    n = g * g
    ids = np.arange(n, dtype=np.int64)
    x, y = ids % g, ids // g
    rs, cs, vs = [], [], []
    for dx, dy, v in ((0, -1, -1.0), (-1, 0, -1.0), (0, 0, 4.0), (1, 0, -1.0), (0, 1, -1.0)):
        ok = (x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g)
        rs.append(ids[ok]); cs.append(ids[ok] + dx + g * dy); vs.append(np.full(int(ok.sum()), v))
    return _from_coo(n, n, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs))


def lap3d(s: int) -> CSR:
    """7-point Laplacian on an s^3 grid, node id x + s*(y + s*z), 6 / -1."""
    n = s ** 3
    ids = np.arange(n, dtype=np.int64)
    x, y, z = ids % s, (ids // s) % s, ids // (s * s)
    rs, cs, vs = [], [], []
    for dx, dy, dz, v in ((0, 0, -1, -1.0), (0, -1, 0, -1.0), (-1, 0, 0, -1.0), (0, 0, 0, 6.0),
                          (1, 0, 0, -1.0), (0, 1, 0, -1.0), (0, 0, 1, -1.0)):
        ok = (x + dx >= 0) & (x + dx < s) & (y + dy >= 0) & (y + dy < s) & (z + dz >= 0) & (z + dz < s)
        rs.append(ids[ok]); cs.append(ids[ok] + dx + s * dy + s * s * dz); vs.append(np.full(int(ok.sum()), v))
    return _from_coo(n, n, np.concatenate(rs), np.concatenate(cs), np.concatenate(vs))


def identity(n: int) -> CSR:
    return CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))


def permutation(n: int, seed: int = DEFAULT_SEED) -> CSR:
    """Row i holds a single 1.0 at column perm[i] (perm drawn by sorting draws)."""
    perm = np.argsort(rand_u64(seed, S_KIND, np.arange(n)), kind="stable").astype(np.int32)
    return CSR(n, n, np.arange(n + 1, dtype=np.int32), perm, np.ones(n))


# ----------------------------------------------------------------------------
# random matrices
# ----------------------------------------------------------------------------
def erdos_renyi(n: int, k: int, seed: int = DEFAULT_SEED, ncols: int | None = None,
                dtype=np.float64) -> CSR:
    """Exactly k distinct uniform columns per row (Floyd's algorithm), U[-1,1) values.

    Floyd's sampling: for j = N-k .. N-1 draw t in [0, j]; take t unless already
    taken, else take j.  Done for all rows at once, one j per step.
    """
    ncols = n if ncols is None else ncols
    assert 0 <= k <= ncols
    rows = np.arange(n, dtype=np.int64)
    S = np.empty((n, k), dtype=np.int64)
    for s, j in enumerate(range(ncols - k, ncols)):
        t = rand_below(seed, S_ER_COL, rows * k + s, j + 1)
        if s:
            taken = (S[:, :s] == t[:, None]).any(axis=1)
            t = np.where(taken, j, t)
        S[:, s] = t
    S.sort(axis=1)
    rp = (np.arange(n + 1, dtype=np.int64) * k).astype(np.int32)
    idx = np.arange(n * k, dtype=np.int64)
    val = rand_sym(seed, S_ER_VAL, idx).astype(dtype)
    return CSR(n, ncols, rp, S.reshape(-1).astype(np.int32), val)


def rmat(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05),
         seed: int = DEFAULT_SEED, dtype=np.float64, chunk: int = 1 << 21) -> CSR:
    """R-MAT graph adjacency: edge_factor * 2^scale edge draws, duplicates removed.

    Each draw descends ``scale`` levels, most significant bit first; at each
    level a 16-bit uniform picks a quadrant with probabilities (a, b, c, d) =
    (top-left, top-right, bottom-left, bottom-right).  One 64-bit draw feeds
    four levels.  The value of entry (i, j) is U[-1, 1) keyed by i*n + j, so it
    does not depend on how many duplicates were removed.
    """
    from concurrent.futures import ThreadPoolExecutor

    n = 1 << scale
    E = edge_factor * n
    a, b, c, _ = abcd
    t1, t2, t3 = (int(round(t * 65536)) for t in (a, a + b, a + b + c))
    words = (scale + 3) // 4

    def draw(e0):
        e = np.arange(e0, min(E, e0 + chunk), dtype=np.int64)
        r = np.zeros(len(e), dtype=np.int64)
        cc = np.zeros(len(e), dtype=np.int64)
        for w in range(words):
            z = rand_u64(seed, S_RMAT_QUAD, e * words + w)
            for f in range(4):
                lvl = 4 * w + f
                if lvl >= scale:
                    break
                u = ((z >> np.uint64(16 * f)) & np.uint64(0xFFFF)).astype(np.int64)
                q = (u >= t1).astype(np.int64) + (u >= t2) + (u >= t3)
                r = (r << 1) | (q >> 1)
                cc = (cc << 1) | (q & 1)
        return r * n + cc

    with ThreadPoolExecutor(8) as ex:
        keys = list(ex.map(draw, range(0, E, chunk)))
    key = np.sort(np.concatenate(keys))
    key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = key // n
    cc = key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(r, minlength=n))
    val = rand_sym(seed, S_RMAT_VAL, key).astype(dtype)
    return CSR(n, n, rp.astype(np.int32), cc.astype(np.int32), val)


def random_int(m: int, k: int, density: float, seed: int, stream_off: int = 0) -> CSR:
    """Small m x k matrix, each entry present with probability ``density``,
    integer values uniform in [-4, 4] (zero allowed: kept as a stored entry)."""
    idx = np.arange(m * k, dtype=np.int64) + stream_off * (m * k + 1)
    present = rand_unit(seed, S_RAND_PAT, idx) < density
    vals = (rand_below(seed, S_RAND_VAL, idx, 9) - 4).astype(np.float64)
    mask = present.reshape(m, k)
    rp = np.zeros(m + 1, dtype=np.int64)
    rp[1:] = np.cumsum(mask.sum(axis=1))
    rr, cc = np.nonzero(mask)
    return CSR(m, k, rp.astype(np.int32), cc.astype(np.int32), vals.reshape(m, k)[rr, cc])


def to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.rows, A.cols), dtype=np.float64)
    for i in range(A.rows):
        c, v = A.row(i)
        D[i, c] = v
    return D


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------
def batched_mix(count: int = 512, seed: int = DEFAULT_SEED, nmin: float = 1e3, nmax: float = 2e5,
                dtype=np.float64, scale_n: float = 1.0):
    """``count`` uneven matrices: n_i = round(exp(U[ln nmin, ln nmax])) * scale_n.

    Even i: 3-D 7-point Laplacian with side round(n_i^(1/3)).  Odd i: ER with
    k_i uniform in {4..32} (one k per matrix).  Returns a list of CSR; each is
    squared on its own (C_i = A_i * A_i).
    """
    out = []
    for i in range(count):
        u = float(rand_unit(seed, S_SIZE, [i])[0])
        ni = max(8, int(round(math.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin))) * scale_n)))
        if i % 2 == 0:
            s = max(2, int(round(ni ** (1.0 / 3.0))))
            out.append(lap3d(s).astype(dtype))
        else:
            k = 4 + int(rand_below(seed, S_KIND, [i], 29)[0])
            out.append(erdos_renyi(ni, min(k, ni), seed=seed + 7919 * i, dtype=dtype))
    return out


def normal_values(A: CSR, seed: int, stream: int = S_NORM, dtype=np.float32) -> CSR:
    """Same pattern, values N(0,1) keyed by (row*cols + col)."""
    rows = np.repeat(np.arange(A.rows, dtype=np.int64), np.diff(A.rp.astype(np.int64)))
    key = rows * A.cols + A.col.astype(np.int64)
    return CSR(A.rows, A.cols, A.rp, A.col, rand_normal(seed, stream, key).astype(dtype))


def pattern_normal(rows: int, cols: int, rp: np.ndarray, col: np.ndarray, seed: int,
                   dtype=np.float32) -> np.ndarray:
    """N(0,1) values on a given pattern (the upstream gradient G of C)."""
    rp = np.asarray(rp, dtype=np.int64)
    r = np.repeat(np.arange(rows, dtype=np.int64), np.diff(rp))
    return rand_normal(seed, S_GRAD, r * cols + np.asarray(col, dtype=np.int64)).astype(dtype)


def workload(name: str, seed: int = DEFAULT_SEED):
    """The named configurations: returns (A, B) (B is A for squares)."""
    if name == "lap2d":
        A = lap2d(64)
        return A, A
    if name == "er":
        A = erdos_renyi(1 << 20, 16, seed=seed)
        return A, A
    if name == "rmat":
        A = rmat(20, 16, seed=seed)
        return A, A
    if name == "diff":
        A = normal_values(rmat(18, 16, seed=seed), seed, dtype=np.float32)
        B = erdos_renyi(1 << 18, 8, seed=seed + 1)
        B = normal_values(B, seed + 1, dtype=np.float32)
        return A, B
    raise KeyError(name)
