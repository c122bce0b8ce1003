"""The order argument behind the column tiles of long rows, checked on the CPU.

The tile kernel (k_long_tile) does not merge a long row's lists round by round;
it cuts the row into column ranges, brings each column's products together in
list order, and adds them by Algorithm 1's rounds restricted to that column:
a live sum and its next live sum of the same column meet in round
bitlen(t_left ^ t_right) (t: the smallest list of a sum), and after taking its
neighbour a sum meets the next one in a later round.  A cell too crowded for
one tile is taken in chunks of aligned list blocks [a 2^k, (a + 1) 2^k) --
complete subtrees of the merge tree -- whose sums of a column are added by a
level stack carried across the chunks (join level bitlen(start1 ^ start2)).

This file restates those steps in plain Python (sequential, in double) and
requires the results to be the bits of the oracle's Algorithm 1 on seeded
random rows: many lists of every length, empty lists, columns shared by many
lists, chunk sizes that force every chunk shape.  It tests the design, not the
CUDA code (the -m gpu tests in test_gpu_long_tiles.py do that).
"""
import numpy as np
import pytest

import oracle
from paper_2206_06611_gb300 import inputs as I


def _bitlen(x: int) -> int:
    return int(x).bit_length()


def _rounds_by_level(prods):
    """Column sums of products (t, c, v) given in list order: the products
    sorted stably by column, then the event-driven rounds on the positions."""
    order = sorted(range(len(prods)), key=lambda p: prods[p][1])   # stable: list order within a column
    t = [prods[p][0] for p in order]
    c = [prods[p][1] for p in order]
    val = [prods[p][2] for p in order]
    n = len(order)
    nxt = list(range(1, n + 1))
    retired = [False] * n
    level = [None] * n
    for s in range(n - 1):
        if c[s + 1] == c[s]:
            level[s] = _bitlen(t[s] ^ t[s + 1])
    h = 1
    while any(lv is not None for lv in level):
        for s in [s for s in range(n) if level[s] == h]:   # disjoint pairs: any order
            if retired[s]:
                level[s] = None
                continue
            j = nxt[s]
            val[s] = val[s] + val[j]
            retired[j] = True
            nxt[s] = nxt[j]
            k = nxt[s]
            level[s] = _bitlen(t[s] ^ t[k]) if k < n and c[k] == c[s] else None
            assert level[s] is None or level[s] > h
        h += 1
    return {c[s]: val[s] for s in range(n) if s == 0 or c[s - 1] != c[s]}


class _LevelStack:
    """Pending sums of one column by level (carried across the chunks)."""

    def __init__(self, v, last):
        self.top, self.pend, self.last = v, {}, last

    def push(self, v, d):
        for h in sorted(x for x in self.pend if x < d):
            self.top = self.pend.pop(h) + self.top
        self.pend[d] = self.top
        self.top = v

    def finish(self):
        v = self.top
        for h in sorted(self.pend):
            v = self.pend[h] + v
        return v


def _tile_row(lists, a, cap, block):
    """One row as the tile kernel takes it when all of it is one cell: lists
    in blocks of `block`, each block in aligned chunks of at most `cap`
    products (a single list is always a chunk), chunk sums carried per column."""
    L = len(lists)
    pre = np.concatenate(([0], np.cumsum([len(x) for x in lists])))
    if pre[-1] <= cap:
        sums = _rounds_by_level([(t, cc, a[t] * vv) for t in range(L) for cc, vv in lists[t]])
        return sorted(sums.items())
    carried = {}
    levels = block.bit_length() - 1
    for lb in range(0, L, block):
        lbe = min(L, lb + block)
        cur = lb
        while cur < lbe:
            k = levels if cur == lb else min((cur & -cur).bit_length() - 1, levels)
            while k > 0 and pre[min(lbe, cur + (1 << k))] - pre[cur] > cap:
                k -= 1
            te = min(lbe, cur + (1 << k))
            sums = _rounds_by_level([(t, cc, a[t] * vv) for t in range(cur, te) for cc, vv in lists[t]])
            for cc, v in sums.items():
                if cc not in carried:
                    carried[cc] = _LevelStack(v, cur)
                else:
                    st = carried[cc]
                    st.push(v, _bitlen(st.last ^ cur))
                    st.last = cur
            cur = te
    return sorted((cc, st.finish()) for cc, st in carried.items())


def _random_case(seed):
    k = int(I.rand_below(seed, 1, [0], 3)[0])
    L = [3, 37, 300][k]
    ncols = int([4, 40, 200][int(I.rand_below(seed, 2, [0], 3)[0])])
    lens = I.rand_below(seed, 3, np.arange(L), ncols + 1)
    lens[I.rand_unit(seed, 4, np.arange(L)) < 0.2] = 0               # empty lists keep their slot
    rows, cols, vals = [], [], []
    for t in range(L):
        keys = I.rand_u64(seed, 5, t * 4096 + np.arange(ncols))
        cs = np.sort(np.argsort(keys, kind="stable")[:int(lens[t])])
        rows.append(cs)
    B = I.CSR(L, ncols, np.concatenate(([0], np.cumsum([len(r) for r in rows]))).astype(np.int32),
              np.concatenate(rows).astype(np.int32) if sum(map(len, rows)) else np.zeros(0, np.int32),
              None)
    B = I.CSR(B.rows, B.cols, B.rp, B.col, I.rand_sym(seed, 6, np.arange(len(B.col))))
    A = I.CSR(1, L, np.array([0, L], np.int32), np.arange(L, dtype=np.int32), I.rand_sym(seed, 7, np.arange(L)))
    return A, B


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("cap,block", [(1 << 30, 1 << 11), (64, 1 << 11), (16, 8), (5, 4)])
def test_tile_order_equals_algorithm_1(seed, cap, block):
    A, B = _random_case(300 + seed)
    lists = [list(zip(B.col[B.rp[t]:B.rp[t + 1]].tolist(), B.val[B.rp[t]:B.rp[t + 1]].tolist()))
             for t in range(B.rows)]
    got = _tile_row(lists, A.val.tolist(), cap, block)
    ref = oracle.alg1(A, B)
    assert [cc for cc, _ in got] == ref.col.tolist()
    assert [v for _, v in got] == ref.val.tolist()   # bit for bit
