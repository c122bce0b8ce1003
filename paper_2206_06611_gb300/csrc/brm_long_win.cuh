// Long rows by column windows.
//
// Algorithm 1 fixes the value at column c of a row as the sum of that column's
// products A_it * B_tc over the lists t that hold c, added in the merge tree's
// order: two products of lists t1 < t2 meet in round bitlen(t1 ^ t2) (the first
// round r with t1 >> r == t2 >> r, Fig. 2), the left partial sum first, a list
// without c passing its partner's sum through.  Any procedure that adds each
// column's products in that aligned binary tree gives Algorithm 1's bits,
// whatever order the columns are visited in -- so a long row can be cut into
// column ranges ("windows") that are merged independently, each by a warp,
// instead of one thread block merging the whole row round by round.
//
// Plan (k_win_plan, one block per long row, index-only work):
//   the row's columns are set in a shared-memory bitmap (one window of 2^20
//   columns of B at a time) and its products counted per cell of 2^sh
//   columns (at most 8192 cells per bitmap window, so a cell is at most 128
//   columns wide).  Consecutive cells are grouped into windows: a cut
//   wherever the running product count crosses a multiple of kWinH, and
//   before and after every cell of more than kWinH products, so that a window
//   holds fewer than 2 kWinH = kWinP products unless it is a single cell.
//   Every window records its first column, its products and where its
//   output starts inside the row (distinct columns before it).  The row's
//   length (distinct columns) is the symbolic pass's result.  Consecutive
//   windows are grouped into spans of at least max(32768, 16 L) products.
// Numeric (k_long_win, persistent warps taking spans from a counter):
//   a warp keeps one cursor per list of the row (the next position of B_t*
//   not yet consumed, and its column), found by binary search at the span's
//   first column.  For each window [c0, c1) in order it advances every cursor
//   past c1: the elements passed form the list's segment in the window
//   (empty for most lists of a wide row), segments in list order.  The
//   window's products get positions p in segment order, hence in list order,
//   and 32-bit keys ((column - c0) << 10) | p; the warp sorts them in
//   registers (32 lanes x 32 keys, bitonic), and every run of equal columns
//   -- its products in list order -- is reduced with a stack of partial sums
//   whose separating levels bitlen(t_prev ^ t) strictly decrease.  Outputs go
//   compacted to the window's known place in C.  A window of more than kWinP
//   products (a single cell: at most 128 columns) is processed in chunks of
//   kWinP products in list order; every column keeps its stack across the
//   chunks (warp-private scratch in device memory) and is written at the end.
// Limits: at most kWinMaxL lists per row (16-bit list index, stack depth),
// B at most 2^24 columns; the host keeps the arena merge rounds otherwise.
#pragma once

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "brm_engine.cuh"
#include "brm_internal.h"
#include "brm_long_rows.cuh"
#include "brm_reg_rows.cuh"

namespace brm {

static_assert(kLsWinBits == kWinBitmapCols, "the plan's bitmap window is the symbolic kernel's");
static_assert(kWinCells % kLsThreads == 0, "plan: whole cells per thread");

// Rows of at most this many lists keep their cursors in shared memory, longer
// ones in the warp's slice of device memory.
constexpr int kWinSmemL = 256;
// Cursors loaded at once per lane (lists 32 apart).
constexpr int kWinCurU = 4;

// Cell shift for a bitmap window of wn columns: the smallest sh with
// ceil(wn / 2^sh) <= kWinCells.
__host__ __device__ constexpr int win_shift(int64_t wn) {
    const int b = lb_bitlen((uint64_t)(wn > 1 ? wn - 1 : 0));
    return b > 13 ? b - 13 : 0;
}

// Levels of the tree stack: two lists t1 < t2 < 65536 meet at level
// bitlen(t1 ^ t2) in 1 .. 16.
constexpr int kWinLevels = 16;
constexpr uint32_t kWinEmpty = 0xffffffffu;   // carried state of a column that has no product yet

// Per-warp scratch in device memory.  A window of more than kWinP products
// (one cell, at most 128 columns) carries from chunk to chunk, for every
// column, its tree stack (see WinStack): the top partial sum, the mask of
// pending levels (kWinEmpty: no product yet), the last list added, and the
// pending sums by level.  Then every lane's closed groups (see win_replay).
template <class P>
struct WinHot {
    using T = typename P::T;
    static constexpr size_t kTop = 0;                                       // T[128]
    static constexpr size_t kMask = kTop + sizeof(T) * kWinCellMax;         // uint32[128]
    static constexpr size_t kLast = kMask + 4 * kWinCellMax;                // int32[128]
    static constexpr size_t kPend = kLast + 4 * kWinCellMax;                // T[kWinLevels][128]
    static constexpr size_t kClosed = kPend + sizeof(T) * kWinLevels * kWinCellMax;   // T[32][kWinLevels]
    static constexpr size_t kBytes = align_up(kClosed + sizeof(T) * 32 * kWinLevels, 256);
    static_assert(kBytes <= kWinHotBytes, "per-warp hot-window scratch");
};

// Shared memory of one warp of the numeric kernel.  The segment tables are
// read only by the gather; the sorted keys and the lanes' tree stacks
// (two regions per lane: the run in progress, and the piece's first run when
// it continues one from the lane before) are used only after it.
template <class P>
struct WinSmem {
    using T = typename P::T;
    static constexpr size_t kSegB = 0;                                      // int32[kWinP] B position - p
    static constexpr size_t kSegT = kSegB + 4 * kWinP;                      // uint16[kWinP] list index
    static constexpr size_t kBits = align_up(kSegT + 2 * kWinP, 16);        // uint32[32] segment starts
    static constexpr size_t kWpre = kBits + 4 * 32;                         // int32[32] starts before a word
    static constexpr size_t kGatherEnd = kWpre + 4 * 32;
    static constexpr size_t kStage = 0;                                     // uint32[32 x 33] sorted keys
    static constexpr size_t kPend = align_up(4 * 32 * 33, 16);              // T[2][32][kWinLevels]
    static constexpr size_t kRunEnd = kPend + sizeof(T) * 2 * 32 * kWinLevels;
    static constexpr size_t kVals = align_up(kGatherEnd > kRunEnd ? kGatherEnd : kRunEnd, 16);  // T[kWinP]
    static constexpr size_t kLidx = kVals + sizeof(T) * kWinP;              // uint16[kWinP] list of position p
    static constexpr size_t kHead = align_up(kLidx + 2 * kWinP, 16);        // T[32] top, then int4[32]
    static constexpr size_t kHeadI = kHead + sizeof(T) * 32;                // int4: mask, g, closed | whole, last
    static constexpr size_t kCur = align_up(kHeadI + 16 * 32, 16);          // int4[kWinSmemL] list cursors
    static constexpr size_t kBytes = align_up(kCur + 16 * (size_t)kWinSmemL, 16);
};

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kLsThreads, 1) k_win_plan(RowJob j) {
    extern __shared__ __align__(16) uint32_t bm[];
    uint32_t *hist = bm + kLsWinBits / 32;
    __shared__ int32_t s_q0[kLsThreads];
    __shared__ int32_t s_off[kLsThreads + 1];
    __shared__ int ws[kLsThreads / 32 + 1];
    __shared__ int64_t s_span[2];
    constexpr int NT = kLsThreads, PER = kWinCells / NT, K = 8;
    BlockGrp<NT> g;
    g.ws = ws;
    const int tid = (int)threadIdx.x;
    const int64_t ncols = j.bcols;
    for (int r = blockIdx.x; r < j.count; r += gridDim.x) {
        const int row = j.rows[r];
        const RowIn<float> ri = row_in<float>(j, row);
        WinRec *wr = j.win + j.win_base[r];
        const int64_t cap = j.win_base[r + 1] - j.win_base[r];
        int64_t count = 0, prod = 0, nwin = 0;
        for (int64_t w0 = 0; w0 < ncols; w0 += kLsWinBits) {
            const uint32_t wn = (uint32_t)(ncols - w0 < kLsWinBits ? ncols - w0 : kLsWinBits);
            const int words = (int)((wn + 31) >> 5);
            const int sh = win_shift(wn);
            const int nc = (int)(((int64_t)wn + (1 << sh) - 1) >> sh);
            for (int i = tid; i < words; i += NT) bm[i] = 0u;
            for (int i = tid; i < nc; i += NT) hist[i] = 0u;
            g.sync();
            for (int t0 = 0; t0 < ri.L; t0 += NT) {
                const int ncl = min(NT, ri.L - t0);
                const int tot = lb_load_chunk<float, NT>(g, ri, t0, s_q0, s_off, nullptr);
                for (int base = 0; base < tot; base += NT * K) {
                    const int p0 = base + tid * K;
                    if (p0 < tot) {
                        int tl[K], q[K];
                        lb_locate<K>(s_off, s_q0, ncl, tot, p0, tl, q);
                        int32_t c[K];
#pragma unroll
                        for (int k = 0; k < K; ++k) c[k] = q[k] >= 0 ? __ldg(ri.bcol + q[k]) : -1;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const uint32_t u = (uint32_t)((int64_t)c[k] - w0);
                            if (q[k] >= 0 && c[k] >= 0 && u < wn) {
                                atomicOr(&bm[u >> 5], 1u << (u & 31));
                                atomicAdd(&hist[u >> sh], 1u);
                            }
                        }
                    }
                }
                g.sync();
            }
            // products and distinct columns of this thread's cells
            const int cb = tid * PER;
            int cp[PER], cd[PER];
            int sp = 0, sd = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int d = cb + e;
                cp[e] = 0;
                cd[e] = 0;
                if (d < nc) {
                    cp[e] = (int)hist[d];
                    const uint32_t lo = (uint32_t)d << sh, hi = min(lo + (1u << sh), wn);
                    for (uint32_t b = lo; b < hi;) {
                        const uint32_t wi = b >> 5, sb = b & 31, nb = min(32u - sb, hi - b);
                        const uint32_t msk = nb == 32 ? 0xffffffffu : (((1u << nb) - 1u) << sb);
                        cd[e] += __popc(bm[wi] & msk);
                        b += nb;
                    }
                }
                sp += cp[e];
                sd += cd[e];
            }
            const int prevc = (cb > 0 && cb - 1 < nc) ? (int)hist[cb - 1] : 0;
            int totp, totd;
            int Sx = g.scan_excl(sp, totp);
            int Dx = g.scan_excl(sd, totd);
            if (totp == 0) {   // no product of this row falls into this bitmap window
                g.sync();
                continue;
            }
            // cuts: the first cell, around cells of more than kWinH products,
            // and where the running count crosses a multiple of kWinH
            unsigned flags = 0;
            int nflag = 0;
            {
                int S = Sx, pc = prevc;
#pragma unroll
                for (int e = 0; e < PER; ++e) {
                    const int d = cb + e;
                    if (d < nc) {
                        const int Sp = S - pc;
                        const bool cut = d == 0 || cp[e] > kWinH || pc > kWinH || (S / kWinH) != (Sp / kWinH);
                        if (cut) {
                            flags |= 1u << e;
                            ++nflag;
                        }
                    }
                    pc = cp[e];
                    S += cp[e];
                }
            }
            int ftot;
            int fk = g.scan_excl(nflag, ftot);
            g.sync();   // every thread has read the bitmap and the histogram
            // the bitmap's memory now holds the cut list and the cells'
            // exclusive product and distinct-column counts
            int32_t *ul = reinterpret_cast<int32_t *>(bm);
            int32_t *Sc = ul + kWinCells + 1;
            int32_t *Dc = Sc + kWinCells + 1;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int d = cb + e;
                if (d < nc) {
                    Sc[d] = Sx;
                    Dc[d] = Dx;
                    if ((flags >> e) & 1u) ul[fk++] = d;
                }
                Sx += cp[e];
                Dx += cd[e];
            }
            if (tid == 0) {
                ul[ftot] = nc;
                Sc[nc] = totp;
                Dc[nc] = totd;
            }
            g.sync();
            if (nwin + ftot <= cap) {
                for (int q = tid; q < ftot; q += NT) {
                    const int d0 = ul[q], d1 = ul[q + 1];
                    WinRec rec;
                    rec.c0 = (int32_t)(w0 + ((int64_t)d0 << sh));
                    rec.np = Sc[d1] - Sc[d0];
                    rec.off = count + Dc[d0];
                    wr[nwin + q] = rec;
                }
            } else if (tid == 0 && j.err != nullptr) {
                atomicOr(j.err, 2u);   // cannot happen: the capacity bounds the cuts
            }
            nwin = min(nwin + ftot, cap);
            count += totd;
            prod += totp;
            g.sync();   // the cut list is read before the bitmap is cleared again
        }
        if (tid == 0) {
            j.win_n[r] = (int32_t)nwin;
            j.win_rownnz[r] = count;
            if (j.out_cnt != nullptr) j.out_cnt[row] = count;
            // spans of consecutive windows: at least max(kWinSpanMin, 16 L)
            // products each, on average
            const int64_t target = max(kWinSpanMin, (int64_t)kWinSpanPerList * ri.L);
            int64_t nws = prod > 0 ? target * nwin / prod : 1;
            if (nws > nwin) nws = nwin;
            if (nws < 1) nws = 1;
            j.win_nws[r] = (int32_t)nws;
            int64_t nsp = (nwin + nws - 1) / nws;
            const int64_t scap = win_span_cap(j.slot_nprod[r]);
            if (nsp > scap) {
                if (j.err != nullptr) atomicOr(j.err, 2u);   // cannot happen: see win_span_cap
                nsp = scap;
            }
            s_span[0] = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(j.win_ctr),
                                           (unsigned long long)nsp);
            s_span[1] = nsp;
        }
        g.sync();
        for (int64_t k = tid; k < s_span[1]; k += NT) j.win_spans[s_span[0] + k] = make_int2(r, (int)k);
        g.sync();
    }
}

// ---------------------------------------------------------------------------
// Numeric pass
// ---------------------------------------------------------------------------

// Tree stack of one column's products in list order, by level.  The products
// added so far (lists up to `last`) form partial sums waiting for their
// right neighbours: pend[h] is the one that meets the sums after it at level
// h (bit h of mask), top the most recent one.  The pending levels strictly
// decrease from the oldest sum to the newest, so the mask determines the
// order.  Adding a product (or a finished group of them) whose join level
// with the previous one is d first completes every sum below level d --
// lowest level first, the older (left) sum first -- then parks the result at
// level d.  This performs the additions of Algorithm 1's merge rounds for
// the column in their order.  Pending sums live in memory with a stride.
template <class P, class Ptr>
struct WinStack {
    using T = typename P::T;
    Ptr pend;          // pend[(h - 1) * stride]
    int stride;
    T top;
    uint32_t mask;
    int last;

    __device__ __forceinline__ void push(T v, int d) {
        d = d < 1 ? 1 : (d > kWinLevels ? kWinLevels : d);   // out of range only for invalid input
        const uint32_t below = (1u << d) - 1u;
        uint32_t m = mask & below;
        while (m) {
            const int h = __ffs(m) - 1;
            top = P::add(pend[(h - 1) * stride], top);
            m &= m - 1u;
        }
        mask &= ~below;
        pend[(d - 1) * stride] = top;
        mask |= 1u << d;
        top = v;
    }
    __device__ __forceinline__ T finish() const {
        T v = top;
        uint32_t m = mask;
        while (m) {
            const int h = __ffs(m) - 1;
            v = P::add(pend[(h - 1) * stride], v);
            m &= m - 1u;
        }
        return v;
    }
};

// A lane's piece that continues a run from the lane before it cannot add its
// products to the sums before it, but knows the level g at which its first
// product meets the run's previous one.  While the levels it sees stay below
// g it is an ordinary tree stack; when a product arrives whose level d is
// above g, the whole stack would join the sums before it first, so it is
// finished and set aside as a closed group at level g, and the product starts
// a new stack at level d.  The lane that owns the run appends the closed
// groups (at their levels, lowest first) and then the open stack, oldest sum
// first, which repeats the additions of one tree stack fed product by
// product.
template <class P, class PtrA>
__device__ __forceinline__ void win_replay(WinStack<P, PtrA> &acc, const typename P::T *closed, uint32_t cmask,
                                           const typename P::T *pend, uint32_t mask, int g, typename P::T top,
                                           int last) {
    while (cmask) {
        const int h = __ffs(cmask) - 1;
        acc.push(closed[h - 1], h);
        cmask &= cmask - 1u;
    }
    int d = g;
    while (mask) {
        const int h = 31 - __clz(mask);
        acc.push(pend[h - 1], d);
        d = h;
        mask &= ~(1u << h);
    }
    acc.push(top, d);
    acc.last = last;
}

// Segment (index) of window position p: the starts up to p, minus one.
__device__ __forceinline__ int win_seg(const uint32_t *bits, const int32_t *wpre, int p) {
    const uint32_t m = bits[p >> 5] & (0xffffffffu >> (31 - (p & 31)));
    return wpre[p >> 5] + __popc(m) - 1;
}

// What the chunk step of a window needs.
template <class P>
struct WinCtx {
    unsigned char *wb;       // the warp's shared memory (WinSmem layout)
    unsigned char *hs;       // the warp's hot-window scratch
    typename P::T *closed;   // the warp's closed groups: 32 lanes x kWinLevels
    const typename P::In *aval;
    const int32_t *bcol;
    const typename P::In *bval;
    uint64_t keep;
    int c0;
    bool hot;
    int32_t *ocol;           // the window's first output
    typename P::Out *oval;
    int64_t expect;          // the window's distinct columns
};

// A finished run of column c0 + cr: written at output wpos (a window that
// fits one sort), or stored as the column's carried stack (a hot window).
template <class P, class Ptr>
__device__ __forceinline__ void win_emit(const WinCtx<P> &x, uint32_t cr, int64_t wpos, const WinStack<P, Ptr> &st) {
    using T = typename P::T;
    using H = WinHot<P>;
    if (!x.hot) {
        if (wpos < x.expect) {
            __stcs(x.ocol + wpos, (int32_t)(x.c0 + (int)cr));
            __stcs(x.oval + wpos, P::fin(st.finish()));
        }
        return;
    }
    T *gpend = reinterpret_cast<T *>(x.hs + H::kPend) + cr;
    uint32_t m = st.mask;
    while (m) {
        const int h = __ffs(m) - 1;
        gpend[(h - 1) * kWinCellMax] = st.pend[(h - 1) * st.stride];
        m &= m - 1u;
    }
    reinterpret_cast<T *>(x.hs + H::kTop)[cr] = st.top;
    reinterpret_cast<uint32_t *>(x.hs + H::kMask)[cr] = st.mask;
    reinterpret_cast<int32_t *>(x.hs + H::kLast)[cr] = st.last;
}

// One chunk of n products of a window (positions 0 .. n-1 in list order,
// segments recorded in the gather tables): gather the products, sort the
// keys ((column - c0) << 10 | p) in registers, then reduce the runs of equal
// columns.  Lane l reduces sorted positions 32 l .. 32 l + 31 with its tree
// stack; a run that continues into later lanes is finished by the lane where
// it starts, which appends the later lanes' stacks in order.  Returns the
// outputs written (a window that fits one sort).
template <class P>
__device__ __noinline__ int win_chunk(const WinCtx<P> &x, int n, int64_t count) {
    using In = typename P::In;
    using T = typename P::T;
    using S = WinSmem<P>;
    constexpr unsigned kFull = 0xffffffffu;
    constexpr uint32_t PM = (1u << kWinPBits) - 1u;
    const int lane = threadIdx.x & 31;
    int32_t *segb = reinterpret_cast<int32_t *>(x.wb + S::kSegB);
    uint16_t *segt = reinterpret_cast<uint16_t *>(x.wb + S::kSegT);
    uint32_t *bits = reinterpret_cast<uint32_t *>(x.wb + S::kBits);
    int32_t *wpre = reinterpret_cast<int32_t *>(x.wb + S::kWpre);
    uint32_t *stage = reinterpret_cast<uint32_t *>(x.wb + S::kStage);
    T *pendb = reinterpret_cast<T *>(x.wb + S::kPend);
    T *vals = reinterpret_cast<T *>(x.wb + S::kVals);
    uint16_t *lidx = reinterpret_cast<uint16_t *>(x.wb + S::kLidx);
    T *htop = reinterpret_cast<T *>(x.wb + S::kHead);
    int4 *hinfo = reinterpret_cast<int4 *>(x.wb + S::kHeadI);
    // segment starts before every word of the start bitmap
    {
        const int c = __popc(bits[lane]);
        int v = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, v, d);
            if (lane >= d) v += y;
        }
        wpre[lane] = v - c;
    }
    __syncwarp();
    uint32_t key[32];
#pragma unroll
    for (int i0 = 0; i0 < 32; i0 += kRegU) {
        int q[kRegU], t[kRegU];
        In a[kRegU];
#pragma unroll
        for (int u = 0; u < kRegU; ++u) {
            const int p = (i0 + u) * 32 + lane;
            q[u] = -1;
            t[u] = 0;
            a[u] = In();
            if (p < n) {
                const int sg = win_seg(bits, wpre, p);
                q[u] = segb[sg] + p;
                t[u] = segt[sg];
                a[u] = __ldg(x.aval + t[u]);
            }
        }
        int32_t c[kRegU];
        In v[kRegU];
#pragma unroll
        for (int u = 0; u < kRegU; ++u) {
            c[u] = 0;
            v[u] = In();
            if (q[u] >= 0) {
                c[u] = ld_keep(x.bcol + q[u], x.keep);
                v[u] = ld_keep(x.bval + q[u], x.keep);
            }
        }
#pragma unroll
        for (int u = 0; u < kRegU; ++u) {
            const int p = (i0 + u) * 32 + lane;
            key[i0 + u] = kKeyPad;
            if (q[u] >= 0) {
                key[i0 + u] = ((uint32_t)(c[u] - x.c0) << kWinPBits) | (uint32_t)p;
                vals[p] = P::mul(a[u], v[u]);
                lidx[p] = (uint16_t)t[u];
            }
        }
    }
    reg_bitonic_sort<32, 32>(key, lane);
    __syncwarp();   // every lane's gather has read the tables the key tile overwrites
    // lane l holds sorted positions 32 l + i in key[i]; run starts and the
    // runs that cross from one lane into the next
    const uint32_t prv = __shfl_up_sync(kFull, key[31], 1);
    const uint32_t nxt = __shfl_down_sync(kFull, key[0], 1);
    const bool cont_in = lane > 0 && key[0] != kKeyPad && (prv >> kWinPBits) == (key[0] >> kWinPBits);
    const bool cont_out = lane < 31 && key[31] != kKeyPad && nxt != kKeyPad &&
                          (nxt >> kWinPBits) == (key[31] >> kWinPBits);
    int nst = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        stage[i * 33 + lane] = key[i];
        const bool real = key[i] != kKeyPad;
        const bool start = real && (i == 0 ? !cont_in : (key[i] >> kWinPBits) != (key[i - 1] >> kWinPBits));
        nst += start ? 1 : 0;
    }
    int base = nst;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, base, d);
        if (lane >= d) base += y;
    }
    const int total = __shfl_sync(kFull, base, 31);
    base = base - nst;
    __syncwarp();

    // this lane's piece, position by position: runs that start here are
    // reduced in pendR (a hot window's continuing from the column's carried
    // stack); a first run that continues one from the lane before, in pendH
    // with closed groups (see win_replay)
    using H = WinHot<P>;
    T *pendR = pendb + lane * kWinLevels, *pendH = pendb + (32 + lane) * kWinLevels;
    T *closedL = x.closed + lane * kWinLevels;
    int g0 = 0;
    if (cont_in) g0 = 32 - __clz((int)lidx[prv & PM] ^ (int)lidx[key[0] & PM]);
    WinStack<P, T *> st{pendR, 1, T(), 0u, 0};
    uint32_t cc = kKeyPad;   // column of the run in progress
    int done = 0, g = 0;
    uint32_t cmask = 0;
    bool head = false;
    for (int i = 0; i < 32; ++i) {
        const uint32_t k = stage[i * 33 + lane];
        if (k == kKeyPad) break;
        const uint32_t c = k >> kWinPBits;
        const int p = (int)(k & PM);
        const T v = vals[p];
        const int t = lidx[p];
        if (c != cc) {
            if (cc != kKeyPad) {
                if (head) {
                    htop[lane] = st.top;
                    hinfo[lane] = make_int4((int)st.mask, g, (int)cmask, st.last);
                } else {
                    win_emit<P>(x, cc, count + base + done, st);
                    ++done;
                }
            }
            head = i == 0 && cont_in;
            cc = c;
            if (head) {
                st.pend = pendH;
                st.top = v;
                st.mask = 0u;
                st.last = t;
                g = g0;
                cmask = 0u;
            } else {
                st.pend = pendR;
                const uint32_t gm = x.hot ? reinterpret_cast<const uint32_t *>(x.hs + H::kMask)[c] : kWinEmpty;
                if (gm != kWinEmpty) {
                    // the column's stack from the chunks before
                    const T *gpend = reinterpret_cast<const T *>(x.hs + H::kPend) + c;
                    uint32_t m = gm;
                    while (m) {
                        const int h = __ffs(m) - 1;
                        pendR[h - 1] = gpend[(h - 1) * kWinCellMax];
                        m &= m - 1u;
                    }
                    st.top = reinterpret_cast<const T *>(x.hs + H::kTop)[c];
                    st.mask = gm;
                    st.last = reinterpret_cast<const int32_t *>(x.hs + H::kLast)[c];
                    st.push(v, 32 - __clz(st.last ^ t));
                    st.last = t;
                } else {
                    st.top = v;
                    st.mask = 0u;
                    st.last = t;
                }
            }
        } else if (head) {
            const int d = 32 - __clz(st.last ^ t);
            if (d < g) {
                st.push(v, d);
            } else {
                closedL[g - 1] = st.finish();
                cmask |= 1u << g;
                st.top = v;
                st.mask = 0u;
                g = d;
            }
            st.last = t;
        } else {
            st.push(v, 32 - __clz(st.last ^ t));
            st.last = t;
        }
    }
    // the last run of the piece: finished here, or continued by the next lanes
    bool own_tail = false;
    if (cc != kKeyPad) {
        if (head) {
            htop[lane] = st.top;
            hinfo[lane] = make_int4((int)st.mask, g, (int)(cmask | (cont_out ? 0x80000000u : 0u)), st.last);
        } else if (cont_out) {
            own_tail = true;
        } else {
            win_emit<P>(x, cc, count + base + done, st);
            ++done;
        }
    }
    __syncwarp();   // every lane's first-run stack is published
    if (own_tail) {
        for (int l = lane + 1; l < 32; ++l) {
            const int4 hi = hinfo[l];
            const uint32_t cm = (uint32_t)hi.z;
            win_replay<P>(st, x.closed + l * kWinLevels, cm & 0x7fffffffu, pendb + (32 + l) * kWinLevels,
                          (uint32_t)hi.x, hi.y, htop[l], hi.w);
            if (!(cm >> 31)) break;
        }
        win_emit<P>(x, cc, count + base + done, st);
        ++done;
    }
    __syncwarp();   // the chunk's buffers are refilled next
    bits[lane] = 0u;
    __syncwarp();
    return x.hot ? 0 : total;
}

template <class P>
__global__ void __launch_bounds__(kWinWarps * 32) k_long_win(RowJob j) {
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    using S = WinSmem<P>;
    using H = WinHot<P>;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *wb = smem + (size_t)wid * S::kBytes;
    int32_t *segb = reinterpret_cast<int32_t *>(wb + S::kSegB);
    uint16_t *segt = reinterpret_cast<uint16_t *>(wb + S::kSegT);
    uint32_t *bits = reinterpret_cast<uint32_t *>(wb + S::kBits);
    const int64_t gw = (int64_t)blockIdx.x * kWinWarps + wid;
    int4 *cur_g = j.win_cur + gw * (int64_t)j.win_maxL;
    int4 *cur_s = reinterpret_cast<int4 *>(wb + S::kCur);
    unsigned char *hs = reinterpret_cast<unsigned char *>(j.win_hot) + gw * (int64_t)H::kBytes;
    const uint64_t keep = l2_keep_policy();
    const unsigned lt = (1u << lane) - 1u;
    const unsigned long long nspans = *reinterpret_cast<const unsigned long long *>(j.win_ctr);
    unsigned long long *taken = reinterpret_cast<unsigned long long *>(j.win_ctr) + 1;

    for (;;) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(taken, 1ull);
        s = __shfl_sync(kFull, s, 0);
        if (s >= nspans) break;
        const int2 sp = j.win_spans[s];
        const int r = sp.x, row = j.rows[r];
        const RowIn<In> ri = row_in<In>(j, row);
        const int L = ri.L;
        const int nwin = j.win_n[r], nws = j.win_nws[r];
        const int w0 = sp.y * nws, w1 = min(nwin, w0 + nws);
        const WinRec *wr = j.win + j.win_base[r];
        const int64_t rownnz = j.win_rownnz[r];
        const int64_t obase = j.out_rp[row];
        const int64_t slot = j.out_rp[row + 1] - obase;
        if (sp.y == 0 && lane == 0 && (rownnz > slot || (j.exact && rownnz != slot))) atomicOr(j.err, 1u);
        int32_t *ocol = j.out_col + obase;
        Out *oval = static_cast<Out *>(j.out_val) + obase;
        if (w0 >= w1) continue;

        // cursors at the span's first column (position, end of the list, the
        // column at the position or INT_MAX); lane l owns lists l, l + 32, ...
        int4 *cur = L <= kWinSmemL ? cur_s : cur_g;
        const int cstart = wr[w0].c0;
        for (int t = lane; t < L; t += 32) {
            const int k = ri.acol[t];
            int lo = ri.brp[k];
            const int q1 = ri.brp[k + 1];
            int hi = q1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(ri.bcol + mid) < cstart) lo = mid + 1; else hi = mid;
            }
            cur[t] = make_int4(lo, q1, lo < q1 ? __ldg(ri.bcol + lo) : INT_MAX, 0);
        }

        for (int w = w0; w < w1; ++w) {
            const WinRec rec = wr[w];
            if (rec.np == 0) continue;
            const int c0 = rec.c0;
            const int c1 = w + 1 < nwin ? wr[w + 1].c0 : INT_MAX;
            const int64_t expect = (w + 1 < nwin ? wr[w + 1].off : rownnz) - rec.off;
            const bool hot = rec.np > kWinP;
            if (hot) {
                uint32_t *gmask = reinterpret_cast<uint32_t *>(hs + H::kMask);
                for (int c = lane; c < kWinCellMax; c += 32) gmask[c] = kWinEmpty;
            }
            int64_t count = 0;   // outputs written
            int fill = 0, nseg = 0;
            bits[lane] = 0u;
            __syncwarp();
            const WinCtx<P> cx{wb, hs, reinterpret_cast<T *>(hs + H::kClosed), ri.aval, ri.bcol, ri.bval, keep, c0,
                               hot, ocol + rec.off, oval + rec.off, expect};

            // segments: every list's elements in [c0, c1), in list order;
            // kWinCurU cursors per lane are loaded before any is used
            for (int tb = 0; tb < L; tb += 32 * kWinCurU) {
                int4 cs[kWinCurU];
#pragma unroll
                for (int u = 0; u < kWinCurU; ++u) {
                    const int t = tb + 32 * u + lane;
                    cs[u] = t < L ? cur[t] : make_int4(0, 0, INT_MAX, 0);
                }
#pragma unroll
                for (int u = 0; u < kWinCurU; ++u) {
                    const int t = tb + 32 * u + lane;
                    if (!__any_sync(kFull, cs[u].z < c1)) continue;
                    int q = 0, len = 0;
                    if (cs[u].z < c1) {
                        int e = cs[u].x + 1, nx = INT_MAX;
                        while (e < cs[u].y) {
                            const int cc = __ldg(ri.bcol + e);
                            if (cc >= c1) {
                                nx = cc;
                                break;
                            }
                            ++e;
                        }
                        q = cs[u].x;
                        len = e - cs[u].x;
                        cur[t] = make_int4(e, cs[u].y, nx, 0);
                    }
                    while (__any_sync(kFull, len > 0)) {
                        int xs = len;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const int y = __shfl_up_sync(kFull, xs, d);
                            if (lane >= d) xs += y;
                        }
                        const int tot = __shfl_sync(kFull, xs, 31);
                        const int ex = xs - len;
                        const int room = kWinP - fill;
                        const int take = max(0, min(len, room - ex));
                        const unsigned tm = __ballot_sync(kFull, take > 0);
                        if (take > 0) {
                            const int sg = nseg + __popc(tm & lt);
                            const int p0 = fill + ex;
                            segb[sg] = q - p0;
                            segt[sg] = (uint16_t)t;
                            atomicOr(&bits[p0 >> 5], 1u << (p0 & 31));
                        }
                        nseg += __popc(tm);
                        fill += min(tot, room);
                        q += take;
                        len -= take;
                        __syncwarp();
                        if (fill == kWinP && (hot || __any_sync(kFull, len > 0))) {
                            count += win_chunk<P>(cx, fill, count);
                            fill = 0;
                            nseg = 0;
                        }
                    }
                }
            }
            if (fill > 0) count += win_chunk<P>(cx, fill, count);

            if (hot) {
                // every present column of the cell, in column order
                __syncwarp();
                T *gtop = reinterpret_cast<T *>(hs + H::kTop);
                uint32_t *gmask = reinterpret_cast<uint32_t *>(hs + H::kMask);
                T *gpend = reinterpret_cast<T *>(hs + H::kPend);
                for (int cb = 0; cb < kWinCellMax; cb += 32) {
                    const int c = cb + lane;
                    const uint32_t gm = gmask[c];
                    const bool has = gm != kWinEmpty;
                    T v = T();
                    if (has) {
                        const WinStack<P, T *> g{gpend + c, kWinCellMax, gtop[c], gm, 0};
                        v = g.finish();
                    }
                    const unsigned msk = __ballot_sync(kFull, has);
                    if (has) {
                        const int64_t wpos = count + __popc(msk & lt);
                        if (wpos < expect) {
                            __stcs(ocol + rec.off + wpos, (int32_t)(c0 + c));
                            __stcs(oval + rec.off + wpos, P::fin(v));
                        }
                    }
                    count += __popc(msk);
                }
                __syncwarp();
            }
            if (lane == 0 && count != expect) atomicOr(j.err, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Blocks of the numeric kernel: every SM's resident blocks (the per-warp
// scratch is allocated for exactly this many).
template <class P>
int win_grid_t() {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = kWinWarps * WinSmem<P>::kBytes;
    if (cudaFuncSetAttribute(k_long_win<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_long_win<P>, kWinWarps * 32, sm) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(sms, 1) * std::max(occ, 1);
}

// The long rows of one pass by column windows: the plan (when this pass makes
// it: the symbolic pass, or BRMerge-Upper's numeric pass), then -- for a
// value pass -- the windows.
template <class P>
cudaError_t launch_long_win(const RowJob &j, cudaStream_t st) {
    cudaError_t e;
    if (j.win_plan) {
        const size_t smb = (size_t)kLsWinBits / 8 + sizeof(uint32_t) * kWinCells;
        auto kp = k_win_plan<PIdx>;
        if ((e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(j.win_ctr, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        kp<<<j.count, kLsThreads, smb, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if constexpr (P::kVal) {
        const size_t sm = kWinWarps * WinSmem<P>::kBytes;
        auto kw = k_long_win<P>;
        if ((e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(j.win_ctr + 1, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        kw<<<j.win_grid, kWinWarps * 32, sm, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return cudaGetLastError();
}

// Bytes of the per-warp scratch of the numeric kernel.
template <class P>
__host__ __device__ constexpr size_t win_hot_bytes() { return WinHot<P>::kBytes; }

}  // namespace brm
