// Long rows by column tiles.
//
// Algorithm 1 fixes the value at column c of a row as the sum of that column's
// products A_it * B_tc over the lists t that hold c, added in the merge tree's
// order: two products of lists t1 < t2 meet in round bitlen(t1 ^ t2) (the first
// round r with t1 >> r == t2 >> r, Fig. 2), the left partial sum first, a list
// without c passing its partner's sum through.  Any procedure that adds each
// column's products in that aligned binary tree gives Algorithm 1's bits,
// whatever order the columns are visited in -- so a long row can be cut into
// column ranges ("tiles") that are reduced independently, each by one thread
// block in shared memory, instead of one block merging the whole row round by
// round through device memory.
//
// Plan (k_tile_plan, one block per long row, index-only work):
//   the row's columns are set in a shared-memory bitmap (one window of 2^20
//   columns of B at a time) and its products counted per cell of 2^sh
//   columns (at most 8192 cells per bitmap window, so a cell is at most 128
//   columns wide).  Consecutive cells are grouped into pieces -- a cut
//   wherever the running product count crosses a multiple of kTilePiece, and
//   before and after every cell of more than kTilePiece products, so that a piece
//   holds fewer than 2 kTilePiece products unless it is a single cell -- and the
//   pieces are packed greedily into tiles of at most kTileP products (a
//   piece of more is a single cell, and a tile of its own).  Every tile
//   records its first column, its products and where its output starts
//   inside the row (distinct columns before it).  The row's length (distinct
//   columns) is the symbolic pass's result.  Consecutive tiles are grouped
//   into spans of at least max(32768, 16 L) products.
// Numeric (k_long_tile, persistent blocks taking spans from a counter):
//   the block keeps one cursor per list of the row (the next position of
//   B_t* not yet consumed, its column, the list's end), found by binary
//   search at the span's first column.  For a tile [c0, c1):
//   1. every list's elements below c1 form its segment (a probe of the next
//      four columns, for four lists at once, then a binary search bounded by
//      c1 - column: B's columns are distinct), segments numbered in list
//      order;
//   2. the products are formed in that order -- position p in list order --
//      with 32-bit keys ((column - c0) << kTilePBits) | p;
//   3. a stable radix sort by column (8-bit digits, as many passes as the
//      tile's columns need) puts every column's products together, still in
//      list order;
//   4. Algorithm 1's merge rounds run on the sorted positions: in round h
//      every live sum takes the next live sum of its column when both have
//      the same t >> h (left first), which is exactly what the rounds do to
//      that column (a list without the column passes its partner through);
//      every position is owned by one thread, which keeps the round in
//      which its sum meets the next one, so a round touches only those
//      sums; the rounds end when no sum can take a partner any more;
//   5. the sums are written, compacted, at the tile's place in C.
//   A hot tile (one cell of at most 128 columns with more than kTileP
//   products) is taken in chunks of aligned list blocks [a 2^k, (a + 1) 2^k)
//   of at most kTileP products: a chunk's sum at a column is the sum of a
//   complete subtree of the merge tree, and the chunks' sums of every column
//   are added by a tree stack per column, carried across the chunks, with
//   the join level of two blocks bitlen(a1 2^k1 ^ a2 2^k2).
// Lists are taken in blocks of kTileSmemL (an aligned subtree): the segment
// search runs block by block, a hot tile is chunked block by block, and a
// row of more than kTileSmemL lists keeps its cursors in the block's slice
// of device memory.
// Limits: at most kTileMaxL lists per row (16-bit list index), B at most
// 2^24 columns; the host keeps the arena merge rounds for other long rows.
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

static_assert(kLsWinBits == kTileBitmapCols, "the plan's bitmap window is the symbolic kernel's");
static_assert(kTileCells % kLsThreads == 0, "plan: whole cells per thread");

// Cell shift for a bitmap window of wn columns: the smallest sh with
// ceil(wn / 2^sh) <= kTileCells.
__host__ __device__ constexpr int tile_cell_shift(int64_t wn) {
    const int b = lb_bitlen((uint64_t)(wn > 1 ? wn - 1 : 0));
    return b > 13 ? b - 13 : 0;
}

// Levels of the tree: two lists t1 < t2 <= kTileMaxL meet at level
// bitlen(t1 ^ t2) in 1 .. 16; a block of kTileSmemL lists spans 11 of them.
constexpr int kTileLevels = 16;
static_assert((1 << kTileLevels) == kTileMaxL + 1, "list levels");
constexpr int kTileChunkLevels = 11;
static_assert((1 << kTileChunkLevels) == kTileSmemL, "a list block is an aligned subtree");
constexpr uint32_t kTileEmpty = 0xffffffffu;   // carried state of a column that has no sum yet
constexpr uint32_t kTilePMask = (1u << kTilePBits) - 1u;
constexpr uint16_t kTileRet = 0x8000u;         // a retired position of the merge rounds
static_assert(kTileP < kTileRet, "positions fit 15 bits");
constexpr int kTileNW = kTileThreads / 32;
// 5-bit fields of the merge rounds' meeting levels, one per owned position
constexpr uint64_t kTileField1 = 0x0000000842108421ull;   // 1 in each of 8 fields
constexpr uint64_t kTileFieldLo = kTileField1 * 15u;        // the low 4 bits of each field
constexpr uint64_t kTileFieldHi = kTileField1 * 16u;        // the top bit of each field
constexpr uint64_t kTileNoMeetAll = kTileField1 * 31u;      // every field 31: no meeting
constexpr int kTileQ = kTileP / kTileThreads;   // sorted positions per thread
static_assert(kTileQ == 8, "eight 5-bit level fields per thread");
static_assert(kTileThreads >= 256 && kTileThreads % 256 == 0, "a radix digit per thread of the first 256");
constexpr int kTileWords = kTileP / 32;            // words of a position bitmap
static_assert(kTileWords % 32 == 0, "whole words per lane");

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kLsThreads, 1) k_tile_plan(RowJob j) {
    extern __shared__ __align__(16) uint32_t bm[];
    uint32_t *hist = bm + kLsWinBits / 32;
    __shared__ int32_t s_q0[kLsThreads];
    __shared__ int32_t s_off[kLsThreads + 1];
    __shared__ int ws[kLsThreads / 32 + 1];
    __shared__ int64_t s_span[2];
    __shared__ int64_t s_nwin;
    constexpr int NT = kLsThreads, PER = kTileCells / NT, K = 8;
    BlockGrp<NT> g;
    g.ws = ws;
    const int tid = (int)threadIdx.x;
    const int64_t ncols = j.bcols;
    for (int r = blockIdx.x; r < j.count; r += gridDim.x) {
        const int row = j.rows[r];
        const RowIn<float> ri = row_in<float>(j, row);
        TileRec *wr = j.tiles + j.tile_base[r];
        const int64_t cap = j.tile_base[r + 1] - j.tile_base[r];
        int64_t count = 0, prod = 0, nwin = 0;
        for (int64_t w0 = 0; w0 < ncols; w0 += kLsWinBits) {
            const uint32_t wn = (uint32_t)(ncols - w0 < kLsWinBits ? ncols - w0 : kLsWinBits);
            const int words = (int)((wn + 31) >> 5);
            const int sh = tile_cell_shift(wn);
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
                                // a column already set needs no atomic (hub
                                // columns recur in many lists)
                                if (!(bm[u >> 5] & (1u << (u & 31)))) atomicOr(&bm[u >> 5], 1u << (u & 31));
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
            // cuts: the first cell, around cells of more than kTilePiece products,
            // and where the running count crosses a multiple of kTilePiece
            unsigned flags = 0;
            int nflag = 0;
            {
                int S = Sx, pc = prevc;
#pragma unroll
                for (int e = 0; e < PER; ++e) {
                    const int d = cb + e;
                    if (d < nc) {
                        const int Sp = S - pc;
                        const bool cut = d == 0 || cp[e] > kTilePiece || pc > kTilePiece || (S / kTilePiece) != (Sp / kTilePiece);
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
            int32_t *Sc = ul + kTileCells + 1;
            int32_t *Dc = Sc + kTileCells + 1;
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
            // tiles: consecutive pieces packed greedily up to kTileP products
            // (a piece of more is one cell and a tile of its own)
            if (tid == 0) {
                int64_t nw = nwin;
                for (int q = 0; q < ftot;) {
                    const int d0 = ul[q];
                    int q1 = q + 1;
                    while (q1 < ftot && Sc[ul[q1 + 1]] - Sc[d0] <= kTileP) ++q1;
                    if (nw < cap) {
                        TileRec rec;
                        rec.c0 = (int32_t)(w0 + ((int64_t)d0 << sh));
                        rec.np = Sc[ul[q1]] - Sc[d0];
                        rec.off = count + Dc[d0];
                        wr[nw] = rec;
                    } else if (j.err != nullptr) {
                        atomicOr(j.err, 2u);   // cannot happen: the capacity bounds the pieces
                    }
                    ++nw;
                    q = q1;
                }
                s_nwin = min(nw, cap);
            }
            g.sync();
            nwin = s_nwin;
            count += totd;
            prod += totp;
            g.sync();   // the cut list is read before the bitmap is cleared again
        }
        if (tid == 0) {
            j.tile_n[r] = (int32_t)nwin;
            j.tile_rownnz[r] = count;
            if (j.out_cnt != nullptr) j.out_cnt[row] = count;
            // spans of consecutive tiles: at least max(kTileSpanMin, 16 L)
            // products each, on average
            const int64_t target = max(kTileSpanMin, (int64_t)kTileSpanPerList * ri.L);
            int64_t nws = prod > 0 ? target * nwin / prod : 1;
            if (nws > nwin) nws = nwin;
            if (nws < 1) nws = 1;
            j.tile_nws[r] = (int32_t)nws;
            int64_t nsp = (nwin + nws - 1) / nws;
            const int64_t scap = tile_span_cap(j.slot_nprod[r]);
            if (nsp > scap) {
                if (j.err != nullptr) atomicOr(j.err, 2u);   // cannot happen: see tile_span_cap
                nsp = scap;
            }
            s_span[0] = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(j.tile_ctr),
                                           (unsigned long long)nsp);
            s_span[1] = nsp;
        }
        g.sync();
        for (int64_t k = tid; k < s_span[1]; k += NT) j.tile_spans[s_span[0] + k] = make_int2(r, (int)k);
        g.sync();
    }
}

// ---------------------------------------------------------------------------
// Numeric pass
// ---------------------------------------------------------------------------

// Tree stack of one column's sums in list order, by level.  The sums added so
// far (lists up to `last`) form partial sums waiting for their right
// neighbours: pend[h] is the one that meets the sums after it at level h (bit
// h of mask), top the most recent one.  The pending levels strictly decrease
// from the oldest sum to the newest, so the mask determines the order.
// Adding a product (or the finished sum of a complete subtree) whose join
// level with the previous one is d first completes every sum below level d
// -- lowest level first, the older (left) sum first -- then parks the result
// at level d.  This performs the additions of Algorithm 1's merge rounds for
// the column in their order.  Pending sums live in memory with a stride
// (the carried stacks of a hot tile's columns).
template <class P, class Ptr>
struct LevelStack {
    using T = typename P::T;
    Ptr pend;          // pend[(h - 1) * stride]
    int stride;
    T top;
    uint32_t mask;
    int last;

    __device__ __forceinline__ void push(T v, int d) {
        d = d < 1 ? 1 : (d > kTileLevels ? kTileLevels : d);   // out of range only for invalid input
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

__device__ __forceinline__ int tile_bitlen(uint32_t x) { return 32 - __clz((int)x); }

// Shared memory of the numeric kernel (one block).  The per-list scratch of
// the segment search (lengths and first positions) borrows the key buffers,
// which the products fill only after it; the merge rounds' links borrow the
// key buffer that does not hold the sorted keys.
template <class P>
struct TileSmem {
    using T = typename P::T;
    static constexpr size_t kCpos = 0;                                              // int32[kTileSmemL]
    static constexpr size_t kCcol = kCpos + 4 * kTileSmemL;                          // int32[kTileSmemL]
    static constexpr size_t kCend = kCcol + 4 * kTileSmemL;                          // int32[kTileSmemL]
    static constexpr size_t kSegQ = kCend + 4 * kTileSmemL;                          // int32[kTileSmemL]
    static constexpr size_t kSegOff = kSegQ + 4 * kTileSmemL;                        // int32[kTileSmemL + 1]
    static constexpr size_t kSegT = align_up(kSegOff + 4 * (kTileSmemL + 1), 16);    // uint16[kTileSmemL]
    static constexpr size_t kBits = align_up(kSegT + 2 * kTileSmemL, 16);            // uint32[kTileP / 32]
    static constexpr size_t kWpre = kBits + 4 * (kTileP / 32);                      // int32[kTileP / 32]
    static constexpr size_t kKeyA = kWpre + 4 * (kTileP / 32);                      // uint32[kTileP]
    static constexpr size_t kKeyB = kKeyA + 4 * kTileP;                             // uint32[kTileP]
    static constexpr size_t kVals = kKeyB + 4 * kTileP;                             // T[kTileP]
    static constexpr size_t kLidx = kVals + sizeof(T) * kTileP;                     // uint16[kTileP]
    static constexpr size_t kCnt = align_up(kLidx + 2 * kTileP, 16);                // uint32[kTileNW][256]
    static constexpr size_t kHTop = align_up(kCnt + 4 * kTileNW * 256, 16);         // T[kTileCellMax]
    static constexpr size_t kHPend = kHTop + sizeof(T) * kTileCellMax;               // T[kTileLevels][kTileCellMax]
    static constexpr size_t kHMask = kHPend + sizeof(T) * kTileLevels * kTileCellMax;   // uint32[kTileCellMax]
    static constexpr size_t kHLast = kHMask + 4 * kTileCellMax;                      // int32[kTileCellMax]
    static constexpr size_t kBytes = align_up(kHLast + 4 * kTileCellMax, 16);
    static_assert(kTileP >= kTileSmemL, "the search scratch of a list block fits a key buffer");
};

// Exclusive prefix sums of (a, b) over the block, totals in (ta, tb).
__device__ __forceinline__ int2 tile_scan2(int a, int b, int &ta, int &tb, int2 *ws) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = a, y = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int ux = __shfl_up_sync(0xffffffffu, x, d);
        const int uy = __shfl_up_sync(0xffffffffu, y, d);
        if (lane >= d) {
            x += ux;
            y += uy;
        }
    }
    if (lane == 31) ws[wid] = make_int2(x, y);
    __syncthreads();
    if (wid == 0) {
        int2 w = lane < kTileNW ? ws[lane] : make_int2(0, 0);
        const int2 w0 = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int ux = __shfl_up_sync(0xffffffffu, w.x, d);
            const int uy = __shfl_up_sync(0xffffffffu, w.y, d);
            if (lane >= d) {
                w.x += ux;
                w.y += uy;
            }
        }
        if (lane < kTileNW) ws[lane] = make_int2(w.x - w0.x, w.y - w0.y);
        if (lane == kTileNW - 1) ws[kTileNW] = w;
    }
    __syncthreads();
    const int2 r = make_int2(ws[wid].x + x - a, ws[wid].y + y - b);
    ta = ws[kTileNW].x;
    tb = ws[kTileNW].y;
    __syncthreads();   // ws may be reused right away
    return r;
}

// One pass of a stable radix sort of n <= kTileP keys by the 8-bit digit at
// `shift`: warp w ranks keys [w * kTileQ * 32, (w + 1) * kTileQ * 32) in
// order -- the lanes with equal digits found by __match_any_sync, the lowest
// of them adding their number to the warp's digit counter; the warp's kTileQ
// steps add in turn (a warp barrier between them), so each step's old value
// counts the equal digits of the steps before it -- the digit
// offsets are laid out digit-major and warp-minor, and every key moves to its
// digit's offset plus its rank.
__device__ __forceinline__ void tile_radix_pass(const uint32_t *src, uint32_t *dst, int n, int shift, uint32_t *cnt,
                                                int *ws) {
    BlockGrp<kTileThreads> g;
    g.ws = ws;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < kTileNW * 256; i += kTileThreads) cnt[i] = 0u;
    __syncthreads();
    uint32_t *wc = cnt + w * 256;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kTileQ];
    int dg[kTileQ], rk[kTileQ], ld[kTileQ];
    unsigned pe[kTileQ];
#pragma unroll
    for (int it = 0; it < kTileQ; ++it) {
        const int idx = w * (32 * kTileQ) + it * 32 + lane;
        const bool ok = idx < n;
        key[it] = ok ? src[idx] : 0u;
        dg[it] = ok ? (int)((key[it] >> shift) & 255u) : 256;
        pe[it] = __match_any_sync(0xffffffffu, dg[it]);
        ld[it] = __ffs(pe[it]) - 1;
    }
#pragma unroll
    for (int it = 0; it < kTileQ; ++it) {
        uint32_t old = 0u;
        if (dg[it] < 256 && lane == ld[it]) old = atomicAdd(&wc[dg[it]], (uint32_t)__popc(pe[it]));
        rk[it] = (int)old;
        __syncwarp();   // orders the steps' adds to a counter
    }
#pragma unroll
    for (int it = 0; it < kTileQ; ++it) rk[it] = __shfl_sync(0xffffffffu, rk[it], ld[it]) + __popc(pe[it] & lt);
    __syncthreads();
    {
        // thread tid < 256 lays out digit tid
        uint32_t c[kTileNW];
        int tot = 0;
#pragma unroll
        for (int v = 0; v < kTileNW; ++v) {
            c[v] = tid < 256 ? cnt[v * 256 + tid] : 0u;
            tot += (int)c[v];
        }
        int all;
        int base = g.scan_excl(tot, all);
        if (tid < 256) {
#pragma unroll
            for (int v = 0; v < kTileNW; ++v) {
                cnt[v * 256 + tid] = (uint32_t)base;
                base += (int)c[v];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kTileQ; ++it)
        if (dg[it] < 256) dst[(int)wc[dg[it]] + rk[it]] = key[it];
    __syncthreads();
}

// Exclusive prefix of the set bits of words [0, nw) of a position bitmap
// (nw <= kTileWords) into pre, by one warp: lane l takes words
// l * kTileWords / 32 .. + kTileWords / 32 - 1.
__device__ __forceinline__ void tile_word_prefix(const uint32_t *bits, int32_t *pre, int nw) {
    constexpr int PW = kTileWords / 32;
    const int lane = threadIdx.x & 31;
    int c[PW], v = 0;
#pragma unroll
    for (int u = 0; u < PW; ++u) {
        const int i = lane * PW + u;
        c[u] = i < nw ? __popc(bits[i]) : 0;
        v += c[u];
    }
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    int ex = incl - v;
#pragma unroll
    for (int u = 0; u < PW; ++u) {
        const int i = lane * PW + u;
        if (i < nw) pre[i] = ex;
        ex += c[u];
    }
}

// What the chunk step of a tile needs (shared memory, the row, the tile).
template <class P>
struct TileCtx {
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    const int32_t *segq, *segoff;
    const uint16_t *segt;
    uint32_t *bits;
    int32_t *wpre;
    uint32_t *keyA, *keyB;
    T *vals;
    uint16_t *lidx;
    uint32_t *cnt;
    T *htop, *hpend;
    uint32_t *hmask;
    int32_t *hlast;
    int *s_int;            // [0] largest column offset
    int *ws;               // block scan scratch
    const In *aval;
    const int32_t *bcol;
    const In *bval;
    uint64_t keep;
    int c0;
    int32_t *ocol;         // the tile's first output
    Out *oval;
    int64_t expect;        // the tile's distinct columns
    unsigned int *err;
};

// A finished sum of column c0 + col: written at the tile's output ridx, or --
// in a hot tile's chunk, whose sum is that of the aligned list block starting
// at tb -- added to the column's carried stack.
template <class P>
__device__ __forceinline__ void tile_emit(const TileCtx<P> &x, bool hot, int tb, int ridx, uint32_t col,
                                          typename P::T v) {
    using T = typename P::T;
    if (!hot) {
        if (ridx < x.expect) {
            __stcs(x.ocol + ridx, (int32_t)(x.c0 + (int)col));
            __stcs(x.oval + ridx, P::fin(v));
        }
        return;
    }
    if (col >= (uint32_t)kTileCellMax) {
        atomicOr(x.err, 2u);   // cannot happen: a hot tile is one cell
        return;
    }
    const uint32_t hm = x.hmask[col];
    if (hm == kTileEmpty) {
        x.htop[col] = v;
        x.hmask[col] = 0u;
    } else {
        LevelStack<P, T *> st{x.hpend + col, kTileCellMax, x.htop[col], hm, 0};
        st.push(v, tile_bitlen((uint32_t)(x.hlast[col] ^ tb)));
        x.htop[col] = st.top;
        x.hmask[col] = st.mask;
    }
    x.hlast[col] = tb;
}

// One chunk of a tile: the products of segments [sa, sb), tile positions
// [pos0, pos0 + n), 0 < n <= kTileP: gather in list order, sort by column,
// add every column's products in tree order, emit.  Called by every thread of
// the block; returns the columns of the chunk.
template <class P>
__device__ int tile_chunk(const TileCtx<P> &x, int sa, int sb, int pos0, int n, bool hot, int tb) {
    using In = typename P::In;
    constexpr unsigned kFull = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // 1. segment starts of the chunk, and the starts before every word
    const int nw = (n + 31) >> 5;
    for (int i = tid; i < nw; i += kTileThreads) x.bits[i] = 0u;
    if (tid == 0) x.s_int[0] = 0;
    __syncthreads();
    for (int s = sa + tid; s < sb; s += kTileThreads) {
        const int st = max(x.segoff[s], pos0) - pos0;
        atomicOr(&x.bits[st >> 5], 1u << (st & 31));
    }
    __syncthreads();
    if (wid == 0) tile_word_prefix(x.bits, x.wpre, nw);
    __syncthreads();
    // 2. the products in list order: key ((column - c0) << kTilePBits) | position
    {
        int q[kTileQ], t[kTileQ];
#pragma unroll
        for (int i = 0; i < kTileQ; ++i) {
            const int p = tid + kTileThreads * i;
            q[i] = -1;
            t[i] = 0;
            if (p < n) {
                const int w = p >> 5;
                const int sg = sa + x.wpre[w] + __popc(x.bits[w] & (kFull >> (31 - (p & 31)))) - 1;
                q[i] = x.segq[sg] + (pos0 + p - x.segoff[sg]);
                t[i] = x.segt[sg];
            }
        }
        int32_t c[kTileQ];
        In v[kTileQ], a[kTileQ];
#pragma unroll
        for (int i = 0; i < kTileQ; ++i) {
            c[i] = 0;
            v[i] = In();
            a[i] = In();
            if (q[i] >= 0) {
                c[i] = ld_keep(x.bcol + q[i], x.keep);
                v[i] = ld_keep(x.bval + q[i], x.keep);
                a[i] = __ldg(x.aval + t[i]);
            }
        }
        uint32_t mx = 0;
#pragma unroll
        for (int i = 0; i < kTileQ; ++i) {
            const int p = tid + kTileThreads * i;
            if (q[i] >= 0) {
                uint32_t co = (uint32_t)(c[i] - x.c0);
                if (co >= (uint32_t)kTileBitmapCols) {
                    atomicOr(x.err, 2u);   // cannot happen: a tile lies inside one bitmap window
                    co = (uint32_t)kTileBitmapCols - 1u;
                }
                x.keyA[p] = (co << kTilePBits) | (uint32_t)p;
                x.vals[p] = P::mul(a[i], v[i]);
                x.lidx[p] = (uint16_t)t[i];
                mx = max(mx, co);
            }
        }
        mx = __reduce_max_sync(kFull, mx);
        if (lane == 0 && mx) atomicMax(reinterpret_cast<unsigned int *>(&x.s_int[0]), mx);
    }
    __syncthreads();
    // 3. stable sort by column: the positions of equal columns stay in list order
    const uint32_t maxco = (uint32_t)x.s_int[0];
    const int cbits = maxco ? tile_bitlen(maxco) : 0;
    uint32_t *src = x.keyA, *dst = x.keyB;
    for (int sh = 0; sh < cbits; sh += 8) {
        tile_radix_pass(src, dst, n, kTilePBits + sh, x.cnt, x.ws);
        uint32_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    const uint32_t *K = src;
    // 4. Algorithm 1's merge rounds on the sorted positions.  Within a column
    // the positions are in list order; after round h - 1 the live sums of a
    // column have distinct t >> (h - 1), t the smallest list of the sum.
    // Round h adds to every live sum the next live sum of its column when
    // both have the same t >> h (the left one first) and retires the right
    // one.  A live sum and its next live sum of the same column therefore
    // meet in round bitlen(t_left ^ t_right), and nothing changes that round
    // before it: the right one can be retired only by its left neighbour, and
    // the left one gets a new neighbour only by taking this one.  Each
    // position keeps that level (31: no next sum in its column) and
    // round h handles just the positions whose level is h; after taking its
    // neighbour, a sum meets the next one in a later round (three live sums
    // of one column cannot share t >> h).  The leftmost sum of a column is
    // never retired: it ends as the column's value.
    uint16_t *nxt = reinterpret_cast<uint16_t *>(dst);           // next live position (kTileRet: retired)
    uint16_t *st = nxt + kTileP;                                  // smallest list of the sum at a position
    uint32_t *rs = x.bits;                                        // run starts, one bit per position
    int32_t *rpre = x.wpre;                                       // run starts before every word
    // thread tid owns positions tid + kTileThreads * i, with their meeting
    // levels in the 5-bit fields of lv; warp w's lanes cover the word i * kTileNW +
    // w of the run-start bitmap
    uint32_t ck[kTileQ];   // the owned sorted keys
#pragma unroll
    for (int i = 0; i < kTileQ; ++i) {
        const int s = tid + kTileThreads * i;
        ck[i] = kKeyPad;
        if (s < n) {
            ck[i] = K[s];
            st[s] = x.lidx[ck[i] & kTilePMask];
            nxt[s] = (uint16_t)(s + 1);
        }
    }
    __syncthreads();
    uint64_t lv = kTileNoMeetAll;
#pragma unroll
    for (int i = 0; i < kTileQ; ++i) {
        const int s = tid + kTileThreads * i;
        bool start = false;
        if (s < n) {
            start = s == 0 || (K[s - 1] >> kTilePBits) != (ck[i] >> kTilePBits);
            if (s + 1 < n && (K[s + 1] >> kTilePBits) == (ck[i] >> kTilePBits)) {
                const uint64_t m = (uint64_t)tile_bitlen((uint32_t)(st[s] ^ st[s + 1]));
                lv = (lv & ~(31ull << (5 * i))) | (m << (5 * i));
            }
        }
        const unsigned b = __ballot_sync(kFull, start);
        if (lane == 0) rs[i * kTileNW + wid] = b;
    }
    __syncthreads();
    if (wid == 0) tile_word_prefix(rs, rpre, kTileWords);
    for (int h = 1; h <= kTileLevels && __syncthreads_or(lv != kTileNoMeetAll); ++h) {
        // owned positions whose level is h: the zero fields of lv ^ h...h
        const uint64_t e = lv ^ (kTileField1 * (uint64_t)h);
        uint64_t z = ~(((e & kTileFieldLo) + kTileFieldLo) | e) & kTileFieldHi;
        while (z) {
            const int bit = __ffsll((long long)z) - 1;
            z &= z - 1u;
            const int i = bit / 5;
            const int s = tid + kTileThreads * i;
            const int j = nxt[s];
            if (j & kTileRet) {   // retired by its left neighbour: it meets nothing any more
                lv |= 31ull << (5 * i);
                continue;
            }
            const uint32_t kss = K[s], kjj = K[j];
            const int ps = (int)(kss & kTilePMask), pj = (int)(kjj & kTilePMask);
            x.vals[ps] = P::add(x.vals[ps], x.vals[pj]);
            const int k = nxt[j];
            nxt[s] = (uint16_t)k;
            nxt[j] = (uint16_t)(k | kTileRet);
            uint64_t m = 31u;
            if (k < n && (K[k] >> kTilePBits) == (kss >> kTilePBits))
                m = (uint64_t)tile_bitlen((uint32_t)(st[s] ^ st[k]));
            lv = (lv & ~(31ull << (5 * i))) | (m << (5 * i));
        }
    }
    __syncthreads();
    // 5. the columns' values: a column's output is the rank of its first position
    const int nruns = rpre[kTileWords - 1] + __popc(rs[kTileWords - 1]);
#pragma unroll
    for (int i = 0; i < kTileQ; ++i) {
        const int s = tid + kTileThreads * i;
        if ((rs[s >> 5] >> (s & 31)) & 1u) {
            const int ridx = rpre[s >> 5] + __popc(rs[s >> 5] & ((1u << (s & 31)) - 1u));
            tile_emit<P>(x, hot, tb, ridx, ck[i] >> kTilePBits, x.vals[ck[i] & kTilePMask]);
        }
    }
    __syncthreads();   // the chunk's buffers are refilled next
    return nruns;
}

__device__ __forceinline__ void tile_prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// First position of B_t*[pos + 1 .. hi) whose column is c1 or more (hi if
// none, also when the range is empty), by binary search.
__device__ __forceinline__ int tile_seg_end(const int32_t *bcol, int pos, int hi, int c1) {
    int lo = pos + 1, h = hi;
    while (lo < h) {
        const int mid = (lo + h) >> 1;
        if (__ldg(bcol + mid) < c1) lo = mid + 1; else h = mid;
    }
    return lo < hi ? lo : hi;
}

template <class P>
__global__ void __launch_bounds__(kTileThreads, 2) k_long_tile(RowJob j) {
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    using S = TileSmem<P>;
    constexpr int NT = kTileThreads;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int ws[kTileNW + 1];
    __shared__ int2 ws2[kTileNW + 1];
    __shared__ int s_int[1];
    __shared__ int s_chunk[4];
    __shared__ unsigned long long s_span;
    const int tid = threadIdx.x;
    int32_t *cpos_s = reinterpret_cast<int32_t *>(sm + S::kCpos);
    int32_t *ccol_s = reinterpret_cast<int32_t *>(sm + S::kCcol);
    int32_t *cend_s = reinterpret_cast<int32_t *>(sm + S::kCend);
    int32_t *segq = reinterpret_cast<int32_t *>(sm + S::kSegQ);
    int32_t *segoff = reinterpret_cast<int32_t *>(sm + S::kSegOff);
    uint16_t *segt = reinterpret_cast<uint16_t *>(sm + S::kSegT);
    int32_t *tlen = reinterpret_cast<int32_t *>(sm + S::kKeyA);   // segment search scratch
    int32_t *tpos = reinterpret_cast<int32_t *>(sm + S::kKeyB);
    BlockGrp<NT> g;
    g.ws = ws;
    const uint64_t keep = l2_keep_policy();
    const unsigned long long nspans = *reinterpret_cast<const unsigned long long *>(j.tile_ctr);
    unsigned long long *taken = reinterpret_cast<unsigned long long *>(j.tile_ctr) + 1;

    TileCtx<P> x;
    x.segq = segq;
    x.segoff = segoff;
    x.segt = segt;
    x.bits = reinterpret_cast<uint32_t *>(sm + S::kBits);
    x.wpre = reinterpret_cast<int32_t *>(sm + S::kWpre);
    x.keyA = reinterpret_cast<uint32_t *>(sm + S::kKeyA);
    x.keyB = reinterpret_cast<uint32_t *>(sm + S::kKeyB);
    x.vals = reinterpret_cast<T *>(sm + S::kVals);
    x.lidx = reinterpret_cast<uint16_t *>(sm + S::kLidx);
    x.cnt = reinterpret_cast<uint32_t *>(sm + S::kCnt);
    x.htop = reinterpret_cast<T *>(sm + S::kHTop);
    x.hpend = reinterpret_cast<T *>(sm + S::kHPend);
    x.hmask = reinterpret_cast<uint32_t *>(sm + S::kHMask);
    x.hlast = reinterpret_cast<int32_t *>(sm + S::kHLast);
    x.s_int = s_int;
    x.ws = ws;
    x.keep = keep;
    x.err = j.err;

    for (;;) {
        if (tid == 0) s_span = atomicAdd(taken, 1ull);
        __syncthreads();
        const unsigned long long s = s_span;
        __syncthreads();
        if (s >= nspans) break;
        const int2 sp = j.tile_spans[s];
        const int r = sp.x, row = j.rows[r];
        const RowIn<In> ri = row_in<In>(j, row);
        const int L = ri.L;
        const int nwin = j.tile_n[r], nws = j.tile_nws[r];
        const int w0 = sp.y * nws, w1 = min(nwin, w0 + nws);
        const TileRec *wr = j.tiles + j.tile_base[r];
        const int64_t rownnz = j.tile_rownnz[r];
        const int64_t obase = j.out_rp[row];
        const int64_t slot = j.out_rp[row + 1] - obase;
        if (sp.y == 0 && tid == 0 && (rownnz > slot || (j.exact && rownnz != slot))) atomicOr(j.err, 1u);
        if (w0 >= w1) continue;
        if (L > kTileMaxL || (L > kTileSmemL && (j.tile_cur == nullptr || L > j.tile_maxL))) {
            if (tid == 0) atomicOr(j.err, 2u);   // cannot happen: the host gives such rows the merge rounds
            continue;
        }
        x.aval = ri.aval;
        x.bcol = ri.bcol;
        x.bval = ri.bval;
        // cursors: in shared memory, or for rows of more lists in this block's
        // slice of device memory
        int32_t *cpos = cpos_s, *ccol = ccol_s, *cend = cend_s;
        if (L > kTileSmemL) {
            int32_t *cg = j.tile_cur + (size_t)blockIdx.x * 3 * (size_t)j.tile_maxL;
            cpos = cg;
            ccol = cg + j.tile_maxL;
            cend = cg + 2 * (size_t)j.tile_maxL;
        }

        // cursors at the span's first column
        const int cstart = wr[w0].c0;
        for (int t = tid; t < L; t += NT) {
            const int k = ri.acol[t];
            int lo = ri.brp[k];
            const int q1 = ri.brp[k + 1];
            int hi = q1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(ri.bcol + mid) < cstart) lo = mid + 1; else hi = mid;
            }
            cpos[t] = lo;
            cend[t] = q1;
            ccol[t] = lo < q1 ? __ldg(ri.bcol + lo) : INT_MAX;
        }
        __syncthreads();

        for (int w = w0; w < w1; ++w) {
            const TileRec rec = wr[w];
            if (rec.np == 0) continue;
            const int c0 = rec.c0;
            const int c1 = w + 1 < nwin ? wr[w + 1].c0 : INT_MAX;
            x.c0 = c0;
            x.ocol = j.out_col + obase + rec.off;
            x.oval = static_cast<Out *>(j.out_val) + obase + rec.off;
            x.expect = (w + 1 < nwin ? wr[w + 1].off : rownnz) - rec.off;
            if (rec.off + x.expect > slot) x.expect = rec.off < slot ? slot - rec.off : 0;   // flagged above
            const bool hot = rec.np > kTileP;
            if (hot)
                for (int c = tid; c < kTileCellMax; c += NT) x.hmask[c] = kTileEmpty;
            // the lists in blocks of kTileSmemL: a tile that fits one sort
            // gathers every block's segments into one table (at most kTileP of
            // them: a segment holds a product), a hot tile takes each block's
            // segments in chunks before the next block
            int tns = 0, tnp = 0;
            for (int lb = 0; lb < L; lb += kTileSmemL) {
                const int lbe = min(L, lb + kTileSmemL);
                const int J = (lbe - lb + NT - 1) / NT;
                const int t0 = min(lbe, lb + tid * J), t1 = min(lbe, t0 + J);
                // 1. every list's segment below c1, numbered in list order; the
                // next four columns of up to four lists are loaded at once
                int ns = 0, np = 0;
                for (int tq = t0; tq < t1; tq += 4) {
                    int cu[4][4], pos[4], hi[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int t = tq + u;
                        pos[u] = -1;
                        hi[u] = 0;
                        if (t < t1) {
                            const int col = ccol[t];
                            if (col < c1) {
                                pos[u] = cpos[t];
                                hi[u] = (int)min((int64_t)cend[t], (int64_t)pos[u] + ((int64_t)c1 - col));
                            }
                        }
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            cu[u][v] = pos[u] >= 0 && pos[u] + 1 + v < hi[u] ? __ldg(ri.bcol + pos[u] + 1 + v)
                                                                            : INT_MAX;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int t = tq + u;
                        if (t < t1) {
                            int len = 0;
                            if (pos[u] >= 0) {
                                const int p = pos[u], end = cend[t];
                                int e = -1, ncol = INT_MAX;
#pragma unroll
                                for (int v = 0; v < 4; ++v)
                                    if (e < 0 && p + 1 + v < hi[u] && cu[u][v] >= c1) {
                                        e = p + 1 + v;
                                        ncol = cu[u][v];
                                    }
                                if (e < 0) {
                                    e = tile_seg_end(ri.bcol, p + 4, hi[u], c1);
                                    ncol = e < end ? __ldg(ri.bcol + e) : INT_MAX;
                                }
                                len = e - p;
                                cpos[t] = e;
                                ccol[t] = ncol;
                                tpos[t - lb] = p;
                                if (e < end) {
                                    // where the list continues: the next tile's probes
                                    // and products, fetched into L2 ahead of them
                                    tile_prefetch_l2(ri.bcol + e);
                                    tile_prefetch_l2(ri.bval + e);
                                }
                            }
                            tlen[t - lb] = len;
                            ns += len > 0 ? 1 : 0;
                            np += len;
                        }
                    }
                }
                int bns, bnp;
                const int2 ex = tile_scan2(ns, np, bns, bnp, ws2);
                const int sbase = hot ? 0 : tns, pbase = hot ? 0 : tnp;
                if (sbase + bns > kTileSmemL) {
                    // cannot happen: the plan's count bounds the segments of a tile that fits one sort
                    if (tid == 0) atomicOr(j.err, 1u);
                    tns = -1;
                    break;
                }
                {
                    int si = sbase + ex.x, po = pbase + ex.y;
                    for (int t = t0; t < t1; ++t) {
                        const int len = tlen[t - lb];
                        if (len > 0) {
                            segq[si] = tpos[t - lb];
                            segoff[si] = po;
                            segt[si] = (uint16_t)t;
                            ++si;
                            po += len;
                        }
                    }
                }
                tns = sbase + bns;
                tnp += bnp;
                if (tid == 0) segoff[tns] = hot ? bnp : tnp;
                __syncthreads();
                if (!hot || bnp == 0) continue;
                // 2. a hot tile: this block's lists in chunks of aligned list
                // blocks, every column's chunk sums added by its carried stack
                int cur = lb;
                while (cur < lbe) {
                    if (tid == 0) {
                        // first segment of a list >= t
                        auto seg_at = [&](int t) {
                            int lo = 0, hi = tns;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if ((int)segt[mid] < t) lo = mid + 1; else hi = mid;
                            }
                            return lo;
                        };
                        int k = cur == lb ? kTileChunkLevels : min(__ffs(cur) - 1, kTileChunkLevels);
                        const int sa = seg_at(cur);
                        int sb = sa;
                        for (;; --k) {
                            sb = seg_at(min(lbe, cur + (1 << k)));
                            if (segoff[sb] - segoff[sa] <= kTileP || k == 0) break;
                        }
                        s_chunk[0] = sa;
                        s_chunk[1] = sb;
                        s_chunk[2] = min(lbe, cur + (1 << k));
                        s_chunk[3] = cur;
                    }
                    __syncthreads();
                    const int sa = s_chunk[0], sb = s_chunk[1], nxt = s_chunk[2], tb = s_chunk[3];
                    const int pos0 = segoff[sa], n = segoff[sb] - pos0;
                    __syncthreads();   // s_chunk is rewritten next
                    if (n > kTileP) {
                        if (tid == 0) atomicOr(j.err, 2u);   // cannot happen: one list holds at most one cell
                    } else if (n > 0) {
                        tile_chunk<P>(x, sa, sb, pos0, n, true, tb);
                    }
                    cur = nxt;
                }
            }
            if (tns < 0) continue;
            if (tid == 0 && tnp != rec.np) atomicOr(j.err, 1u);
            if (!hot) {
                if (tnp > 0) {
                    const int nout = tile_chunk<P>(x, 0, tns, 0, tnp, false, 0);
                    if (tid == 0 && nout != x.expect) atomicOr(j.err, 1u);
                }
                continue;
            }
            // the columns of the cell in order
            __syncthreads();
            bool has = false;
            T v = T();
            if (tid < kTileCellMax) {
                const uint32_t hm = x.hmask[tid];
                has = hm != kTileEmpty;
                if (has) {
                    const LevelStack<P, T *> st{x.hpend + tid, kTileCellMax, x.htop[tid], hm, 0};
                    v = st.finish();
                }
            }
            int tot;
            const int wpos = g.scan_excl(has ? 1 : 0, tot);
            if (has && wpos < x.expect) {
                __stcs(x.ocol + wpos, (int32_t)(c0 + tid));
                __stcs(x.oval + wpos, P::fin(v));
            }
            if (tid == 0 && tot != x.expect) atomicOr(j.err, 1u);
            __syncthreads();
        }
        __syncthreads();   // the cursors are reloaded for the next span
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Blocks of the numeric kernel: every SM's resident blocks.
template <class P>
int tile_grid_t() {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = TileSmem<P>::kBytes;
    if (cudaFuncSetAttribute(k_long_tile<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_long_tile<P>, kTileThreads, sm) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(sms, 1) * std::max(occ, 1);
}

// The long rows of one pass by column tiles: the plan (when this pass makes
// it: the symbolic pass, or BRMerge-Upper's numeric pass), then -- for a
// value pass -- the tiles.
template <class P>
cudaError_t launch_long_tiles(const RowJob &j, cudaStream_t st) {
    cudaError_t e;
    if (j.tile_plan) {
        const size_t smb = (size_t)kLsWinBits / 8 + sizeof(uint32_t) * kTileCells;
        auto kp = k_tile_plan<PIdx>;
        if ((e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(j.tile_ctr, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        kp<<<j.count, kLsThreads, smb, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if constexpr (P::kVal) {
        const size_t sm = TileSmem<P>::kBytes;
        auto kw = k_long_tile<P>;
        if ((e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(j.tile_ctr + 1, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        kw<<<j.tile_grid, kTileThreads, sm, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return cudaGetLastError();
}

}  // namespace brm
