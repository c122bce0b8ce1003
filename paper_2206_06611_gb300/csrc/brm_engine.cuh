// BRMerge row engine for sm_103a.
//
// One output row C_i* = sum over k in A_i* of A_ik * B_k* (Eq. 2) is built the
// way Algorithm 1 builds it:
//   * multiplying phase: the scaled rows A_ik * B_k* are written one after the
//     other, in the order of A_i*, into the "ping" buffer; the end of each list
//     is recorded in a list-offset array -- also for an empty B_k*, so that an
//     empty list keeps its place in the tree;
//   * accumulating phase: while more than one list is left, lists (0,1), (2,3),
//     ... are merged like merge sort, equal columns added once, a last odd list
//     copied; the merged lists go to the other buffer and the buffers swap
//     roles (ceil(log2 L) rounds, Fig. 2).
// A row is processed by a cooperating thread group (a warp or a thread block)
// instead of one CPU thread.  Each merging round is split over the group by
// merge path: the concatenation of all merged pairs is cut into tiles of
// G::N * K output positions ("diagonals"), thread t owns K consecutive
// diagonals, locates the pair and the co-rank (how many elements of the left
// list precede its first diagonal) by binary search, merges its K steps in
// registers and writes them after a group prefix sum of the element counts
// (equal columns make one element out of two diagonals).  The result of every
// merge -- and therefore every floating-point sum -- is exactly the one of the
// sequential algorithm: the same pairs are merged, and the values of two
// equal columns are added once, left list's value first.
//
// Buffers are plain pointers, so the same code runs on shared memory (warp and
// block kernels) and on the device-memory arena (long rows).  In the arena a
// round goes tile by tile through shared memory instead (merge_round_tiled):
// the same merge, with the searches in device memory done once per tile end
// rather than once per thread.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace brm {

constexpr int32_t kColEnd = 0x7fffffff;   // larger than any column index (< 2^31 - 1)

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// Value policies.  Products are rounded before any addition and additions are
// never contracted into an FMA (explicit _rn intrinsics).
// ---------------------------------------------------------------------------
struct PF64 {
    using In = double; using T = double; using Out = double;
    static constexpr bool kVal = true;
    static constexpr bool kPerm = false;
    __device__ static __forceinline__ T mul(In a, In b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ T add(T x, T y) { return __dadd_rn(x, y); }
    __device__ static __forceinline__ Out fin(T x) { return x; }
};

struct PF32 {
    using In = float; using T = float; using Out = float;
    static constexpr bool kVal = true;
    static constexpr bool kPerm = false;
    __device__ static __forceinline__ T mul(In a, In b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ T add(T x, T y) { return __fadd_rn(x, y); }
    __device__ static __forceinline__ Out fin(T x) { return x; }
};

// FP32 with TwoSum-compensated merge additions: an element is (s, e), a
// product starts as (a*b, 0); adding (x, y) gives s = fl(x.s + y.s), t the
// exact rounding error of that sum (Knuth's TwoSum, TAOCP vol. 2, 4.2.2),
// e = fl(fl(x.e + y.e) + t).  The stored value is fl(s + e).
struct PF32C {
    using In = float; using T = float2; using Out = float;
    static constexpr bool kVal = true;
    static constexpr bool kPerm = false;
    __device__ static __forceinline__ T mul(In a, In b) { return make_float2(__fmul_rn(a, b), 0.0f); }
    __device__ static __forceinline__ T add(T x, T y) {
        const float s = __fadd_rn(x.x, y.x);
        const float bb = __fsub_rn(s, x.x);
        const float t = __fadd_rn(__fsub_rn(x.x, __fsub_rn(s, bb)), __fsub_rn(y.x, bb));
        return make_float2(s, __fadd_rn(__fadd_rn(x.y, y.y), t));
    }
    __device__ static __forceinline__ Out fin(T x) { return __fadd_rn(x.x, x.y); }
};

// Column indices only (the symbolic pass of BRMerge-Precise).
struct PIdx {
    using In = float; using T = float; using Out = float;   // never loaded or stored
    static constexpr bool kVal = false;
    static constexpr bool kPerm = false;
    __device__ static __forceinline__ T mul(In, In) { return 0.0f; }
    __device__ static __forceinline__ T add(T, T) { return 0.0f; }
    __device__ static __forceinline__ Out fin(T) { return 0.0f; }
};

// The symbolic pass that also records, for every register-bin row, the order
// in which its merge tree leaves the products: their positions sorted by
// (column, list), with the start of every run of equal columns marked.
struct PPerm : PIdx {
    static constexpr bool kPerm = true;
};

// Entries of a recorded row order (one 16-bit word per product).
constexpr uint32_t kPermPos = 0x03ffu;     // the product's position in the row (< 1024)
constexpr uint32_t kPermStart = 0x8000u;   // first element of a run of equal columns
constexpr uint32_t kPermMulti = 0x4000u;   // ... of a run of two or more elements

// ---------------------------------------------------------------------------
// Thread groups.
// ---------------------------------------------------------------------------
struct WarpGrp {
    static constexpr int N = 32;
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    // exclusive prefix sum of x over the group; total = sum over the group
    __device__ __forceinline__ int scan_excl(int x, int &total) const {
        const int lane = threadIdx.x & 31;
        int v = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        total = __shfl_sync(0xffffffffu, v, 31);
        return v - x;
    }
};

template <int NT>
struct BlockGrp {
    static constexpr int N = NT;
    static constexpr int NW = NT / 32;
    int *ws;   // shared scratch of NW + 1 ints
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int scan_excl(int x, int &total) const {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int v = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) ws[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = lane < NW ? ws[lane] : 0;
            const int w0 = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            if (lane < NW) ws[lane] = w - w0;
            if (lane == NW - 1) ws[NW] = w;
        }
        __syncthreads();
        const int r = ws[wid] + v - x;
        total = ws[NW];
        __syncthreads();   // ws may be reused right away
        return r;
    }
};

// A ping or pong buffer: parallel column / value arrays (the paper's buffers
// hold (col, val) pairs) and the list-offset array.
template <class P>
struct Buf {
    int32_t *col;
    typename P::T *val;
    int32_t *off;
};

// One product of a batch (a device-side table; see brm_spgemm_batched): its
// A and B and the first row of its block in the stacked row space.
struct ProdDesc {
    const int32_t *arp, *acol; const void *aval;
    const int32_t *brp, *bcol; const void *bval;
    int64_t row0;
};

// Everything a row kernel reads and writes.
struct RowJob {
    // batched products: row ids are rows of the stacked product and each row
    // finds its own A and B through prod_of / prods (null: one product)
    const ProdDesc *prods;
    const int32_t *prod_of;
    const int32_t *arp, *acol; const void *aval;
    const int32_t *brp, *bcol; const void *bval;
    const int32_t *rows;        // row ids of this bin (or batch)
    int32_t count;              // number of rows in the list
    const int64_t *out_rp;      // numeric: where row i starts in out_col/out_val
    int32_t *out_col;
    void *out_val;
    int64_t *out_cnt;           // optional: receives each row's length
    unsigned int *err;          // set to 1 if a row's length disagrees with its slot
    int32_t exact;              // 1: a numeric row must fill its slot exactly (Precise)
    int32_t reg_keys;           // register bins: keys per thread (8, 16 or 32)
    int32_t reg_warps;          // register bins: warps per block
    int32_t sym_hash;           // register bins, symbolic pass: 1 = count by hashing, 0 = by sorting
    // register bins: the rows' recorded orders (written by the symbolic pass,
    // applied by the numeric pass); null: the numeric pass sorts by itself
    uint16_t *perm;
    const int64_t *perm_off;    // per row: where its order starts in perm
    int32_t num_half;           // numeric from a recorded order: half the keys, twice the threads
    int32_t num_direct;         // numeric from a recorded order, 32-key rows: products read from B directly
    // long rows only: 1 = column buckets (brm_long_rows.cuh), 0 = merge
    // rounds in the arena; B's column count (the largest of a batch); per
    // slot, the arena offset (bytes) and the product count
    int32_t long_bucket;
    int64_t bcols;
    // numeric bucket kernels: the batch's work list (lb_cap records), its two
    // counters (records written, records taken) and the giant-column slots
    void *lb_work;
    int32_t *lb_ctr;
    void *lb_slots;
    int64_t lb_cap;
    char *arena;
    const int64_t *arena_off;
    const int64_t *slot_nprod;
    // merge rounds in the arena: long_grid > 0 launches that many persistent
    // blocks; block b takes slot b, then slots long_grid, long_grid + 1, ...
    // from the counter (zero at launch), in the arena at arena_off[b]
    int32_t *long_ctr;
    int32_t long_grid;
    // long rows by column tiles (brm_long_tiles.cuh): per long slot, where its
    // tiles start (count + 1 entries), how many it has, tiles per span, the
    // row's distinct columns; the span list and its two counters (spans
    // written, spans taken); per block of the numeric kernel, cursors for the
    // rows of more than kTileSmemL lists (3 x tile_maxL ints, or null)
    struct TileRec *tiles;
    const int64_t *tile_base;
    int32_t *tile_n;
    int32_t *tile_nws;
    int64_t *tile_rownnz;
    int2 *tile_spans;
    unsigned long long *tile_ctr;
    int32_t *tile_cur;
    int32_t tile_maxL;
    int32_t tile_grid;       // persistent blocks of the numeric kernel
    int32_t tile_plan;       // 1: this pass computes the plan first (symbolic pass, or Upper)
};

// The inputs one output row needs: its row of A (columns and values from the
// row's first entry on, L entries) and B.
template <class In>
struct RowIn {
    const int32_t *acol;
    const In *aval;
    const int32_t *brp, *bcol;
    const In *bval;
    int L;
};

template <class In>
__device__ __forceinline__ RowIn<In> row_in(const RowJob &j, int row) {
    const int32_t *arp = j.arp, *acol = j.acol, *brp = j.brp, *bcol = j.bcol;
    const void *aval = j.aval, *bval = j.bval;
    int i = row;
    if (j.prods != nullptr) {
        const ProdDesc &d = j.prods[j.prod_of[row]];
        arp = d.arp; acol = d.acol; aval = d.aval;
        brp = d.brp; bcol = d.bcol; bval = d.bval;
        i = row - (int)d.row0;
    }
    const int a0 = arp[i];
    RowIn<In> r;
    r.acol = acol + a0;
    r.aval = static_cast<const In *>(aval) + a0;
    r.brp = brp;
    r.bcol = bcol;
    r.bval = static_cast<const In *>(bval);
    r.L = arp[i + 1] - a0;
    return r;
}

// Largest t in [0, L) with off[t] <= p (off non-decreasing, off[0] = 0 <= p).
__device__ __forceinline__ int find_last_le(const int32_t *off, int L, int p) {
    int lo = 0, hi = L - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Multiplying phase.  Fills b.off[0..L] and the N products; returns N.
// First every list's descriptor is read once (k = A's column, the start of
// B_k* and its length, A_ik) with one thread per list, and the list ends are
// prefix-summed; the descriptors are parked in the other buffer (`spare`,
// unused until the first merge).  Then every thread gathers UNR products at
// a time -- positions p, p + G, p + 2G, ... so that a group reads a B row
// with consecutive threads -- issuing all loads before using any.
// ---------------------------------------------------------------------------
template <class P, class G, int UNR>
__device__ __forceinline__ int multiply_phase(const G &g, int L, const int32_t *__restrict__ acol,
                                              const typename P::In *__restrict__ aval,
                                              const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                                              const typename P::In *__restrict__ bval, const Buf<P> b,
                                              const Buf<P> spare) {
    using In = typename P::In;
    int32_t *q0s = spare.off;                                   // L entries
    In *as = reinterpret_cast<In *>(spare.val);                 // L entries (capacity >= L)
    int carry = 0;
    if (g.rank() == 0) b.off[0] = 0;
    for (int base = 0; base < L; base += G::N) {
        const int t = base + g.rank();
        int len = 0;
        if (t < L) {
            const int k = acol[t];
            const int q0 = brp[k];
            len = brp[k + 1] - q0;
            q0s[t] = q0;
            if constexpr (P::kVal) as[t] = aval[t];
        }
        int tot;
        const int ex = g.scan_excl(len, tot);
        if (t < L) b.off[t + 1] = carry + ex + len;
        carry += tot;
    }
    g.sync();
    const int N = carry;
    for (int base = 0; base < N; base += G::N * UNR) {
        int q[UNR];
        In a[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int p = base + u * G::N + g.rank();
            q[u] = -1;
            if (p < N) {
                const int t = find_last_le(b.off, L, p);
                q[u] = q0s[t] + (p - b.off[t]);
                if constexpr (P::kVal) a[u] = as[t];
            }
        }
        int32_t c[UNR];
        In v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (q[u] >= 0) {
                c[u] = __ldg(bcol + q[u]);
                if constexpr (P::kVal) v[u] = __ldg(bval + q[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int p = base + u * G::N + g.rank();
            if (q[u] >= 0) {
                b.col[p] = c[u];
                if constexpr (P::kVal) b.val[p] = P::mul(a[u], v[u]);
            }
        }
    }
    g.sync();
    return N;
}

// ---------------------------------------------------------------------------
// Where a merging round puts its output.
//   BufSink   the other ping-pong buffer, with the new list offsets;
//   OutSink   the row's slot in C (or C_bar) -- the last round of a numeric
//             pass writes its single list there directly;
//   CountSink nowhere -- the last round of the symbolic pass only counts.
// ---------------------------------------------------------------------------
template <class P>
struct BufSink {
    Buf<P> d;
    static constexpr bool kOffsets = true;
    __device__ __forceinline__ void put(int w, int32_t c, typename P::T v) const {
        d.col[w] = c;
        if constexpr (P::kVal) d.val[w] = v;
    }
};

template <class P>
struct OutSink {
    int32_t *col;
    typename P::Out *val;
    int cap;
    static constexpr bool kOffsets = false;
    __device__ __forceinline__ void put(int w, int32_t c, typename P::T v) const {
        if (w < cap) {
            col[w] = c;
            val[w] = P::fin(v);
        }
    }
};

template <class P>
struct CountSink {
    static constexpr bool kOffsets = false;
    __device__ __forceinline__ void put(int, int32_t, typename P::T) const {}
};

// ---------------------------------------------------------------------------
// One merging round: nl lists in s -> ceil(nl/2) lists in d.
// ---------------------------------------------------------------------------
template <class P, class G, int K, class Sink>
__device__ __forceinline__ int merge_round(const G &g, int nl, const Buf<P> s, const Sink &sink) {
    using T = typename P::T;
    const int N = s.off[nl];
    const int np = (nl + 1) >> 1;
    int base = 0;
    for (int tile = 0; tile < N; tile += G::N * K) {
        const int d0 = tile + g.rank() * K;
        const int end = min(d0 + K, N);
        int cnt = 0;
        unsigned vmask = 0;
        int32_t oc[K];
        T ov[K];
        int mfirst = 0, mlast = -1;
        if (d0 < N) {
            // the pair whose diagonals contain d0: the last one starting at or before it
            int lo = 0, hi = np - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s.off[2 * mid] <= d0) lo = mid; else hi = mid - 1;
            }
            int m = lo;
            int xi = s.off[2 * m], xlim = s.off[2 * m + 1];
            int yj = xlim, ylim = (2 * m + 2 <= nl) ? s.off[2 * m + 2] : xlim;
            const int dd = d0 - xi;
            // co-rank: left-list elements among the first dd outputs (left first on ties)
            int l = max(0, dd - (ylim - yj)), h = min(dd, xlim - xi);
            while (l < h) {
                const int mid = (l + h) >> 1;
                if (s.col[xi + mid] <= s.col[yj + dd - 1 - mid]) l = mid + 1; else h = mid;
            }
            if constexpr (Sink::kOffsets) {
                if (dd == 0) {
                    // pair m -- and any empty pairs right before it -- start here
                    mfirst = m;
                    while (mfirst > 0 && s.off[2 * (mfirst - 1)] == d0) --mfirst;
                    for (int mm = mfirst; mm <= m; ++mm) sink.d.off[mm] = 0;
                    mlast = m;
                }
            }
            yj += dd - l;
            xi += l;
            {
                int32_t xc = xi < xlim ? s.col[xi] : kColEnd;
                int32_t yc = yj < ylim ? s.col[yj] : kColEnd;
                T xv = T(), yv = T();
                if constexpr (P::kVal) {
                    if (xi < xlim) xv = s.val[xi];
                    if (yj < ylim) yv = s.val[yj];
                }
                // the first diagonal may be a right-list element already added
                // to its equal left partner by the previous thread
                bool skip = (yj < ylim) && (l > 0) && (s.col[xi - 1] == yc);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (d0 + k < end) {
                        if (skip) {
                            skip = false;
                            ++yj;
                            yc = yj < ylim ? s.col[yj] : kColEnd;
                            if constexpr (P::kVal) { if (yj < ylim) yv = s.val[yj]; }
                        } else {
                            while (xc == kColEnd && yc == kColEnd && m + 1 < np) {
                                // this pair is done; the next non-empty pair starts here
                                ++m;
                                xi = s.off[2 * m];
                                xlim = s.off[2 * m + 1];
                                yj = xlim;
                                ylim = (2 * m + 2 <= nl) ? s.off[2 * m + 2] : xlim;
                                if constexpr (Sink::kOffsets) {
                                    sink.d.off[m] = cnt;
                                    if (mlast < 0) mfirst = m;
                                    mlast = m;
                                }
                                xc = xi < xlim ? s.col[xi] : kColEnd;
                                yc = yj < ylim ? s.col[yj] : kColEnd;
                                if constexpr (P::kVal) {
                                    if (xi < xlim) xv = s.val[xi];
                                    if (yj < ylim) yv = s.val[yj];
                                }
                            }
                            int32_t c;
                            T v;
                            if (xc <= yc) {
                                c = xc;
                                v = xv;
                                if (xc == yc) { v = P::add(xv, yv); skip = true; }
                                ++xi;
                                xc = xi < xlim ? s.col[xi] : kColEnd;
                                if constexpr (P::kVal) { if (xi < xlim) xv = s.val[xi]; }
                            } else {
                                c = yc;
                                v = yv;
                                ++yj;
                                yc = yj < ylim ? s.col[yj] : kColEnd;
                                if constexpr (P::kVal) { if (yj < ylim) yv = s.val[yj]; }
                            }
                            oc[k] = c;
                            ov[k] = v;
                            vmask |= 1u << k;
                            ++cnt;
                        }
                    }
                }
            }
        }
        int tot;
        const int ex = g.scan_excl(cnt, tot);
        int w = base + ex;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if ((vmask >> k) & 1u) {
                sink.put(w, oc[k], ov[k]);
                ++w;
            }
        }
        if constexpr (Sink::kOffsets) {
            for (int mm = mfirst; mm <= mlast; ++mm) sink.d.off[mm] += base + ex;
        }
        base += tot;
    }
    if constexpr (Sink::kOffsets) {
        // pairs that start after the last element (trailing empty lists) and the end
        for (int m = g.rank(); m < np; m += G::N)
            if (s.off[2 * m] == N) sink.d.off[m] = base;
        if (g.rank() == 0) sink.d.off[np] = base;
    }
    g.sync();
    return base;
}

// ---------------------------------------------------------------------------
// One merging round in device memory, tile by tile through shared memory
// (long rows).  The same merge as merge_round -- the same pairs, the same
// merge-path cut into tiles of NT * K diagonals, left list first on ties --
// but no thread searches device memory per tile: the block first finds the
// pair and co-rank at the ends of NT / 4 tiles at once (one search per
// thread), then every tile's consumed elements are copied into shared memory
// with cp.async (the next tile's while the current one merges), and each
// thread searches and merges there, K steps without divergent branches
// (left or right, tie and skip are selects), into a shared-memory buffer
// that it copies out after the block's prefix sum of the counts.
//
// A tile [D0, D1) takes pairs m0 .. m1.  The diagonals of a tile consume
// exactly D1 - D0 elements, laid out in shared memory as
//   pair m0:        its left-list part, then its right-list part (both cut
//                   at the tile's start co-rank, and at the end one when
//                   m1 == m0);
//   pairs m0+1 .. m1-1: whole, in buffer order;
//   pair m1 > m0:   the left-list prefix, then the right-list prefix;
// so that pair m > m0 starts at local position s.off[2m] - D0.  Three
// elements outside the tile complete it: the left element before the tile
// (a right element equal to it at the tile's start was already added), and
// the next left and right elements after it (a left element at the tile's
// end equal to the next right one adds that one's value).
// ---------------------------------------------------------------------------
template <class P, int NT, int K>
struct TiledRoundSmem {
    using T = typename P::T;
    static constexpr int TS = NT * K;   // diagonals per tile
    static constexpr int CH = NT / 4;   // tiles per partition chunk
    static constexpr int NB = CH + 1;   // cuts per chunk: the chunk's tile starts and its end
    static constexpr int TAB = 1024;    // list offsets a tile stages (else read from device memory)
    // per tile end: pair, co-rank, pair's left start / left end / right end,
    // left element before, left element after, right element after (columns)
    static constexpr int kFields = 8;
    // two tiles (the next one is loaded while the current one is merged)
    static constexpr size_t kVal = 0;
    static constexpr size_t kCol = kVal + (P::kVal ? 2 * sizeof(T) * TS : 0);
    static constexpr size_t kBV = align_up(kCol + 2 * sizeof(int32_t) * TS, 16);
    static constexpr size_t kBI = align_up(kBV + (P::kVal ? sizeof(T) * NB : 0), 16);
    static constexpr size_t kTab = align_up(kBI + sizeof(int32_t) * kFields * NB, 16);
    // each thread's merged elements, diagonal k of thread t at k * NT + t
    static constexpr size_t kOV = align_up(kTab + 2 * sizeof(int32_t) * TAB, 16);
    static constexpr size_t kOC = kOV + (P::kVal ? sizeof(T) * TS : 0);
    static constexpr size_t kBytes = align_up(kOC + sizeof(int32_t) * TS, 16);
};

// Pair and co-rank at diagonal D of a round (s, nl lists, np pairs), with the
// pair's list bounds and the elements around the cut, into entry e.
template <class P, int NB>
__device__ __forceinline__ void tiled_cut(const Buf<P> s, int nl, int np, int D, int32_t *bi,
                                          typename P::T *bv, int e) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s.off[2 * mid] <= D) lo = mid; else hi = mid - 1;
    }
    const int m = lo;
    const int xs = s.off[2 * m], xl = s.off[2 * m + 1];
    const int yl = (2 * m + 2 <= nl) ? s.off[2 * m + 2] : xl;
    const int dd = D - xs;
    int l = max(0, dd - (yl - xl)), h = min(dd, xl - xs);
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (s.col[xs + mid] <= s.col[xl + dd - 1 - mid]) l = mid + 1; else h = mid;
    }
    const int yp = xl + dd - l;
    bi[0 * NB + e] = m;
    bi[1 * NB + e] = l;
    bi[2 * NB + e] = xs;
    bi[3 * NB + e] = xl;
    bi[4 * NB + e] = yl;
    bi[5 * NB + e] = l > 0 ? s.col[xs + l - 1] : -1;
    bi[6 * NB + e] = xs + l < xl ? s.col[xs + l] : kColEnd;
    bi[7 * NB + e] = yp < yl ? s.col[yp] : kColEnd;
    if constexpr (P::kVal) bv[e] = yp < yl ? s.val[yp] : typename P::T();
}

// Asynchronous 4- and 8-byte copies device memory -> shared memory.
__device__ __forceinline__ void tiled_cp4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
template <class T>
__device__ __forceinline__ void tiled_cpv(T *dst, const T *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void tiled_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tiled_cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Issues the copies of tile c (cut entries ea = c - c0 and ea + 1) into one
// of the two tile buffers: the elements its diagonals consume, in the order
// described above, and the list offsets of its pairs when they fit.
template <class P, int NT, int K>
__device__ __forceinline__ void tiled_stage(const Buf<P> s, int nl, int N, int c, int ea, const int32_t *bi,
                                            int32_t *tc, typename P::T *tv, int32_t *tab) {
    using S = TiledRoundSmem<P, NT, K>;
    constexpr int TS = S::TS, NB = S::NB;
    const int tid = (int)threadIdx.x;
    const int eb = ea + 1;
    const int D0 = c * TS, TL = (int)min((int64_t)TS, (int64_t)N - D0);
    const int m0 = bi[0 * NB + ea], l0 = bi[1 * NB + ea], xs0 = bi[2 * NB + ea];
    const int xl0 = bi[3 * NB + ea], yl0 = bi[4 * NB + ea];
    const int m1 = bi[0 * NB + eb], l1 = bi[1 * NB + eb], xs1 = bi[2 * NB + eb], xl1 = bi[3 * NB + eb];
    const int dd0 = D0 - xs0, dd1 = D0 + TL - xs1;
    const int nx0 = (m0 == m1 ? l1 : xl0 - xs0) - l0;
    const int ny0 = (m0 == m1 ? dd1 - l1 : yl0 - xl0) - (dd0 - l0);
    const int e0 = nx0 + ny0;
    const int xb0 = xs0 + l0, yb0 = xl0 + dd0 - l0;
    const int sl1 = xs1 - D0;
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const int i = tid + u * NT;
        if (i < TL) {
            const int src = i < nx0 ? xb0 + i : i < e0 ? yb0 + (i - nx0) : i < sl1 + l1 ? D0 + i : xl1 + (i - sl1 - l1);
            tiled_cp4(tc + i, s.col + src);
            if constexpr (P::kVal) tiled_cpv(tv + i, s.val + src);
        }
    }
    const int tlo = 2 * m0;
    const int nent = min(2 * m1 + 2, nl) - tlo + 1;
    if (nent <= S::TAB)
        for (int i = tid; i < nent; i += NT) tiled_cp4(tab + i, s.off + tlo + i);
    tiled_cp_commit();
}

template <class P, int NT, int K, class Sink>
__device__ int merge_round_tiled(const BlockGrp<NT> &g, int nl, const Buf<P> s, const Sink &sink,
                                 unsigned char *sm) {
    using T = typename P::T;
    using S = TiledRoundSmem<P, NT, K>;
    constexpr int TS = S::TS, NB = S::NB;
    T *tv0 = reinterpret_cast<T *>(sm + S::kVal);
    int32_t *tc0 = reinterpret_cast<int32_t *>(sm + S::kCol);
    T *bv = reinterpret_cast<T *>(sm + S::kBV);
    int32_t *bi = reinterpret_cast<int32_t *>(sm + S::kBI);
    int32_t *tab0 = reinterpret_cast<int32_t *>(sm + S::kTab);
    T *ovs = reinterpret_cast<T *>(sm + S::kOV);
    int32_t *ocs = reinterpret_cast<int32_t *>(sm + S::kOC);
    const int tid = (int)threadIdx.x;
    const int N = s.off[nl];
    const int np = (nl + 1) >> 1;
    const int ntiles = (int)(((int64_t)N + TS - 1) / TS);
    int base = 0;
    for (int c0 = 0; c0 < ntiles; c0 += S::CH) {
        // cuts at the starts of tiles c0 .. c0 + CH (entry c - c0)
        {
            const int c = c0 + tid;
            if (tid <= S::CH && c <= ntiles)
                tiled_cut<P, NB>(s, nl, np, (int)min((int64_t)c * TS, (int64_t)N), bi, bv, tid);
        }
        g.sync();
        const int ce = min(ntiles, c0 + S::CH);
        tiled_stage<P, NT, K>(s, nl, N, c0, 0, bi, tc0 + (c0 & 1) * TS, tv0 + (c0 & 1) * TS, tab0 + (c0 & 1) * S::TAB);
        for (int c = c0; c < ce; ++c) {
            // tile c is in buffer c & 1; every thread is done with tile c - 1,
            // whose buffer takes tile c + 1
            tiled_cp_wait();
            g.sync();
            if (c + 1 < ce)
                tiled_stage<P, NT, K>(s, nl, N, c + 1, c + 1 - c0, bi, tc0 + ((c + 1) & 1) * TS,
                                      tv0 + ((c + 1) & 1) * TS, tab0 + ((c + 1) & 1) * S::TAB);
            const int32_t *tc = tc0 + (c & 1) * TS;
            const T *tv = tv0 + (c & 1) * TS;
            const int32_t *tab = tab0 + (c & 1) * S::TAB;
            const int ea = c - c0, eb = ea + 1;
            const int D0 = c * TS, D1 = (int)min((int64_t)D0 + TS, (int64_t)N), TL = D1 - D0;
            const int m0 = bi[0 * NB + ea], l0 = bi[1 * NB + ea], xs0 = bi[2 * NB + ea];
            const int xl0 = bi[3 * NB + ea], yl0 = bi[4 * NB + ea];
            const int m1 = bi[0 * NB + eb], l1 = bi[1 * NB + eb], xs1 = bi[2 * NB + eb];
            const int dd0 = D0 - xs0, dd1 = D1 - xs1;
            const int nx0 = (m0 == m1 ? l1 : xl0 - xs0) - l0;
            const int ny0 = (m0 == m1 ? dd1 - l1 : yl0 - xl0) - (dd0 - l0);
            const int tlo = 2 * m0;
            const int nent = min(2 * m1 + 2, nl) - tlo + 1;
            const bool staged = nent <= S::TAB;
            auto off = [&](int idx) -> int {
                return (staged && idx >= tlo && idx < tlo + nent) ? tab[idx - tlo] : s.off[idx];
            };
            const int px0 = bi[5 * NB + ea];
            const int xe1 = bi[6 * NB + eb], ye1 = bi[7 * NB + eb];
            T yev = T();
            if constexpr (P::kVal) yev = bv[eb];

            const int p0 = tid * K;
            const int pend = min(p0 + K, TL);
            int cnt = 0;
            unsigned vmask = 0;
            int mfirst = 0, mlast = -1;
            if (p0 < TL) {
                // the pair holding local diagonal p0: the last one starting at or before it
                int lo = m0, hi = m1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off(2 * mid) - D0 <= p0) lo = mid; else hi = mid - 1;
                }
                int m = lo;
                // the pair's part of the tile: local start, left and right counts,
                // the columns after both parts (and the value after the right one)
                int sl, nx, ny, xe, ye;
                T yv_e = T();
                auto part = [&](int mm) {
                    if (mm == m0) {
                        sl = 0;
                        nx = nx0;
                        ny = ny0;
                    } else {
                        const int xsm = off(2 * mm), xlm = off(2 * mm + 1);
                        sl = xsm - D0;
                        if (mm == m1) {
                            nx = l1;
                            ny = dd1 - l1;
                        } else {
                            const int ylm = (2 * mm + 2 <= nl) ? off(2 * mm + 2) : xlm;
                            nx = xlm - xsm;
                            ny = ylm - xlm;
                        }
                    }
                    if (mm == m1) {
                        xe = xe1;
                        ye = ye1;
                        yv_e = yev;
                    } else {
                        xe = kColEnd;
                        ye = kColEnd;
                    }
                };
                part(m);
                const int dd = p0 - sl;
                int l = max(0, dd - ny), h = min(dd, nx);
                while (l < h) {
                    const int mid = (l + h) >> 1;
                    if (tc[sl + mid] <= tc[sl + nx + dd - 1 - mid]) l = mid + 1; else h = mid;
                }
                int xi = l, yj = dd - l;
                if constexpr (Sink::kOffsets) {
                    if (dd == 0 && (m != m0 || dd0 == 0)) {
                        // pair m -- and any empty pairs right before it -- start here
                        const int st = off(2 * m);
                        mfirst = m;
                        while (mfirst > 0 && off(2 * (mfirst - 1)) == st) --mfirst;
                        for (int mm = mfirst; mm <= m; ++mm) sink.d.off[mm] = 0;
                        mlast = m;
                    }
                }
                // current left and right elements (the columns after a part
                // when it is used up); loads are clamped into the tile and the
                // result selected, so that the lanes of a warp do not diverge
                int32_t xc, yc;
                T xv = T(), yv = T();
                auto load_x = [&]() {
                    const int i = min(sl + xi, TS - 1);
                    const bool in = xi < nx;
                    xc = in ? tc[i] : xe;
                    if constexpr (P::kVal) xv = tv[i];
                };
                auto load_y = [&]() {
                    const int i = min(sl + nx + yj, TS - 1);
                    const bool in = yj < ny;
                    yc = in ? tc[i] : ye;
                    if constexpr (P::kVal) { const T t = tv[i]; yv = in ? t : yv_e; }
                };
                load_x();
                load_y();
                // column of the last left element taken: a right element equal
                // to it was added by that element's diagonal and is skipped
                int32_t lastx = xi > 0 ? tc[sl + xi - 1] : (m == m0 && l0 > 0 ? px0 : -1);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (p0 + k < pend) {
                        while (xi >= nx && yj >= ny && m < m1) {
                            // this pair's part is done; the next pair starts here
                            ++m;
                            part(m);
                            xi = 0;
                            yj = 0;
                            if constexpr (Sink::kOffsets) {
                                sink.d.off[m] = cnt;
                                if (mlast < 0) mfirst = m;
                                mlast = m;
                            }
                            lastx = -1;
                            load_x();
                            load_y();
                        }
                        const bool takex = xc <= yc;
                        const bool skip = !takex && yc == lastx;
                        T v = yv;
                        if constexpr (P::kVal) {
                            const T sum = P::add(xv, yv);
                            v = takex ? (xc == yc ? sum : xv) : yv;
                        }
                        ocs[k * NT + tid] = takex ? xc : yc;
                        if constexpr (P::kVal) ovs[k * NT + tid] = v;
                        vmask |= (skip ? 0u : 1u) << k;
                        cnt += skip ? 0 : 1;
                        lastx = takex ? xc : lastx;
                        xi += takex ? 1 : 0;
                        yj += takex ? 0 : 1;
                        if (takex) load_x(); else load_y();
                    }
                }
            }
            // exclusive prefix of the counts over the block with one barrier:
            // the warp sums are read again only after the next tile's barrier
            int tot, ex;
            {
                const int lane = tid & 31, wid = tid >> 5;
                int v = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, v, d);
                    if (lane >= d) v += u;
                }
                if (lane == 31) g.ws[wid] = v;
                g.sync();
                const int ws_l = lane < BlockGrp<NT>::NW ? g.ws[lane] : 0;
                int w = ws_l;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, w, d);
                    if (lane >= d) w += u;
                }
                tot = __shfl_sync(0xffffffffu, w, BlockGrp<NT>::NW - 1);
                ex = __shfl_sync(0xffffffffu, w - ws_l, wid) + v - cnt;
            }
            int w = base + ex;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if ((vmask >> k) & 1u) {
                    sink.put(w, ocs[k * NT + tid], P::kVal ? ovs[k * NT + tid] : T());
                    ++w;
                }
            }
            if constexpr (Sink::kOffsets) {
                for (int mm = mfirst; mm <= mlast; ++mm) sink.d.off[mm] += base + ex;
            }
            base += tot;
        }
        g.sync();   // the cuts are replaced by the next chunk's
    }
    if constexpr (Sink::kOffsets) {
        // pairs that start after the last element (trailing empty lists) and the end
        for (int m = tid; m < np; m += NT)
            if (s.off[2 * m] == N) sink.d.off[m] = base;
        if (tid == 0) sink.d.off[np] = base;
    }
    g.sync();
    return base;
}

template <bool kTiled, class P, class G, int K, class Sink>
__device__ __forceinline__ int round_of(const G &g, int nl, const Buf<P> s, const Sink &sink, unsigned char *tsm) {
    if constexpr (kTiled) return merge_round_tiled<P, G::N, K>(g, nl, s, sink, tsm);
    else return merge_round<P, G, K>(g, nl, s, sink);
}

// Whole row (Algorithm 1 for one i): the multiplying phase into b0, merging
// rounds between b0 and b1 while more than two lists are left, then the last
// round -- or, for a row of one list, a copy -- into the row's output slot
// (the store that ends Algorithm 1).  Numeric passes write C (or C_bar) at
// out_rp[row]; every pass may record the row length in out_cnt[row].
template <class P, class G, int K, int UNR, bool kTiled = false>
__device__ __forceinline__ void brm_row(const G &g, int row, const RowJob &j, const Buf<P> &b0, const Buf<P> &b1,
                                        unsigned char *tsm = nullptr) {
    using In = typename P::In;
    const RowIn<In> ri = row_in<In>(j, row);
    const int L = ri.L;
    multiply_phase<P, G, UNR>(g, L, ri.acol, ri.aval, ri.brp, ri.bcol, ri.bval, b0, b1);
    Buf<P> s = b0, d = b1;
    int nl = L;
    while (nl > 2) {
        round_of<kTiled, P, G, K>(g, nl, s, BufSink<P>{d}, tsm);
        const Buf<P> t = s; s = d; d = t;
        nl = (nl + 1) >> 1;
    }
    int len;
    if constexpr (P::kVal) {
        const int64_t base = j.out_rp[row];
        // the row's slot: exactly nnz(C_i*) (Precise) or nprod_i (Upper)
        const int cap = (int)(j.out_rp[row + 1] - base);
        const OutSink<P> out{j.out_col + base, static_cast<typename P::Out *>(j.out_val) + base, cap};
        if (nl == 2) {
            len = round_of<kTiled, P, G, K>(g, nl, s, out, tsm);
        } else {
            len = s.off[nl];
            for (int p = g.rank(); p < len; p += G::N) out.put(p, s.col[p], s.val[p]);
        }
        if (len > cap || (j.exact && len != cap)) {
            if (g.rank() == 0) atomicOr(j.err, 1u);
        }
    } else {
        if (nl == 2) len = round_of<kTiled, P, G, K>(g, nl, s, CountSink<P>{}, tsm);
        else len = s.off[nl];
    }
    if (j.out_cnt != nullptr && g.rank() == 0) j.out_cnt[row] = len;
    g.sync();
}

}  // namespace brm
