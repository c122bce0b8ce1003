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
// block kernels) and on the device-memory arena (long rows).
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

// Whole row (Algorithm 1 for one i): the multiplying phase into b0, merging
// rounds between b0 and b1 while more than two lists are left, then the last
// round -- or, for a row of one list, a copy -- into the row's output slot
// (the last line of Algorithm 1).  Numeric passes write C (or C_bar) at
// out_rp[row]; every pass may record the row length in out_cnt[row].
template <class P, class G, int K, int UNR>
__device__ __forceinline__ void brm_row(const G &g, int row, const RowJob &j, const Buf<P> &b0, const Buf<P> &b1) {
    using In = typename P::In;
    const RowIn<In> ri = row_in<In>(j, row);
    const int L = ri.L;
    multiply_phase<P, G, UNR>(g, L, ri.acol, ri.aval, ri.brp, ri.bcol, ri.bval, b0, b1);
    Buf<P> s = b0, d = b1;
    int nl = L;
    while (nl > 2) {
        merge_round<P, G, K>(g, nl, s, BufSink<P>{d});
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
            len = merge_round<P, G, K>(g, nl, s, out);
        } else {
            len = s.off[nl];
            for (int p = g.rank(); p < len; p += G::N) out.put(p, s.col[p], s.val[p]);
        }
        if (len > cap || (j.exact && len != cap)) {
            if (g.rank() == 0) atomicOr(j.err, 1u);
        }
    } else {
        if (nl == 2) len = merge_round<P, G, K>(g, nl, s, CountSink<P>{});
        else len = s.off[nl];
    }
    if (j.out_cnt != nullptr && g.rank() == 0) j.out_cnt[row] = len;
    g.sync();
}

}  // namespace brm
