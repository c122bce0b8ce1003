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

// ---------------------------------------------------------------------------
// Value policies.  Products are rounded before any addition and additions are
// never contracted into an FMA (explicit _rn intrinsics).
// ---------------------------------------------------------------------------
struct PF64 {
    using In = double; using T = double; using Out = double;
    static constexpr bool kVal = true;
    __device__ static __forceinline__ T mul(In a, In b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ T add(T x, T y) { return __dadd_rn(x, y); }
    __device__ static __forceinline__ Out fin(T x) { return x; }
};

struct PF32 {
    using In = float; using T = float; using Out = float;
    static constexpr bool kVal = true;
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
    __device__ static __forceinline__ T mul(In, In) { return 0.0f; }
    __device__ static __forceinline__ T add(T, T) { return 0.0f; }
    __device__ static __forceinline__ Out fin(T) { return 0.0f; }
};

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

// Everything a row kernel reads and writes.
struct RowJob {
    const int32_t *arp, *acol; const void *aval;
    const int32_t *brp, *bcol; const void *bval;
    const int32_t *rows;        // row ids of this bin (or batch)
    int32_t count;              // number of rows in the list
    const int64_t *out_rp;      // numeric: where row i starts in out_col/out_val
    int32_t *out_col;
    void *out_val;
    int64_t *out_cnt;           // optional: receives each row's length
    unsigned int *err;          // set to 1 if a row's length disagrees with its slot
    // long rows only: per slot, the arena offset (bytes) and the product count
    char *arena;
    const int64_t *arena_off;
    const int64_t *slot_nprod;
};

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
// ---------------------------------------------------------------------------
template <class P, class G>
__device__ __forceinline__ int multiply_phase(const G &g, int L, const int32_t *__restrict__ acol,
                                              const typename P::In *__restrict__ aval,
                                              const int32_t *__restrict__ brp, const int32_t *__restrict__ bcol,
                                              const typename P::In *__restrict__ bval, Buf<P> b) {
    int carry = 0;
    if (g.rank() == 0) b.off[0] = 0;
    for (int base = 0; base < L; base += G::N) {
        const int t = base + g.rank();
        int len = 0;
        if (t < L) { const int k = acol[t]; len = brp[k + 1] - brp[k]; }
        int tot;
        const int ex = g.scan_excl(len, tot);
        if (t < L) b.off[t + 1] = carry + ex + len;
        carry += tot;
    }
    g.sync();
    const int N = carry;
    int t = -1, lo = 0, hi = 0, q0 = 0;
    typename P::In a = typename P::In();
    for (int p = g.rank(); p < N; p += G::N) {
        if (p >= hi) {
            if (t >= 0) {
                int s = 0;
                while (s < 4 && b.off[t + 1] <= p) { ++t; ++s; }
                if (b.off[t + 1] <= p) t = t + find_last_le(b.off + t, L - t, p);
            } else {
                t = find_last_le(b.off, L, p);
            }
            lo = b.off[t];
            hi = b.off[t + 1];
            const int k = acol[t];
            q0 = brp[k];
            if constexpr (P::kVal) a = aval[t];
        }
        const int q = q0 + (p - lo);
        b.col[p] = bcol[q];
        if constexpr (P::kVal) b.val[p] = P::mul(a, bval[q]);
    }
    g.sync();
    return N;
}

// ---------------------------------------------------------------------------
// One merging round: nl lists in s -> ceil(nl/2) lists in d.
// ---------------------------------------------------------------------------
template <class P, class G, int K>
__device__ __forceinline__ void merge_round(const G &g, int nl, const Buf<P> s, const Buf<P> d) {
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
            if (dd == 0) {
                // pair m -- and any empty pairs right before it -- start here
                mfirst = m;
                while (mfirst > 0 && s.off[2 * (mfirst - 1)] == d0) --mfirst;
                for (int mm = mfirst; mm <= m; ++mm) d.off[mm] = 0;
                mlast = m;
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
                                d.off[m] = cnt;
                                if (mlast < 0) mfirst = m;
                                mlast = m;
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
                d.col[w] = oc[k];
                if constexpr (P::kVal) d.val[w] = ov[k];
                ++w;
            }
        }
        for (int mm = mfirst; mm <= mlast; ++mm) d.off[mm] += base + ex;
        base += tot;
    }
    // pairs that start after the last element (trailing empty lists) and the end
    for (int m = g.rank(); m < np; m += G::N)
        if (s.off[2 * m] == N) d.off[m] = base;
    if (g.rank() == 0) d.off[np] = base;
    g.sync();
}

// Whole row: multiplying phase into b0, then the accumulating phase.
// Returns the buffer holding the result (0: b0, 1: b1) and its length.
template <class P, class G, int K>
__device__ __forceinline__ int brm_row(const G &g, int row, const RowJob &j, const Buf<P> &b0, const Buf<P> &b1,
                                       int &len) {
    using In = typename P::In;
    const int a0 = j.arp[row];
    const int L = j.arp[row + 1] - a0;
    multiply_phase<P, G>(g, L, j.acol + a0, static_cast<const In *>(j.aval) + a0, j.brp, j.bcol,
                         static_cast<const In *>(j.bval), b0);
    Buf<P> s = b0, d = b1;
    int which = 0, nl = L;
    while (nl > 1) {
        merge_round<P, G, K>(g, nl, s, d);
        const Buf<P> t = s; s = d; d = t;
        which ^= 1;
        nl = (nl + 1) >> 1;
    }
    len = s.off[nl];
    return which;
}

// Row store (Algorithm 1, last step): numeric passes copy the row to
// out_col/out_val at out_rp[row]; every pass may record the row length.
template <class P, class G>
__device__ __forceinline__ void store_row(const G &g, int row, const RowJob &j, const Buf<P> &s, int len) {
    if constexpr (P::kVal) {
        using Out = typename P::Out;
        const int64_t base = j.out_rp[row];
        // the row's slot: exactly nnz(C_i*) (Precise) or nprod_i (Upper)
        const int64_t cap = j.out_rp[row + 1] - base;
        if (len > cap) {
            if (g.rank() == 0) atomicOr(j.err, 1u);
            len = (int)cap;
        }
        Out *ov = static_cast<Out *>(j.out_val);
        for (int p = g.rank(); p < len; p += G::N) {
            j.out_col[base + p] = s.col[p];
            ov[base + p] = P::fin(s.val[p]);
        }
    }
    if (j.out_cnt != nullptr && g.rank() == 0) j.out_cnt[row] = len;
    g.sync();
}

}  // namespace brm
