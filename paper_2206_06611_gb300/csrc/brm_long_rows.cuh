// Long rows by column buckets (the default long-row path).
//
// Algorithm 1 fixes every value of a row column by column: the value at
// column c is the sum of the products A_it * B_tc over the lists t whose B
// row holds c, added in the merge tree's order.  Two products of lists
// t1 < t2 first meet in round bitlen(t1 ^ t2) -- the first round r with
// t1 >> r == t2 >> r -- and there the left partial sum is added first; a list
// without column c passes its partner's partial sum through unchanged.  Any
// procedure that adds the products of each column in that aligned binary tree
// gives Algorithm 1's result bit for bit, whatever order the columns are
// visited in.  The merge rounds of the arena kernel read and write a long row
// once per round; here a row is read twice and its products are written and
// read once.
//
// Symbolic pass (column counts only): the row's columns are set in a
// shared-memory bitmap (one window of 2^20 columns at a time) and counted.
//
// Numeric pass, one thread block per row:
//  1. histogram: the row's products are counted per cell of 2^sh columns
//     (at most 4096 cells cover B's columns);
//  2. plan: consecutive cells are grouped into units of at most 256
//     products: a cut wherever the running count crosses a multiple of 128,
//     before and after every cell of more than 128 products, and at every
//     aligned window of 2^16 columns;
//  3. scatter: every product goes to its cell's region of a device-memory
//     arena as a 32-bit key (the column's low 16 bits above the list index)
//     and its rounded value;
//  4. units in column order, one warp per unit, 16 units at a time: the
//     warp sorts its unit's keys (and values) in registers with a bitonic
//     network (8 per lane), and every run of equal columns is reduced in tree
//     order -- by one lane with a stack of partial sums when short; when
//     long, each lane reduces an aligned range of lists and the lanes'
//     results are combined as the five tree levels above them; the warps'
//     column counts give the units' output offsets;
//  5. a single cell of more than 256 products is split again by column (its
//     products are counted per column, planned into units the same way and
//     copied to a second arena region in column order); a column of more than
//     256 products is reduced densely: its values go to one slot per list and
//     the tree is evaluated over the slots by the block.
// A row qualifies when it has at most 65535 lists and B at most 2^24 columns
// (a key never equals the all-ones padding); the host otherwise keeps the
// arena kernel for the whole pass.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "brm_engine.cuh"
#include "brm_internal.h"

namespace brm {

constexpr int kLsThreads = 1024;            // symbolic bitmap kernel
constexpr int kLsWinBits = 1 << 20;         // columns per bitmap window (128 KB)
constexpr int kLbThreads = 512;             // numeric bucket kernel
constexpr int kLbWarps = kLbThreads / 32;
constexpr int kLbCells = 4096;              // histogram cells of a row
constexpr int kLbUnit = 256;                // products of a unit (one warp, 8 per lane)
constexpr int kLbHalf = kLbUnit / 2;        // cut spacing of the plan
constexpr int kLbRunShort = 32;             // runs up to this size: one lane reduces
constexpr int kLbDepth = 18;                // partial-sum stack (tree height <= 16, +1)
constexpr uint32_t kLbPad = 0xffffffffu;    // padding key, above every real key
constexpr size_t kLbBmBytes = 8192;         // giant column: one bit per list (65536 lists)

static_assert(kLbCells % kLbThreads == 0 && kLbThreads % 32 == 0, "bucket kernel: per-thread shares must be whole");
static_assert(kLbMaxL <= 65535, "list index and column must never form the padding key");

__host__ __device__ constexpr int lb_bitlen(uint64_t x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

// Cell shift of a row: the smallest sh with ceil(ncols / 2^sh) <= kLbCells.
__host__ __device__ constexpr int lb_shift(int64_t ncols) {
    const int b = lb_bitlen((uint64_t)(ncols > 1 ? ncols - 1 : 0));
    return b > 12 ? b - 12 : 0;
}

// Device-memory arena of one long row of the numeric bucket kernel: level-1
// keys and values, level-2 keys and values (hot cells), one slot per list
// (giant columns), and the level-2 plan of the cell being split.
struct LbLayout {
    size_t k1, v1, k2, v2, slots, meta, wmeta, defer, total;
};

// Per warp, the state of the hot cell it is splitting: column ends, nonzero
// columns before each column, cut marks.
constexpr int kLbWmeta = 2 * 256 + 8;

// Work deferred to the whole block: a giant column (level 1 or 2) or a hot
// cell too wide for a warp.  Each holds more than kLbUnit products of its
// own, so a row of n products defers at most n / 257 of them.
struct LbDefer {
    int32_t kind, st, m, pad;
    int64_t col, ob;
};
constexpr int32_t kLbDeferGiant1 = 0, kLbDeferGiant2 = 1, kLbDeferHot = 2;

__host__ __device__ constexpr int64_t lb_defer_cap(int64_t n) { return n / (kLbUnit + 1) + 1; }

template <class P>
__host__ __device__ constexpr LbLayout lb_layout(int64_t n, int64_t L) {
    using T = typename P::T;
    const size_t kb = align_up(sizeof(uint32_t) * (size_t)n, 256);
    const size_t vb = align_up(sizeof(T) * (size_t)n, 256);
    const size_t sb = align_up(sizeof(T) * (size_t)(L > 0 ? L : 1), 256);
    const size_t mb = align_up(sizeof(int32_t) * (size_t)(2 * kLbCells + 2), 256);
    const size_t wb = align_up(sizeof(int32_t) * (size_t)kLbWmeta * (kLbThreads / 32), 256);
    const size_t db = align_up(sizeof(LbDefer) * (size_t)lb_defer_cap(n), 256);
    const size_t s0 = 2 * kb + 2 * vb;
    return LbLayout{0, kb, kb + vb, 2 * kb + vb, s0, s0 + sb, s0 + sb + mb, s0 + sb + mb + wb, s0 + sb + mb + wb + db};
}

// Shared memory of the numeric bucket kernel (dynamic part).
template <class P>
struct LbSmem {
    using T = typename P::T;
    using In = typename P::In;
    static constexpr int NW = kLbThreads / 32;
    static constexpr size_t kCnt = 0;                                             // int[kLbCells]
    static constexpr size_t kUl = kCnt + sizeof(int32_t) * kLbCells;              // int[kLbCells + 1]
    static constexpr size_t kDoff = align_up(kUl + sizeof(int32_t) * (kLbCells + 1), 16); // int[kLbCells]
    static constexpr size_t kQ0 = kDoff + sizeof(int32_t) * kLbCells;            // int[NT]
    static constexpr size_t kOff = kQ0 + sizeof(int32_t) * kLbThreads;            // int[NT + 1]
    static constexpr size_t kA = align_up(kOff + sizeof(int32_t) * (kLbThreads + 1), 16); // In[NT]
    // unit region: per warp, the sorted keys and values of its unit; overlaid
    // by the level-2 plan of a hot cell and by the giant-column scratch
    static constexpr size_t kUnit = align_up(kA + sizeof(In) * kLbThreads, 16);
    static constexpr size_t kStageK = kUnit;                                      // u32[NW][kLbUnit]
    static constexpr size_t kStageV = kStageK + sizeof(uint32_t) * NW * kLbUnit;  // T[NW][kLbUnit]
    static constexpr size_t kGiant = kLbBmBytes + (sizeof(T) + sizeof(int32_t)) * kLbThreads;
    static constexpr size_t kUnitBytes = std::max(std::max((sizeof(uint32_t) + sizeof(T)) * NW * kLbUnit,
                                                           sizeof(int32_t) * (2 * kLbCells + 2)), kGiant);
    static constexpr size_t kBytes = align_up(kUnit + kUnitBytes, 16);
};

__device__ __forceinline__ double lb_shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float lb_shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float2 lb_shfl_down(float2 v, int d) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// Tree-order sum of items [b, e) of one column, sorted by list (the low 16
// bits of the key): each new item meets the previous one at level
// bitlen(t_prev ^ t); partial sums on the stack that met their predecessor
// below that level are complete and are added first.  The stack lives in the
// items' own shared-memory slots: entry j (its partial sum, and the level at
// which it met the entry below in place of the key) at b + j, which is never
// past the item being read; its top stays in registers.  The levels on the
// stack strictly decrease for valid input (at most 17 entries); repeated
// columns inside a B row (invalid input) only give some order of additions.
// The run's slots are consumed: callers find every run's end before any run
// is reduced.
template <class P>
__device__ __noinline__ typename P::T lb_stack_reduce(uint32_t *ks, typename P::T *vs, int b, int e) {
    using T = typename P::T;
    T top = vs[b];
    uint32_t gtop = 32, prev = ks[b] & 0xffffu;
    int nv = 1;
    for (int i = b + 1; i < e; ++i) {
        const uint32_t t = ks[i] & 0xffffu;
        const T v = vs[i];
        const uint32_t d = 32 - __clz(prev ^ t);
        while (nv > 1 && gtop < d) {
            top = P::add(vs[b + nv - 2], top);
            gtop = ks[b + nv - 2];
            --nv;
        }
        vs[b + nv - 1] = top;
        ks[b + nv - 1] = gtop;
        top = v;
        gtop = d;
        ++nv;
        prev = t;
    }
    while (nv > 1) {
        top = P::add(vs[b + nv - 2], top);
        --nv;
    }
    return top;
}

// First index in [lo, hi) whose key's column part exceeds `col`.
__device__ __forceinline__ int lb_run_end(const uint32_t *ks, int lo, int hi, uint32_t col) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((ks[mid] >> 16) <= col) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// End of the run starting at sorted position idx of a unit of m products:
// the next set bit of the unit's 256-bit run-start mask, else m.
__device__ __forceinline__ int lb_next_start(const uint32_t *stm, int idx, int m) {
    int p = idx + 1;
    while (p < m) {
        const uint32_t x = stm[p >> 5] & (0xffffffffu << (p & 31));
        if (x) return min(m, (p & ~31) + __ffs(x) - 1);
        p = (p & ~31) + 32;
    }
    return m;
}

// First index in [lo, hi) whose list index is >= x (items of one column).
__device__ __forceinline__ int lb_list_lb(const uint32_t *ks, int lo, int hi, uint32_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((ks[mid] & 0xffffu) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// A long run [b, e) of one column, sorted by list, reduced by one warp: lane
// l takes the lists of the aligned node [l << ss, (l + 1) << ss) and reduces
// them with the stack; the 32 node values are then combined pairwise as the
// five tree levels above them.  The result is valid in lane 0.
template <class P>
__device__ typename P::T lb_warp_run(uint32_t *ks, typename P::T *vs, int b, int e, int lbits) {
    using T = typename P::T;
    const int lane = threadIdx.x & 31;
    const int ss = lbits > 5 ? lbits - 5 : 0;
    const int i0 = lb_list_lb(ks, b, e, (uint32_t)lane << ss);
    const int i1 = lb_list_lb(ks, i0, e, (uint32_t)(lane + 1) << ss);
    __syncwarp();   // every lane has found its range before any range is consumed
    bool has = i1 > i0;
    T v = has ? lb_stack_reduce<P>(ks, vs, i0, i1) : T();
#pragma unroll
    for (int h = 1; h < 32; h <<= 1) {
        const T ov = lb_shfl_down(v, h);
        const bool oh = __shfl_down_sync(0xffffffffu, has ? 1 : 0, h) != 0;
        if ((lane & (2 * h - 1)) == 0) {
            if (has && oh) v = P::add(v, ov);
            else if (oh) { v = ov; has = true; }
        }
    }
    return v;
}

// Output of a row: its slot in C (or C_bar).
template <class P>
struct LbOut {
    int32_t *col;
    typename P::Out *val;
    int64_t cap;
    __device__ __forceinline__ void put(int64_t w, int64_t c, typename P::T v) const {
        if (w < cap) {
            col[w] = (int32_t)c;
            val[w] = P::fin(v);
        }
    }
};

// The arrays and scalars of one row that the warp-level steps need.
template <class P>
struct LbRowArgs {
    uint32_t *k1, *k2;
    typename P::T *v1, *v2;
    int lbits;
    LbOut<P> out;
    unsigned *err;
};

// Loads the descriptors of lists [t0, t0 + NT) of a row (B row start, and
// the A value when `s_a` is given) and the exclusive prefix sums of their
// lengths; returns the chunk's product count.  Callers synchronise before
// the next chunk overwrites the arrays.
template <class In, int NT>
__device__ __forceinline__ int lb_load_chunk(const BlockGrp<NT> &g, const RowIn<In> &ri, int t0, int32_t *s_q0,
                                             int32_t *s_off, In *s_a) {
    const int t = t0 + (int)threadIdx.x;
    int len = 0, q0 = 0;
    if (t < ri.L) {
        const int k = ri.acol[t];
        q0 = ri.brp[k];
        len = ri.brp[k + 1] - q0;
        if (s_a != nullptr) s_a[threadIdx.x] = ri.aval[t];
    }
    int tot;
    const int ex = g.scan_excl(len, tot);
    s_q0[threadIdx.x] = q0;
    s_off[threadIdx.x] = ex;
    if (threadIdx.x == 0) s_off[NT] = tot;
    g.sync();
    return tot;
}

// The K products p0 .. p0 + K - 1 of a chunk: list (within the chunk) and
// position in B; q = -1 past the chunk's end.  p0 < tot.
template <int K>
__device__ __forceinline__ void lb_locate(const int32_t *s_off, const int32_t *s_q0, int nc, int tot, int p0,
                                          int (&tl)[K], int (&q)[K]) {
    int t = find_last_le(s_off, nc, p0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int p = p0 + k;
        q[k] = -1;
        tl[k] = t;
        if (p < tot) {
            while (s_off[t + 1] <= p) ++t;
            tl[k] = t;
            q[k] = s_q0[t] + (p - s_off[t]);
        }
    }
}

// ---------------------------------------------------------------------------
// Symbolic pass: distinct columns of each long row, by bitmap.
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kLsThreads, 1) k_long_sym(RowJob j) {
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ int32_t s_q0[kLsThreads];
    __shared__ int32_t s_off[kLsThreads + 1];
    __shared__ int ws[kLsThreads / 32 + 1];
    constexpr int K = 8;
    BlockGrp<kLsThreads> g;
    g.ws = ws;
    const int64_t ncols = j.bcols;
    for (int r = blockIdx.x; r < j.count; r += gridDim.x) {
        const int row = j.rows[r];
        const RowIn<float> ri = row_in<float>(j, row);
        int64_t count = 0;
        for (int64_t w0 = 0; w0 < ncols; w0 += kLsWinBits) {
            const uint32_t wn = (uint32_t)(ncols - w0 < kLsWinBits ? ncols - w0 : kLsWinBits);
            const int words = (int)((wn + 31) >> 5);
            for (int i = threadIdx.x; i < words; i += kLsThreads) bm[i] = 0u;
            g.sync();
            for (int t0 = 0; t0 < ri.L; t0 += kLsThreads) {
                const int nc = min(kLsThreads, ri.L - t0);
                const int tot = lb_load_chunk<float, kLsThreads>(g, ri, t0, s_q0, s_off, nullptr);
                for (int base = 0; base < tot; base += kLsThreads * K) {
                    const int p0 = base + (int)threadIdx.x * K;
                    if (p0 < tot) {
                        int tl[K], q[K];
                        lb_locate<K>(s_off, s_q0, nc, tot, p0, tl, q);
                        int32_t c[K];
#pragma unroll
                        for (int k = 0; k < K; ++k) c[k] = q[k] >= 0 ? __ldg(ri.bcol + q[k]) : -1;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const uint32_t u = (uint32_t)((int64_t)c[k] - w0);
                            if (q[k] >= 0 && c[k] >= 0 && u < wn) atomicOr(&bm[u >> 5], 1u << (u & 31));
                        }
                    }
                }
                g.sync();
            }
            int cnt = 0;
            for (int i = threadIdx.x; i < words; i += kLsThreads) cnt += __popc(bm[i]);
            int tot;
            g.scan_excl(cnt, tot);
            count += tot;
        }
        if (threadIdx.x == 0 && j.out_cnt != nullptr) j.out_cnt[row] = count;
        g.sync();
    }
}

// ---------------------------------------------------------------------------
// Numeric pass.
// ---------------------------------------------------------------------------

// Cuts cells [0, nc) with counts cnt[] into units (see the file comment).  On
// return cnt[d] holds cell d's exclusive start and ul[0 .. nu] the first cell
// of every unit (ul[nu] = nc); returns nu.  `win` > 0 also cuts at every
// multiple of win cells.
template <int NT>
__device__ int lb_plan(const BlockGrp<NT> &g, int32_t *cnt, int nc, int32_t *ul, int win) {
    constexpr int PER = kLbCells / NT;
    const int base = (int)threadIdx.x * PER;
    int c[PER];
    int sum = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int d = base + e;
        c[e] = d < nc ? cnt[d] : 0;
        sum += c[e];
    }
    int prevc = (base > 0 && base - 1 < nc) ? cnt[base - 1] : 0;
    int tot;
    int S = g.scan_excl(sum, tot);
    unsigned flags = 0;
    int nflag = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int d = base + e;
        if (d < nc) {
            const int Sp = S - prevc;   // start of cell d - 1
            const bool cut = d == 0 || c[e] > kLbHalf || prevc > kLbHalf || (S / kLbHalf) != (Sp / kLbHalf) ||
                             (win > 0 && d % win == 0);
            if (cut) {
                flags |= 1u << e;
                ++nflag;
            }
            cnt[d] = S;
        }
        prevc = c[e];
        S += c[e];
    }
    int ftot;
    int k = g.scan_excl(nflag, ftot);
#pragma unroll
    for (int e = 0; e < PER; ++e)
        if ((flags >> e) & 1u) ul[k++] = base + e;
    if (threadIdx.x == 0) ul[ftot] = nc;
    g.sync();
    return ftot;
}

template <class T>
__device__ __forceinline__ void lb_cx(uint32_t &ka, T &va, uint32_t &kb, T &vb) {
    if (ka > kb) {
        const uint32_t k = ka;
        ka = kb;
        kb = k;
        const T v = va;
        va = vb;
        vb = v;
    }
}

// Keeps the smaller (lower) or larger key of a pair exchanged between lanes.
template <class T>
__device__ __forceinline__ void lb_keep(uint32_t &k, T &v, uint32_t ok, T ov, bool lower) {
    if (lower ? (ok < k) : (ok > k)) {
        k = ok;
        v = ov;
    }
}

template <class T>
__device__ __forceinline__ T lb_shfl_xor(T v, int m);
template <>
__device__ __forceinline__ double lb_shfl_xor<double>(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <>
__device__ __forceinline__ float lb_shfl_xor<float>(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <>
__device__ __forceinline__ float2 lb_shfl_xor<float2>(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Sorts the 256 (key, value) pairs of a warp by key, lane l holding sorted
// positions 8l .. 8l + 7: the bitonic network in its all-ascending form (for
// each size, a mirror stage, then half-cleaners); distances below 8 stay in a
// lane's registers, larger ones pair lane l with lane l ^ (distance / 8).
template <class T>
__device__ __forceinline__ void lb_warp_sort(uint32_t (&k)[8], T (&v)[8], int lane) {
#pragma unroll
    for (int kk = 2; kk <= kLbUnit; kk <<= 1) {
        if (kk <= 8) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int ip = i ^ (kk - 1);
                if (ip > i) lb_cx(k[i], v[i], k[ip], v[ip]);
            }
        } else {
            // partner of element i: element 7 - i of lane ^ m
            const int m = (kk - 1) >> 3;
            const bool lower = (lane & (kk >> 4)) == 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t k1 = __shfl_xor_sync(0xffffffffu, k[7 - i], m);
                const T v1 = lb_shfl_xor(v[7 - i], m);
                const uint32_t k2 = __shfl_xor_sync(0xffffffffu, k[i], m);
                const T v2 = lb_shfl_xor(v[i], m);
                lb_keep(k[i], v[i], k1, v1, lower);
                lb_keep(k[7 - i], v[7 - i], k2, v2, lower);
            }
        }
#pragma unroll
        for (int jj = kk >> 2; jj >= 1; jj >>= 1) {
            if (jj < 8) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if ((i & jj) == 0) lb_cx(k[i], v[i], k[i | jj], v[i | jj]);
            } else {
                const int m = jj >> 3;
                const bool lower = (lane & m) == 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t ok = __shfl_xor_sync(0xffffffffu, k[i], m);
                    const T ov = lb_shfl_xor(v[i], m);
                    lb_keep(k[i], v[i], ok, ov, lower);
                }
            }
        }
    }
}

// Up to NW units at once, one per warp (`have`: this warp has a unit of m
// <= kLbUnit products at gk/gv whose columns start at col_lo, inside one
// aligned window of 2^16 columns).  The warps sort, count their distinct
// columns, exchange the counts, then reduce every run and write it at its
// place after obase.  Returns the group's output count (same in every thread).
template <class P, int NT>
__device__ __noinline__ int64_t lb_group(const BlockGrp<NT> &g, bool have, const uint32_t *gk, const typename P::T *gv, int m,
                            int64_t col_lo, int lbits, const LbOut<P> &out, int64_t obase, unsigned char *smem) {
    using T = typename P::T;
    using L_ = LbSmem<P>;
    constexpr int NW = NT / 32;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ int s_gcnt[NW];
    __shared__ uint32_t s_stm[NW][kLbUnit / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *sk = reinterpret_cast<uint32_t *>(smem + L_::kStageK) + warp * kLbUnit;
    T *sv = reinterpret_cast<T *>(smem + L_::kStageV) + warp * kLbUnit;
    uint32_t k[8];
    T v[8];
    unsigned stf = 0;
    int lbase = 0;
    if (have) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = i * 32 + lane;
            k[i] = kLbPad;
            v[i] = T();
            if (idx < m) {
                k[i] = __ldcs(gk + idx);
                v[i] = gv[idx];
            }
        }
        lb_warp_sort<T>(k, v, lane);
        const uint32_t before = __shfl_up_sync(kFull, k[7], 1);
        int nst = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t prv = i ? k[i - 1] : before;
            if (k[i] != kLbPad && ((lane == 0 && i == 0) || (prv >> 16) != (k[i] >> 16))) {
                stf |= 1u << i;
                ++nst;
            }
        }
        int x = nst;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, x, d);
            if (lane >= d) x += y;
        }
        lbase = x - nst;
        if (lane == 31) s_gcnt[warp] = x;
    } else if (lane == 0) {
        s_gcnt[warp] = 0;
    }
    g.sync();
    int64_t wbase = 0, gtot = 0;
#pragma unroll
    for (int x = 0; x < NW; ++x) {
        const int c = s_gcnt[x];
        wbase += x < warp ? c : 0;
        gtot += c;
    }
    if (have) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            sk[lane * 8 + i] = k[i];
            sv[lane * 8 + i] = v[i];
        }
        // start bits of the sorted positions (bit p of word p / 32): four lanes per word
        uint32_t word = stf << (8 * (lane & 3));
        word |= __shfl_xor_sync(kFull, word, 1);
        word |= __shfl_xor_sync(kFull, word, 2);
        if ((lane & 3) == 0) s_stm[warp][lane >> 2] = word;
        __syncwarp();
        const uint32_t *stm = s_stm[warp];
        const int64_t ob = obase + wbase;
        const int64_t wc = col_lo - (col_lo & 0xffff);
        unsigned longm = 0;
        int r = lbase;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((stf >> i) & 1u) {
                const int idx = lane * 8 + i, x = lb_next_start(stm, idx, m);
                if (x - idx > kLbRunShort) {
                    longm |= 1u << i;
                } else {
                    T s;
                    if (x - idx == 1) s = sv[idx];
                    else if (x - idx == 2) s = P::add(sv[idx], sv[idx + 1]);
                    else s = lb_stack_reduce<P>(sk, sv, idx, x);
                    out.put(ob + r, wc + (k[i] >> 16), s);
                }
                ++r;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            unsigned bm = __ballot_sync(kFull, (longm >> i) & 1u);
            const int ri = lbase + __popc(stf & ((1u << i) - 1u));
            while (bm) {
                const int src = __ffs(bm) - 1;
                bm &= bm - 1;
                const int rb = src * 8 + i;
                const int rr = __shfl_sync(kFull, ri, src);
                const uint32_t col = __shfl_sync(kFull, k[i] >> 16, src);
                const int re = lb_next_start(stm, rb, m);
                const T s = lb_warp_run<P>(sk, sv, rb, re, lbits);
                if (lane == 0) out.put(ob + rr, wc + col, s);
            }
        }
    }
    g.sync();
    return gtot;
}

// A column of m > kLbUnit products (keys gk, values gv in device memory):
// values go to their list's slot, present lists are marked in a bitmap, each
// thread reduces an aligned range of lists with the stack and the threads'
// results are combined as the tree levels above.  Writes one output.
template <class P, int NT>
__device__ __noinline__ void lb_giant(const BlockGrp<NT> &g, const uint32_t *gk, const typename P::T *gv, int m, int L, int lbits,
                         typename P::T *slots, const LbOut<P> &out, int64_t w, int64_t col, unsigned char *smem) {
    using T = typename P::T;
    using L_ = LbSmem<P>;
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem + L_::kUnit);
    T *pv = reinterpret_cast<T *>(smem + L_::kUnit + kLbBmBytes);
    int32_t *pf = reinterpret_cast<int32_t *>(smem + L_::kUnit + kLbBmBytes + sizeof(T) * NT);
    const int tid = (int)threadIdx.x;
    const int words = (L + 31) >> 5;
    for (int i = tid; i < words; i += NT) bm[i] = 0u;
    g.sync();
    for (int i = tid; i < m; i += NT) {
        const uint32_t t = __ldcs(gk + i) & 0xffffu;
        if ((int)t < L) {
            slots[t] = gv[i];
            atomicOr(&bm[t >> 5], 1u << (t & 31));
        }
    }
    g.sync();   // slot writes are visible to the block after the barrier
    constexpr int LOGNT = lb_bitlen(NT) - 1;
    const int ss = lbits > LOGNT ? lbits - LOGNT : 0;
    const int t0 = tid << ss, t1 = min((tid + 1) << ss, L);
    T V[kLbDepth];
    int G[kLbDepth];
    int nv = 0, prev = 0;
    for (int t = t0; t < t1; ++t) {
        if (!((bm[t >> 5] >> (t & 31)) & 1u)) {
            // skip the rest of an empty word quickly
            if (((bm[t >> 5] >> (t & 31)) == 0u)) t |= 31;
            continue;
        }
        if (nv > 0) {
            const int d = 32 - __clz(prev ^ t);
            while (nv > 1 && G[nv - 1] < d) {
                V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
                --nv;
            }
            G[nv] = d;
        }
        if (nv == kLbDepth) {
            V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
            --nv;
        }
        V[nv++] = slots[t];
        prev = t;
    }
    while (nv > 1) {
        V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
        --nv;
    }
    pv[tid] = nv ? V[0] : T();
    pf[tid] = nv ? 1 : 0;
    g.sync();
    for (int h = 1; h < NT; h <<= 1) {
        if ((tid & (2 * h - 1)) == 0 && pf[tid + h]) {
            pv[tid] = pf[tid] ? P::add(pv[tid], pv[tid + h]) : pv[tid + h];
            pf[tid] = 1;
        }
        g.sync();
    }
    if (tid == 0) out.put(w, col, pv[0]);
    g.sync();
}

// One unit of m <= kLbUnit products (keys gk, values gv in device memory)
// whose columns start at col_lo, inside one aligned window of 2^16 columns,
// by one warp: sorted in registers, every run of equal columns reduced in tree
// order (one lane per short run, the whole warp per long one) and written at
// out[ob ...].  sk/sv: the warp's staging slots (kLbUnit each).
template <class P>
__device__ __noinline__ void lb_wunit(const uint32_t *gk, const typename P::T *gv, int m, int64_t col_lo, int lbits,
                                      LbOut<P> out, int64_t ob, uint32_t *sk, typename P::T *sv) {
    using T = typename P::T;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ uint32_t s_stm[kLbThreads / 32][kLbUnit / 32];
    const int lane = threadIdx.x & 31;
    uint32_t *stm = s_stm[threadIdx.x >> 5];
    uint32_t k[8];
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane;
        k[i] = kLbPad;
        v[i] = T();
        if (idx < m) {
            k[i] = __ldcs(gk + idx);
            v[i] = gv[idx];
        }
    }
    lb_warp_sort<T>(k, v, lane);
    const uint32_t before = __shfl_up_sync(kFull, k[7], 1);
    unsigned stf = 0;
    int nst = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t prv = i ? k[i - 1] : before;
        if (k[i] != kLbPad && ((lane == 0 && i == 0) || (prv >> 16) != (k[i] >> 16))) {
            stf |= 1u << i;
            ++nst;
        }
    }
    int x = nst;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    const int lbase = x - nst;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        sk[lane * 8 + i] = k[i];
        sv[lane * 8 + i] = v[i];
    }
    // start bits of the sorted positions (bit p of word p / 32): four lanes per word
    uint32_t word = stf << (8 * (lane & 3));
    word |= __shfl_xor_sync(kFull, word, 1);
    word |= __shfl_xor_sync(kFull, word, 2);
    if ((lane & 3) == 0) stm[lane >> 2] = word;
    __syncwarp();
    const int64_t wc = col_lo - (col_lo & 0xffff);
    unsigned longm = 0;
    int r = lbase;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((stf >> i) & 1u) {
            const int idx = lane * 8 + i, e = lb_next_start(stm, idx, m);
            if (e - idx > kLbRunShort) {
                longm |= 1u << i;
            } else {
                T sum;
                if (e - idx == 1) sum = sv[idx];
                else if (e - idx == 2) sum = P::add(sv[idx], sv[idx + 1]);
                else sum = lb_stack_reduce<P>(sk, sv, idx, e);
                out.put(ob + r, wc + (k[i] >> 16), sum);
            }
            ++r;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        unsigned bm = __ballot_sync(kFull, (longm >> i) & 1u);
        const int ri = lbase + __popc(stf & ((1u << i) - 1u));
        while (bm) {
            const int src = __ffs(bm) - 1;
            bm &= bm - 1;
            const int rb = src * 8 + i;
            const int rr = __shfl_sync(kFull, ri, src);
            const uint32_t col = __shfl_sync(kFull, k[i] >> 16, src);
            const int re = lb_next_start(stm, rb, m);
            const T sum = lb_warp_run<P>(sk, sv, rb, re, lbits);
            if (lane == 0) out.put(ob + rr, wc + col, sum);
        }
    }
    __syncwarp();   // the staging slots are reused by the warp's next unit
}

// Records work for the block phase after the warps' units.
__device__ __forceinline__ void lb_defer(LbDefer *dl, int *s_n, int64_t cap, int32_t kind, int st, int m, int64_t col,
                                         int64_t ob, unsigned *err) {
    if ((threadIdx.x & 31) == 0) {
        const int i = atomicAdd(s_n, 1);
        if (i < cap) dl[i] = LbDefer{kind, st, m, 0, col, ob};
        else atomicOr(err, 1u);   // cannot happen: see lb_defer_cap
    }
    __syncwarp();
}

// A hot cell (m > kLbUnit products at [st0, st0 + m) of the level-1 arrays,
// cw <= 256 columns from cell_lo) split by one warp: counted per column in
// the warp's staging slots, cut into units like the cells of the row, copied
// column by column to the same region of the level-2 arrays, then every unit
// processed by the warp at its offset (ob plus the nonzero columns before
// it); a column of more than kLbUnit products is deferred to the block.
template <class P>
__device__ __noinline__ void lb_whot(const LbRowArgs<P> &ra, int st0, int m, int64_t cell_lo, int cw, int64_t ob,
                                     uint32_t *sk, typename P::T *sv, int32_t *wm, LbDefer *dl, int *s_nd,
                                     int64_t dcap) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int32_t *cnt = reinterpret_cast<int32_t *>(sk);
    const uint32_t *k1 = ra.k1 + st0;
    const typename P::T *v1 = ra.v1 + st0;
    uint32_t *k2 = ra.k2 + st0;
    typename P::T *v2 = ra.v2 + st0;
    int32_t *wend = wm, *wnz = wm + 256;
    uint32_t *wcut = reinterpret_cast<uint32_t *>(wm + 512);
    const uint32_t cmask = (uint32_t)cw - 1u;
    for (int c = lane; c < 256; c += 32) cnt[c] = 0;
    __syncwarp();
    for (int i = lane; i < m; i += 32) atomicAdd(&cnt[(__ldcs(k1 + i) >> 16) & cmask], 1);
    __syncwarp();
    // lane l owns columns 8l .. 8l + 7
    int c[8], sum = 0, nz = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        c[e] = cnt[lane * 8 + e];
        sum += c[e];
        nz += c[e] > 0 ? 1 : 0;
    }
    int xs = sum, xn = nz;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int ys = __shfl_up_sync(kFull, xs, d), yn = __shfl_up_sync(kFull, xn, d);
        if (lane >= d) { xs += ys; xn += yn; }
    }
    int S = xs - sum, Z = xn - nz;
    int prevc = __shfl_up_sync(kFull, c[7], 1);
    if (lane == 0) prevc = 0;
    unsigned flags = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int col = lane * 8 + e;
        const int Sp = S - prevc;
        if (col < cw && (col == 0 || c[e] > kLbHalf || prevc > kLbHalf || (S / kLbHalf) != (Sp / kLbHalf)))
            flags |= 1u << e;
        cnt[col] = S;
        wnz[col] = Z;
        Z += c[e] > 0 ? 1 : 0;
        prevc = c[e];
        S += c[e];
    }
    uint32_t word = flags << (8 * (lane & 3));
    word |= __shfl_xor_sync(kFull, word, 1);
    word |= __shfl_xor_sync(kFull, word, 2);
    if ((lane & 3) == 0) wcut[lane >> 2] = word;
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
        const uint32_t key = __ldcs(k1 + i);
        const int pos = atomicAdd(&cnt[(key >> 16) & cmask], 1);
        k2[pos] = key;
        v2[pos] = v1[i];
    }
    __syncwarp();
    for (int col = lane; col < cw; col += 32) wend[col] = cnt[col];
    __syncwarp();
    // units: column ranges between consecutive cut marks
    int c0 = 0;
    while (c0 < cw) {
        int c1 = c0 + 1;
        while (c1 < cw && !((wcut[c1 >> 5] >> (c1 & 31)) & 1u)) ++c1;
        const int st = c0 ? wend[c0 - 1] : 0, en = wend[c1 - 1];
        if (en > st) {
            const int64_t o2 = ob + wnz[c0];
            if (en - st <= kLbUnit)
                lb_wunit<P>(k2 + st, v2 + st, en - st, cell_lo + c0, ra.lbits, ra.out, o2, sk, sv);
            else
                lb_defer(dl, s_nd, dcap, kLbDeferGiant2, st0 + st, en - st, cell_lo + c0, o2, ra.err);
        }
        c0 = c1;
    }
}

// What the levels of one row share (passed by value).
template <class P>
struct LbRow {
    uint32_t *k1, *k2;
    typename P::T *v1, *v2, *slots;
    int32_t *meta;
    int L, lbits, sh;
    LbOut<P> out;
};

// The units of a level in column order: units of at most kLbUnit products
// go to the warps, NW non-empty ones at a time (lb_group); a larger one is a
// giant column (level 2, or level 1 with one-column cells) or a hot cell
// (level 1), split by column.  Level 1 reads the units from the row's plan
// in shared memory (cells ul[u] .. ul[u + 1], cell d ending at cnt[d]);
// level 2 reads the plan of one hot cell from device memory (meta).  Returns
// the output cursor after the level.
template <class P, int NT>
__device__ int64_t lb_hot(const BlockGrp<NT> &g, const LbRow<P> &rw, int st0, int m, int64_t cell_lo, int64_t w,
                          unsigned char *smem);

template <class P, int NT, int LEVEL>
__device__ int64_t lb_level(const BlockGrp<NT> &g, const LbRow<P> &rw, int nu, const int32_t *ul, const int32_t *cnt,
                            int base, int64_t cell_lo, int64_t w, unsigned char *smem) {
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5;
    const uint32_t *k = LEVEL == 1 ? rw.k1 : rw.k2;
    const typename P::T *v = LEVEL == 1 ? rw.v1 : rw.v2;
    int u = 0;
    while (u < nu) {
        int my_st = 0, my_en = 0, taken = 0;
        int64_t my_cl = 0;
        while (u < nu) {
            const int c0 = ul[u], c1 = ul[u + 1];
            const int st = base + (c0 ? cnt[c0 - 1] : 0), en = base + cnt[c1 - 1];
            const int64_t cl = LEVEL == 1 ? (int64_t)c0 << rw.sh : cell_lo + c0;
            if (en - st > kLbUnit) {
                if (taken > 0) break;   // the group first
                bool split = false;
                if constexpr (LEVEL == 1) {
                    if (rw.sh > 0) {
                        w = lb_hot<P, NT>(g, rw, st, en - st, cl, w, smem);
                        split = true;
                    }
                }
                if (!split) {
                    lb_giant<P, NT>(g, k + st, v + st, en - st, rw.L, rw.lbits, rw.slots, rw.out, w, cl, smem);
                    ++w;
                }
                ++u;
                continue;
            }
            if (taken == NW) break;
            if (en > st) {
                if (taken == warp) {
                    my_st = st;
                    my_en = en;
                    my_cl = cl;
                }
                ++taken;
            }
            ++u;
        }
        if (taken > 0)
            w += lb_group<P, NT>(g, warp < taken, k + my_st, v + my_st, my_en - my_st, my_cl, rw.lbits, rw.out, w,
                                 smem);
    }
    return w;
}

// A cell of m > kLbUnit products at [st0, st0 + m) of the level-1 arrays:
// counted per column, planned into units like the cells of the row, copied to
// the same region of the level-2 arrays in column order, and processed as
// level 2.  Returns the output cursor after the cell.
template <class P, int NT>
__device__ int64_t lb_hot(const BlockGrp<NT> &g, const LbRow<P> &rw, int st0, int m, int64_t cell_lo, int64_t w,
                          unsigned char *smem) {
    using L_ = LbSmem<P>;
    int32_t *cnt2 = reinterpret_cast<int32_t *>(smem + L_::kUnit);
    int32_t *ul2 = cnt2 + kLbCells;
    const uint32_t *k1 = rw.k1 + st0;
    const typename P::T *v1 = rw.v1 + st0;
    uint32_t *k2 = rw.k2 + st0;
    typename P::T *v2 = rw.v2 + st0;
    const int cw = 1 << rw.sh;
    const int tid = (int)threadIdx.x;
    for (int i = tid; i < cw; i += NT) cnt2[i] = 0;
    g.sync();
    for (int i = tid; i < m; i += NT) atomicAdd(&cnt2[(k1[i] >> 16) & (uint32_t)(cw - 1)], 1);
    g.sync();
    const int nu2 = lb_plan<NT>(g, cnt2, cw, ul2, 0);
    for (int i = tid; i < m; i += NT) {
        const uint32_t key = k1[i];
        const int pos = atomicAdd(&cnt2[(key >> 16) & (uint32_t)(cw - 1)], 1);
        k2[pos] = key;
        v2[pos] = v1[i];
    }
    g.sync();
    // the plan moves to device memory: the units reuse shared memory
    for (int i = tid; i < cw; i += NT) rw.meta[i] = cnt2[i];
    for (int i = tid; i <= nu2; i += NT) rw.meta[kLbCells + i] = ul2[i];
    g.sync();
    return lb_level<P, NT, 2>(g, rw, nu2, rw.meta + kLbCells, rw.meta, st0, cell_lo, w, smem);
}

template <class P>
__global__ void __launch_bounds__(kLbThreads, 2) k_long_bucket(RowJob j) {
    using T = typename P::T;
    using In = typename P::In;
    using L_ = LbSmem<P>;
    constexpr int NT = kLbThreads;
    constexpr int KH = 8;   // products per thread per step: histogram
    constexpr int KS = 4;   // ... scatter
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ws[NT / 32 + 1];
    BlockGrp<NT> g;
    g.ws = ws;
    int32_t *cnt = reinterpret_cast<int32_t *>(smem + L_::kCnt);
    int32_t *ul = reinterpret_cast<int32_t *>(smem + L_::kUl);
    int32_t *s_q0 = reinterpret_cast<int32_t *>(smem + L_::kQ0);
    int32_t *s_off = reinterpret_cast<int32_t *>(smem + L_::kOff);
    In *s_a = reinterpret_cast<In *>(smem + L_::kA);
    int32_t *doff = reinterpret_cast<int32_t *>(smem + L_::kDoff);
    constexpr int NW = NT / 32;
    __shared__ int s_next, s_nd;
    const int64_t ncols = j.bcols;
    const int sh = lb_shift(ncols);
    const int ncell = (int)(((ncols > 0 ? ncols - 1 : 0) >> sh) + 1);
    const int win = 1 << (16 - sh);
    for (int r = blockIdx.x; r < j.count; r += gridDim.x) {
        const int row = j.rows[r];
        const RowIn<In> ri = row_in<In>(j, row);
        const int L = ri.L;
        const int64_t n = j.slot_nprod[r];
        const int lbits = L > 1 ? lb_bitlen((uint64_t)(L - 1)) : 0;
        unsigned char *ap = reinterpret_cast<unsigned char *>(j.arena) + j.arena_off[r];
        const LbLayout lay = lb_layout<P>(n, L);
        const int64_t obeg = j.out_rp[row];
        LbRow<P> rw;
        rw.k1 = reinterpret_cast<uint32_t *>(ap + lay.k1);
        rw.v1 = reinterpret_cast<T *>(ap + lay.v1);
        rw.k2 = reinterpret_cast<uint32_t *>(ap + lay.k2);
        rw.v2 = reinterpret_cast<T *>(ap + lay.v2);
        rw.slots = reinterpret_cast<T *>(ap + lay.slots);
        rw.meta = reinterpret_cast<int32_t *>(ap + lay.meta);
        rw.L = L;
        rw.lbits = lbits;
        rw.sh = sh;
        rw.out = LbOut<P>{j.out_col + obeg, static_cast<typename P::Out *>(j.out_val) + obeg, j.out_rp[row + 1] - obeg};
        uint32_t *k1 = rw.k1;
        T *v1 = rw.v1;
        // 1. histogram of the row's products over the cells
        for (int d = threadIdx.x; d < kLbCells; d += NT) cnt[d] = 0;
        g.sync();
        for (int t0 = 0; t0 < L; t0 += NT) {
            const int nc = min(NT, L - t0);
            const int tot = lb_load_chunk<In, NT>(g, ri, t0, s_q0, s_off, nullptr);
            for (int base = 0; base < tot; base += NT * KH) {
                const int p0 = base + (int)threadIdx.x * KH;
                if (p0 < tot) {
                    int tl[KH], q[KH];
                    lb_locate<KH>(s_off, s_q0, nc, tot, p0, tl, q);
                    int32_t c[KH];
#pragma unroll
                    for (int k = 0; k < KH; ++k) c[k] = q[k] >= 0 ? __ldg(ri.bcol + q[k]) : 0;
#pragma unroll
                    for (int k = 0; k < KH; ++k) {
                        if (q[k] >= 0) {
                            const uint32_t d = (uint32_t)c[k] >> sh;
                            atomicAdd(&cnt[d < (uint32_t)ncell ? d : ncell - 1], 1);
                        }
                    }
                }
            }
            g.sync();
        }
        // 2. units
        const int nu = lb_plan<NT>(g, cnt, ncell, ul, win);
        // 3. scatter the products to their cells' regions
        for (int t0 = 0; t0 < L; t0 += NT) {
            const int nc = min(NT, L - t0);
            const int tot = lb_load_chunk<In, NT>(g, ri, t0, s_q0, s_off, s_a);
            for (int base = 0; base < tot; base += NT * KS) {
                const int p0 = base + (int)threadIdx.x * KS;
                if (p0 < tot) {
                    int tl[KS], q[KS];
                    lb_locate<KS>(s_off, s_q0, nc, tot, p0, tl, q);
                    int32_t c[KS];
                    In bv[KS];
#pragma unroll
                    for (int k = 0; k < KS; ++k) {
                        if (q[k] >= 0) {
                            c[k] = __ldg(ri.bcol + q[k]);
                            bv[k] = __ldg(ri.bval + q[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < KS; ++k) {
                        if (q[k] >= 0) {
                            const uint32_t d0 = (uint32_t)c[k] >> sh;
                            const int d = d0 < (uint32_t)ncell ? (int)d0 : ncell - 1;
                            const int pos = atomicAdd(&cnt[d], 1);
                            if (pos < n) {   // always true: both passes enumerate the same products
                                k1[pos] = ((uint32_t)c[k] << 16) | (uint32_t)(t0 + tl[k]);
                                v1[pos] = P::mul(s_a[tl[k]], bv[k]);
                            }
                        }
                    }
                }
            }
            g.sync();
        }
        // 4. distinct columns of every cell (one warp per cell, a bitmap of the
        //    cell's columns in the warp's staging slots); cell d ends at cnt[d]
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        uint32_t *sk = reinterpret_cast<uint32_t *>(smem + L_::kStageK) + warp * kLbUnit;
        T *sv = reinterpret_cast<T *>(smem + L_::kStageV) + warp * kLbUnit;
        {
            const int cw = 1 << sh, words = (cw + 31) >> 5;
            for (int d = warp; d < ncell; d += NW) {
                const int st = d ? cnt[d - 1] : 0, m = cnt[d] - st;
                if (m <= 1) {
                    if (lane == 0) doff[d] = m;
                    continue;
                }
                for (int i = lane; i < words; i += 32) sk[i] = 0u;
                __syncwarp();
                for (int i = lane; i < m; i += 32) {
                    const uint32_t c = (k1[st + i] >> 16) & (uint32_t)(cw - 1);
                    atomicOr(&sk[c >> 5], 1u << (c & 31));
                }
                __syncwarp();
                int x = 0;
                for (int i = lane; i < words; i += 32) x += __popc(sk[i]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) doff[d] = x;
                __syncwarp();
            }
        }
        if (threadIdx.x == 0) {
            s_next = 0;
            s_nd = 0;
        }
        g.sync();
        // 5. output offsets of the cells
        int64_t w;
        {
            constexpr int PER = kLbCells / NT;
            int c[PER], sum = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int d = threadIdx.x * PER + e;
                c[e] = d < ncell ? doff[d] : 0;
                sum += c[e];
            }
            int tot;
            int ex = g.scan_excl(sum, tot);
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int d = threadIdx.x * PER + e;
                if (d < ncell) doff[d] = ex;
                ex += c[e];
            }
            w = tot;
        }
        g.sync();
        // 6. the units, taken by the warps one at a time
        const int64_t dcap = lb_defer_cap(n);
        LbDefer *dl = reinterpret_cast<LbDefer *>(ap + lay.defer);
        LbRowArgs<P> ra{rw.k1, rw.k2, rw.v1, rw.v2, lbits, rw.out, j.err};
        int32_t *wm = reinterpret_cast<int32_t *>(ap + lay.wmeta) + warp * kLbWmeta;
        for (;;) {
            int u = 0;
            if (lane == 0) u = atomicAdd(&s_next, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= nu) break;
            const int d0 = ul[u], d1 = ul[u + 1];
            const int st = d0 ? cnt[d0 - 1] : 0, en = cnt[d1 - 1], m = en - st;
            if (m == 0) continue;
            const int64_t ob = doff[d0], cl = (int64_t)d0 << sh;
            if (m <= kLbUnit) lb_wunit<P>(k1 + st, v1 + st, m, cl, lbits, rw.out, ob, sk, sv);
            else if (sh == 0) lb_defer(dl, &s_nd, dcap, kLbDeferGiant1, st, m, cl, ob, j.err);
            else if (sh <= 8) lb_whot<P>(ra, st, m, cl, 1 << sh, ob, sk, sv, wm, dl, &s_nd, dcap);
            else lb_defer(dl, &s_nd, dcap, kLbDeferHot, st, m, cl, ob, j.err);
        }
        g.sync();
        // 7. the deferred work, by the whole block: hot cells of more than 256
        //    columns (split and processed as level 2), then giant columns
        const int nd = min(s_nd, (int)dcap);
        for (int i = 0; i < nd; ++i) {
            const LbDefer e = dl[i];
            if (e.kind == kLbDeferHot) lb_hot<P, NT>(g, rw, e.st, e.m, e.col, e.ob, smem);
        }
        for (int i = 0; i < nd; ++i) {
            const LbDefer e = dl[i];
            if (e.kind == kLbDeferHot) continue;
            const uint32_t *gk = e.kind == kLbDeferGiant1 ? rw.k1 : rw.k2;
            const T *gv = e.kind == kLbDeferGiant1 ? rw.v1 : rw.v2;
            lb_giant<P, NT>(g, gk + e.st, gv + e.st, e.m, L, lbits, rw.slots, rw.out, e.ob, e.col, smem);
        }
        if (threadIdx.x == 0) {
            if (w > rw.out.cap || (j.exact && w != rw.out.cap)) atomicOr(j.err, 1u);
            if (j.out_cnt != nullptr) j.out_cnt[row] = w;
        }
        g.sync();
    }
}

template <class P>
cudaError_t launch_long_bucket(const RowJob &j, cudaStream_t st) {
    if constexpr (P::kVal) {
        const size_t sm = LbSmem<P>::kBytes;
        auto kern = k_long_bucket<P>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kern<<<j.count, kLbThreads, sm, st>>>(j);
    } else {
        const size_t sm = (size_t)kLsWinBits / 8;
        auto kern = k_long_sym<P>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kern<<<j.count, kLsThreads, sm, st>>>(j);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace brm
