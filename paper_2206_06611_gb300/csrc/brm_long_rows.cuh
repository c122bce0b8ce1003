// Long rows by column buckets.
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
// once per round; here a row is read three times and its products are written
// and read once (twice in hot cells).
//
// Symbolic pass (column counts only): the row's columns are set in a
// shared-memory bitmap (one window of 2^20 columns at a time) and counted.
//
// Numeric pass, per batch of long rows, three kernels:
//  0. the bitmap kernel again, writing every row's distinct-column count per
//     cell of 2^sh columns (at most 4096 cells cover B's columns), so that
//     every cell's place in the row's output is known in advance;
//  1. one thread block per row:
//     a. histogram: the row's products are counted per cell;
//     b. plan: consecutive cells are grouped into units of at most 256
//        products -- a cut wherever the running count crosses a multiple of
//        128, before and after every cell of more than 128 products, and at
//        every aligned window of 2^16 columns;
//     c. scatter: every product goes to its cell's region of a device-memory
//        arena as a 32-bit key (the column's low 16 bits above the list
//        index) and its rounded value;
//     d. units, taken by the warps one at a time: the warp sorts its unit's
//        keys and values in registers with a bitonic network (8 per lane) and
//        reduces every run of equal columns in tree order -- by one lane
//        with a stack of partial sums when short; when long, each lane
//        reduces an aligned range of lists and the lanes' results are
//        combined as the five tree levels above them -- writing at the
//        unit's known place; a unit of a single cell of more than 256
//        products goes to a work list;
//  2. persistent thread blocks take the work list: a hot cell is counted per
//     column, planned into units the same way, copied column by column to a
//     second arena region, and its units are taken by the warps; a column of
//     more than 256 products ("giant") is reduced by the block densely: its
//     values go to one slot per list and the tree is evaluated over the slots.
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

constexpr int kLsThreads = 1024;            // bitmap kernel
constexpr int kLsWinBits = 1 << 20;         // columns per bitmap window (128 KB)
constexpr int kLbThreads = 512;             // row and work-list kernels
constexpr int kLbCells = 4096;              // histogram cells of a row
constexpr int kLbHalf = kLbUnit / 2;        // cut spacing of the plan
constexpr int kLbRunShort = 32;             // runs up to this size: one lane reduces
constexpr int kLbDepth = 18;                // giant column: partial-sum stack (tree height <= 16, +1)
constexpr uint32_t kLbPad = 0xffffffffu;    // padding key, above every real key
constexpr size_t kLbBmBytes = 8192;         // giant column: one bit per list (65536 lists)

static_assert(kLbCells % kLbThreads == 0 && kLbThreads % 32 == 0, "bucket kernel: per-thread shares must be whole");
static_assert(kLbMaxL <= 65535, "list index and column must never form the padding key");
static_assert(kLbUnit == 256, "the warp sort holds 8 keys per lane");

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

// Device-memory arena of one long row of the numeric bucket kernels: level-1
// keys and values, level-2 keys and values (hot cells), and the row's
// distinct-column count per cell.
struct LbLayout {
    size_t k1, v1, k2, v2, cells, total;
};

template <class P>
__host__ __device__ constexpr LbLayout lb_layout(int64_t n) {
    using T = typename P::T;
    const size_t kb = align_up(sizeof(uint32_t) * (size_t)n, 256);
    const size_t vb = align_up(sizeof(T) * (size_t)n, 256);
    const size_t cb = align_up(sizeof(uint16_t) * (size_t)kLbCells, 256);
    return LbLayout{0, kb, kb + vb, 2 * kb + vb, 2 * kb + 2 * vb, 2 * kb + 2 * vb + cb};
}

// Shared memory of the row kernel (dynamic part).
template <class P>
struct LbSmemRow {
    using T = typename P::T;
    using In = typename P::In;
    static constexpr int NW = kLbThreads / 32;
    static constexpr size_t kCnt = 0;                                             // int[kLbCells]
    static constexpr size_t kUl = kCnt + sizeof(int32_t) * kLbCells;              // int[kLbCells + 1]
    static constexpr size_t kDoff = align_up(kUl + sizeof(int32_t) * (kLbCells + 1), 16); // int[kLbCells]
    static constexpr size_t kQ0 = kDoff + sizeof(int32_t) * kLbCells;            // int[NT]
    static constexpr size_t kOff = kQ0 + sizeof(int32_t) * kLbThreads;            // int[NT + 1]
    static constexpr size_t kA = align_up(kOff + sizeof(int32_t) * (kLbThreads + 1), 16); // In[NT]
    static constexpr size_t kStageK = align_up(kA + sizeof(In) * kLbThreads, 16); // u32[NW][kLbUnit]
    static constexpr size_t kStageV = kStageK + sizeof(uint32_t) * NW * kLbUnit;  // T[NW][kLbUnit]
    static constexpr size_t kBytes = align_up(kStageV + sizeof(T) * NW * kLbUnit, 16);
};

// Shared memory of the work-list kernel (dynamic part); the staging slots
// double as the giant-column scratch.
template <class P>
struct LbSmemHot {
    using T = typename P::T;
    static constexpr int NW = kLbThreads / 32;
    static constexpr size_t kCnt = 0;                                             // int[kLbCells]
    static constexpr size_t kNz = kCnt + sizeof(int32_t) * kLbCells;              // int[kLbCells]
    static constexpr size_t kUl = kNz + sizeof(int32_t) * kLbCells;               // int[kLbCells + 1]
    static constexpr size_t kStageK = align_up(kUl + sizeof(int32_t) * (kLbCells + 1), 16);
    static constexpr size_t kStageV = kStageK + sizeof(uint32_t) * NW * kLbUnit;
    static constexpr size_t kStageEnd = kStageV + sizeof(T) * NW * kLbUnit;
    static constexpr size_t kGiant = kLbBmBytes + (sizeof(T) + sizeof(int32_t)) * kLbThreads;
    static constexpr size_t kBytes = align_up(kStageK + std::max(kStageEnd - kStageK, kGiant), 16);
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
// Distinct columns of each long row, by bitmap: the symbolic pass's row
// lengths (P = PIdx), or the numeric pass's counts per cell (value P).
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
                            // a column already set needs no atomic (hub columns recur in many lists)
                            if (q[k] >= 0 && c[k] >= 0 && u < wn && !(bm[u >> 5] & (1u << (u & 31))))
                                atomicOr(&bm[u >> 5], 1u << (u & 31));
                        }
                    }
                }
                g.sync();
            }
            if constexpr (P::kVal) {
                // the numeric pass's cells: 2^sh columns each, never across a window
                uint16_t *cells = reinterpret_cast<uint16_t *>(reinterpret_cast<unsigned char *>(j.arena) +
                                                               j.arena_off[r] + lb_layout<P>(j.slot_nprod[r]).cells);
                const int sh = lb_shift(ncols);
                const int d0 = (int)(w0 >> sh), nd = (int)(((int64_t)wn + (1 << sh) - 1) >> sh);
                for (int d = threadIdx.x; d < nd; d += kLsThreads) {
                    const uint32_t lo = (uint32_t)d << sh, hi = min(lo + (1u << sh), wn);
                    int c = 0;
                    for (uint32_t b = lo; b < hi;) {
                        const uint32_t wi = b >> 5, sb = b & 31, nb = min(32u - sb, hi - b);
                        const uint32_t msk = nb == 32 ? 0xffffffffu : (((1u << nb) - 1u) << sb);
                        c += __popc(bm[wi] & msk);
                        b += nb;
                    }
                    cells[d0 + d] = (uint16_t)c;
                }
            } else {
                int cnt = 0;
                for (int i = threadIdx.x; i < words; i += kLsThreads) cnt += __popc(bm[i]);
                int tot;
                g.scan_excl(cnt, tot);
                count += tot;
            }
            g.sync();   // the bitmap is cleared for the next window
        }
        if (!P::kVal && threadIdx.x == 0 && j.out_cnt != nullptr) j.out_cnt[row] = count;
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

// A column of m > kLbUnit products (keys gk, values gv in device memory):
// values go to their list's slot, present lists are marked in a bitmap, each
// thread reduces an aligned range of lists with the stack and the threads'
// results are combined as the tree levels above.  Writes one output.
// `slots` holds kLbSlots values of this block; `scratch` is shared memory of
// at most kLbBmBytes + (sizeof(T) + 4) * NT bytes.
template <class P, int NT>
__device__ __noinline__ void lb_giant(const BlockGrp<NT> &g, const uint32_t *gk, const typename P::T *gv, int m,
                                      int L, int lbits, typename P::T *slots, const LbOut<P> &out, int64_t w,
                                      int64_t col, unsigned char *scratch) {
    using T = typename P::T;
    uint32_t *bm = reinterpret_cast<uint32_t *>(scratch);
    T *pv = reinterpret_cast<T *>(scratch + kLbBmBytes);
    int32_t *pf = reinterpret_cast<int32_t *>(scratch + kLbBmBytes + sizeof(T) * NT);
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

// One record of the work list: a hot cell, or a giant column of a row whose
// cells are single columns, at [st, st + m) of the row's level-1 arrays.
struct LbWork {
    int32_t slot, kind, st, m;
    int64_t col, ob;
};
constexpr int32_t kLbWorkHot = 0, kLbWorkGiant = 1;

static_assert(sizeof(LbWork) == kLbWorkBytes, "work-list record size");

template <class P>
__global__ void __launch_bounds__(kLbThreads, 2) k_long_bucket(RowJob j) {
    using T = typename P::T;
    using In = typename P::In;
    using L_ = LbSmemRow<P>;
    constexpr int NT = kLbThreads;
    constexpr int NW = NT / 32;
    constexpr int KH = 8;   // products per thread per step: histogram
    constexpr int KS = 4;   // ... scatter
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ws[NT / 32 + 1];
    __shared__ int s_next;
    BlockGrp<NT> g;
    g.ws = ws;
    int32_t *cnt = reinterpret_cast<int32_t *>(smem + L_::kCnt);
    int32_t *ul = reinterpret_cast<int32_t *>(smem + L_::kUl);
    int32_t *doff = reinterpret_cast<int32_t *>(smem + L_::kDoff);
    int32_t *s_q0 = reinterpret_cast<int32_t *>(smem + L_::kQ0);
    int32_t *s_off = reinterpret_cast<int32_t *>(smem + L_::kOff);
    In *s_a = reinterpret_cast<In *>(smem + L_::kA);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *sk = reinterpret_cast<uint32_t *>(smem + L_::kStageK) + warp * kLbUnit;
    T *sv = reinterpret_cast<T *>(smem + L_::kStageV) + warp * kLbUnit;
    LbWork *work = static_cast<LbWork *>(j.lb_work);
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
        const LbLayout lay = lb_layout<P>(n);
        uint32_t *k1 = reinterpret_cast<uint32_t *>(ap + lay.k1);
        T *v1 = reinterpret_cast<T *>(ap + lay.v1);
        const uint16_t *cells = reinterpret_cast<const uint16_t *>(ap + lay.cells);
        const int64_t obeg = j.out_rp[row];
        const LbOut<P> out{j.out_col + obeg, static_cast<typename P::Out *>(j.out_val) + obeg,
                           j.out_rp[row + 1] - obeg};
        // a. histogram of the row's products over the cells
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
        // b. units
        const int nu = lb_plan<NT>(g, cnt, ncell, ul, win);
        // c. scatter the products to their cells' regions
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
        // d. the cells' places in the output, from their distinct-column
        //    counts; cell d now ends at cnt[d]
        int64_t len;
        {
            constexpr int PER = kLbCells / NT;
            int c[PER], sum = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int d = threadIdx.x * PER + e;
                c[e] = d < ncell ? cells[d] : 0;
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
            len = tot;
        }
        if (threadIdx.x == 0) s_next = 0;
        g.sync();
        // e. the units, taken by the warps one at a time
        for (;;) {
            int u = 0;
            if (lane == 0) u = atomicAdd(&s_next, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= nu) break;
            const int d0 = ul[u], d1 = ul[u + 1];
            const int st = d0 ? cnt[d0 - 1] : 0, m = cnt[d1 - 1] - st;
            if (m == 0) continue;
            const int64_t ob = doff[d0], cl = (int64_t)d0 << sh;
            if (m <= kLbUnit) {
                lb_wunit<P>(k1 + st, v1 + st, m, cl, lbits, out, ob, sk, sv);
            } else if (lane == 0) {
                const int i = atomicAdd(j.lb_ctr, 1);
                if (i < j.lb_cap) work[i] = LbWork{r, sh == 0 ? kLbWorkGiant : kLbWorkHot, st, m, cl, ob};
                else atomicOr(j.err, 1u);   // cannot happen: see lb_work_cap
            }
        }
        if (threadIdx.x == 0) {
            if (len > out.cap || (j.exact && len != out.cap)) atomicOr(j.err, 1u);
            if (j.out_cnt != nullptr) j.out_cnt[row] = len;
        }
        g.sync();
    }
}

// The work list of a batch (hot cells and giant columns of its rows), taken
// by persistent blocks one record at a time.
template <class P>
__global__ void __launch_bounds__(kLbThreads, 2) k_long_hot(RowJob j) {
    using T = typename P::T;
    using In = typename P::In;
    using L_ = LbSmemHot<P>;
    constexpr int NT = kLbThreads;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ws[NT / 32 + 1];
    __shared__ int s_item, s_next;
    BlockGrp<NT> g;
    g.ws = ws;
    int32_t *cnt = reinterpret_cast<int32_t *>(smem + L_::kCnt);
    int32_t *nzp = reinterpret_cast<int32_t *>(smem + L_::kNz);
    int32_t *ul = reinterpret_cast<int32_t *>(smem + L_::kUl);
    unsigned char *scratch = smem + L_::kStageK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *sk = reinterpret_cast<uint32_t *>(smem + L_::kStageK) + warp * kLbUnit;
    T *sv = reinterpret_cast<T *>(smem + L_::kStageV) + warp * kLbUnit;
    const LbWork *work = static_cast<const LbWork *>(j.lb_work);
    T *slots = static_cast<T *>(j.lb_slots) + (size_t)blockIdx.x * kLbSlots;
    const int sh = lb_shift(j.bcols);
    const int cw = 1 << sh;
    const uint32_t cmask = (uint32_t)cw - 1u;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(j.lb_ctr + 1, 1);
        g.sync();
        const int i = s_item;
        const int count = min(*(volatile int32_t *)j.lb_ctr, (int)j.lb_cap);
        if (i >= count) break;
        const LbWork wk = work[i];
        const int row = j.rows[wk.slot];
        const int L = row_in<In>(j, row).L;
        const int lbits = L > 1 ? lb_bitlen((uint64_t)(L - 1)) : 0;
        unsigned char *ap = reinterpret_cast<unsigned char *>(j.arena) + j.arena_off[wk.slot];
        const LbLayout lay = lb_layout<P>(j.slot_nprod[wk.slot]);
        const uint32_t *k1 = reinterpret_cast<const uint32_t *>(ap + lay.k1) + wk.st;
        const T *v1 = reinterpret_cast<const T *>(ap + lay.v1) + wk.st;
        uint32_t *k2 = reinterpret_cast<uint32_t *>(ap + lay.k2) + wk.st;
        T *v2 = reinterpret_cast<T *>(ap + lay.v2) + wk.st;
        const int64_t obeg = j.out_rp[row];
        const LbOut<P> out{j.out_col + obeg, static_cast<typename P::Out *>(j.out_val) + obeg,
                           j.out_rp[row + 1] - obeg};
        const int m = wk.m;
        if (wk.kind == kLbWorkGiant) {
            lb_giant<P, NT>(g, k1, v1, m, L, lbits, slots, out, wk.ob, wk.col, scratch);
            continue;
        }
        // a hot cell: products per column (one atomic per column and warp)
        for (int c = threadIdx.x; c < cw; c += NT) cnt[c] = 0;
        g.sync();
        for (int b = warp * 32; b < m; b += NT) {
            const int x = b + lane;
            const uint32_t c = x < m ? ((__ldcs(k1 + x) >> 16) & cmask) : 0xffffffffu;
            const unsigned same = __match_any_sync(kFull, c);
            if (x < m && lane == __ffs(same) - 1) atomicAdd(&cnt[c], __popc(same));
        }
        g.sync();
        const int nu = lb_plan<NT>(g, cnt, cw, ul, 0);
        // nonzero columns before each column: its place among the cell's outputs
        {
            constexpr int PER = kLbCells / NT;
            int f[PER], sum = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int c = threadIdx.x * PER + e;
                f[e] = c < cw && (c + 1 < cw ? cnt[c + 1] : m) > cnt[c] ? 1 : 0;
                sum += f[e];
            }
            int tot;
            int ex = g.scan_excl(sum, tot);
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int c = threadIdx.x * PER + e;
                if (c < cw) nzp[c] = ex;
                ex += f[e];
            }
        }
        g.sync();
        for (int b = warp * 32; b < m; b += NT) {
            const int x = b + lane;
            uint32_t key = 0;
            T val = T();
            if (x < m) {
                key = __ldcs(k1 + x);
                val = v1[x];
            }
            const uint32_t c = x < m ? ((key >> 16) & cmask) : 0xffffffffu;
            const unsigned same = __match_any_sync(kFull, c);
            const int leader = __ffs(same) - 1;
            int base = 0;
            if (x < m && lane == leader) base = atomicAdd(&cnt[c], __popc(same));
            base = __shfl_sync(kFull, base, leader);
            if (x < m) {
                const int pos = base + __popc(same & ((1u << lane) - 1u));
                k2[pos] = key;
                v2[pos] = val;
            }
        }
        if (threadIdx.x == 0) s_next = 0;
        g.sync();
        // the cell's units, taken by the warps; column c now ends at cnt[c]
        for (;;) {
            int u = 0;
            if (lane == 0) u = atomicAdd(&s_next, 1);
            u = __shfl_sync(kFull, u, 0);
            if (u >= nu) break;
            const int c0 = ul[u], c1 = ul[u + 1];
            const int st = c0 ? cnt[c0 - 1] : 0, m2 = cnt[c1 - 1] - st;
            if (m2 == 0 || m2 > kLbUnit) continue;
            lb_wunit<P>(k2 + st, v2 + st, m2, wk.col + c0, lbits, out, wk.ob + nzp[c0], sk, sv);
        }
        g.sync();
        // its giant columns, by the block
        for (int u = 0; u < nu; ++u) {
            const int c0 = ul[u], c1 = ul[u + 1];
            const int st = c0 ? cnt[c0 - 1] : 0, m2 = cnt[c1 - 1] - st;
            if (m2 > kLbUnit) lb_giant<P, NT>(g, k2 + st, v2 + st, m2, L, lbits, slots, out, wk.ob + nzp[c0], wk.col + c0,
                                             scratch);
        }
        g.sync();
    }
}

// Blocks of the work-list kernel (persistent; each owns kLbSlots slots).
inline int lb_hot_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return kLbHotPerSm * (sms > 0 ? sms : 1);
}

template <class P>
cudaError_t launch_long_bucket(const RowJob &j, cudaStream_t st) {
    cudaError_t e;
    const size_t smb = (size_t)kLsWinBits / 8;
    auto ks = k_long_sym<P>;
    if ((e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb)) != cudaSuccess) return e;
    if constexpr (P::kVal) {
        if ((e = cudaMemsetAsync(j.lb_ctr, 0, 2 * sizeof(int32_t), st)) != cudaSuccess) return e;
        ks<<<j.count, kLsThreads, smb, st>>>(j);
        auto kr = k_long_bucket<P>;
        if ((e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LbSmemRow<P>::kBytes)))
            return e;
        kr<<<j.count, kLbThreads, LbSmemRow<P>::kBytes, st>>>(j);
        auto kh = k_long_hot<P>;
        if ((e = cudaFuncSetAttribute(kh, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LbSmemHot<P>::kBytes)))
            return e;
        kh<<<lb_hot_blocks(), kLbThreads, LbSmemHot<P>::kBytes, st>>>(j);
        g_launches.fetch_add(3, std::memory_order_relaxed);
    } else {
        ks<<<j.count, kLsThreads, smb, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return cudaGetLastError();
}

}  // namespace brm
