// Register-resident BRMerge rows: nprod_i <= E * TPR and L_i <= E/4 * TPR for
// TPR = 1, 2, 4, ..., 32 threads per row and E = 8, 16 or 32 keys per thread.
//
// Algorithm 1 merges a row's L sorted lists two at a time in a binary tree and
// adds the values of equal columns when their lists meet; the merging rounds
// only move elements, so the floating-point result is fixed by the tree
// alone.  After round r list t has become list t >> r (pairs (0,1), (2,3),
// ...; an odd last list is copied, Fig. 2), hence two elements of lists
// l1 < l2 with the same column meet in round bitlen(l1 ^ l2), and the value of
// a column present in lists l_1 < ... < l_s is the aligned binary-tree sum of
// their products, left subtree first, absent subtrees skipped.
//
// For short rows the same result is computed without moving (column, value)
// pairs through a buffer round after round:
//   1. multiplying phase: every product becomes a 32-bit key
//      (column << SB) | p, p = the product's position in the concatenation of
//      the lists (so p grows with the list index); the rounded product
//      A_ik * B_kj and its list index are parked in shared memory at p;
//   2. the row's keys are sorted in registers by a bitonic network (TPR
//      threads x E keys; stages across threads exchange keys by warp
//      shuffles), which puts every column's products together in list order,
//      the order the merging rounds produce;
//   3. every run of equal columns is reduced in the tree order above (a run of
//      one is its product), and the runs are written, compacted and
//      coalesced, to the row's slot in C.
// The symbolic pass sorts bare column keys and counts distinct ones.
#pragma once

#include "brm_engine.cuh"
#include "brm_internal.h"

namespace brm {

constexpr int kRegU = 8;                     // products gathered per thread at a time
constexpr uint32_t kKeyPad = 0xffffffffu;    // sorts after every real key
constexpr int kRegMaxDepth = 12;             // tree stack: log2(256 lists) + 1 levels suffice

__host__ __device__ constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x >> 1); }
__host__ __device__ constexpr size_t max_c(size_t a, size_t b) { return a > b ? a : b; }

// Per warp: an E x 33-word tile for the sorted keys (padded against bank
// conflicts), which also holds the rows' list descriptors during the gather.
__host__ __device__ constexpr size_t reg_stage_bytes(int E) {
    return max_c((size_t)E * 33 * 4, (size_t)128 * E + 256);
}

template <int TPR, int E>
struct RegCfg {
    static constexpr int CAP = E * TPR;                     // products per row
    static constexpr int LCAP = (E / 4) * TPR;              // lists per row
    static constexpr int SB = ilog2_c(CAP);                 // bits of the position in a key
    static constexpr int LE = ilog2_c(E);
    static constexpr int RPW = 32 / TPR;                    // rows per warp
    static constexpr size_t DESC = 16 * (size_t)LCAP + 8;   // descriptor bytes per row
    static_assert((1 << LE) == E && E >= 8, "E must be a power of two");
    static_assert(RPW * DESC <= reg_stage_bytes(E), "list descriptors must fit the staging tile");
};

// Shared memory of one warp: staging tile, then (numeric passes) the parked
// products and their list indices for the warp's 32 * E positions.
template <class P>
__host__ __device__ constexpr size_t reg_warp_bytes(int E) {
    return reg_stage_bytes(E) + (P::kVal ? (sizeof(typename P::T) + sizeof(uint16_t)) * 32 * (size_t)E : 0);
}

// B is gathered many times over (every row of A that names k reads B_k*) and
// C is written once: B's lines are loaded with an L2 evict-last policy and
// C is stored with the streaming (evict-first) hint.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int32_t ld_keep(const int32_t *a, uint64_t pol) {
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *a, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_keep(const float *a, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ void cmpswap(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Ascending bitonic sort of the CAP = E * TPR keys of a row; thread t of the
// row holds sorted positions E t .. E t + E - 1 in key[0..E-1] afterwards.
// Each merge stage k starts with a "flip" (position x against x ^ (k - 1)) and
// continues with half cleaners (x against x ^ j), the smaller key always to
// the lower position.
// With `presorted`, every thread's E keys are already ascending, so the
// stages of sizes k <= E (all inside a thread's registers) are skipped.
template <int TPR, int E>
__device__ __forceinline__ void reg_bitonic_sort(uint32_t (&key)[E], int t, bool presorted = false) {
    constexpr int CAP = E * TPR, LE = ilog2_c(E);
    constexpr unsigned kFull = 0xffffffffu;
#pragma unroll
    for (int k = 2; k <= CAP; k <<= 1) {
        if (k <= E && presorted) continue;
        if (k <= E) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int ip = i ^ (k - 1);
                if (ip > i) cmpswap(key[i], key[ip]);
            }
        } else {
            // partner: element E-1-i of thread t ^ m
            const int m = (k - 1) >> LE;
            const bool lower = (t & (k >> (LE + 1))) == 0;
#pragma unroll
            for (int i = 0; i < E / 2; ++i) {
                const uint32_t o1 = __shfl_xor_sync(kFull, key[E - 1 - i], m);
                const uint32_t o2 = __shfl_xor_sync(kFull, key[i], m);
                key[i] = lower ? min(key[i], o1) : max(key[i], o1);
                key[E - 1 - i] = lower ? min(key[E - 1 - i], o2) : max(key[E - 1 - i], o2);
            }
        }
#pragma unroll
        for (int jj = k >> 2; jj >= 1; jj >>= 1) {
            if (jj < E) {
#pragma unroll
                for (int i = 0; i < E; ++i)
                    if ((i & jj) == 0) cmpswap(key[i], key[i | jj]);
            } else {
                const int m = jj >> LE;
                const bool lower = (t & m) == 0;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const uint32_t o = __shfl_xor_sync(kFull, key[i], m);
                    key[i] = lower ? min(key[i], o) : max(key[i], o);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ uint32_t reg_sorted_key(const uint32_t *stage, int rowbase, int pos) {
    return stage[(pos & (E - 1)) * 33 + rowbase + (pos >> ilog2_c(E))];
}

// Tree-order sum of a run of equal columns starting at sorted position P0:
// leaves in list order, two neighbours meet at the level bitlen(l1 ^ l2); a
// stack of partial sums whose separating levels strictly decrease is reduced
// whenever the next leaf is separated by a higher level.
template <class P, int SB, int E>
__device__ __noinline__ typename P::T reg_tree_reduce(const uint32_t *stage, int rowbase, int P0, int N,
                                                      const typename P::T *vals, const uint16_t *lidx) {
    using T = typename P::T;
    constexpr uint32_t SMASK = (1u << SB) - 1u;
    T V[kRegMaxDepth];
    int G[kRegMaxDepth];
    const uint32_t c = reg_sorted_key<E>(stage, rowbase, P0) >> SB;
    int nv = 0, prev_l = 0;
    for (int pos = P0; pos < N; ++pos) {
        const uint32_t kk = reg_sorted_key<E>(stage, rowbase, pos);
        if ((kk >> SB) != c) break;
        const int p = (int)(kk & SMASK);
        const int l = lidx[p];
        if (nv > 0) {
            const int d = 32 - __clz(prev_l ^ l);
            while (nv > 1 && G[nv - 1] < d) {
                V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
                --nv;
            }
            G[nv] = d;
        }
        if (nv == kRegMaxDepth) {   // only reachable with duplicate columns inside a B row (invalid input)
            V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
            --nv;
        }
        V[nv++] = vals[p];
        prev_l = l;
    }
    while (nv > 1) {
        V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
        --nv;
    }
    return V[0];
}

template <class P, int TPR, int E>
__global__ void __launch_bounds__(256) k_rows_reg(RowJob j) {
    using Cf = RegCfg<TPR, E>;
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    // the symbolic pass sorts bare columns unless it records the rows' order
    constexpr int SB = (P::kVal || P::kPerm) ? Cf::SB : 0;
    constexpr uint32_t SMASK = (1u << Cf::SB) - 1u;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rho = lane / TPR, t = lane % TPR, rowbase = rho * TPR;
    unsigned char *wb = smem + (size_t)wid * reg_warp_bytes<P>(E);
    uint32_t *stage = reinterpret_cast<uint32_t *>(wb);
    unsigned char *desc = wb + (size_t)rho * Cf::DESC;
    In *d_a = reinterpret_cast<In *>(desc);
    int32_t *d_q0 = reinterpret_cast<int32_t *>(desc + 8 * Cf::LCAP);
    int32_t *d_off = reinterpret_cast<int32_t *>(desc + 12 * Cf::LCAP);
    T *vals = nullptr;
    uint16_t *lidx = nullptr;
    if constexpr (P::kVal) {
        vals = reinterpret_cast<T *>(wb + reg_stage_bytes(E)) + rho * Cf::CAP;
        lidx = reinterpret_cast<uint16_t *>(wb + reg_stage_bytes(E) + sizeof(T) * 32 * E) + rho * Cf::CAP;
    }
    const uint64_t keep = l2_keep_policy();
    const int stride = gridDim.x * nwarps * Cf::RPW;

    for (int r0 = (blockIdx.x * nwarps + wid) * Cf::RPW; r0 < j.count; r0 += stride) {
        const int slot = r0 + rho;
        const bool has_row = slot < j.count;
        const int row = has_row ? j.rows[slot] : 0;
        RowIn<In> ri{};
        if (has_row) ri = row_in<In>(j, row);
        const int L = has_row ? ri.L : 0;

        // ---- list descriptors: start of B_k*, A_ik, and the list ends ------
        int carry = 0, maxlen = 0;
        for (int c0 = 0; __any_sync(kFull, c0 < L); c0 += TPR) {
            const int l = c0 + t;
            int len = 0;
            if (l < L) {
                const int k = ri.acol[l];
                const int q0 = ri.brp[k];
                len = ri.brp[k + 1] - q0;
                d_q0[l] = q0;
                if constexpr (P::kVal) d_a[l] = ri.aval[l];
            }
            maxlen = max(maxlen, len);
            int incl = len;
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) {
                const int u = __shfl_up_sync(kFull, incl, d, TPR);
                if (t >= d) incl += u;
            }
            if (l < L) d_off[l + 1] = carry + incl;
            carry += __shfl_sync(kFull, incl, TPR - 1, TPR);
        }
        if (t == 0) d_off[0] = 0;
        const int N = carry;
#pragma unroll
        for (int d = TPR / 2; d > 0; d >>= 1) maxlen = max(maxlen, __shfl_xor_sync(kFull, maxlen, d, TPR));
        // every list of every row of the warp fits one thread: thread t then
        // holds list t, whose keys ascend, and the sort skips its first stages
        const bool presorted = __all_sync(kFull, !has_row || (L <= TPR && maxlen <= E));
        __syncwarp();

        // ---- multiplying phase -----------------------------------------------
        uint32_t key[E];
#pragma unroll
        for (int i = 0; i < E; ++i) key[i] = kKeyPad;
        if (presorted) {
            // thread t: the products of list t in order, positions d_off[t] + i
            const bool mine = has_row && t < L;
            const int len = mine ? d_off[t + 1] - d_off[t] : 0;
            const int q0 = mine ? d_q0[t] : 0, p0 = mine ? d_off[t] : 0;
            In a = In();
            if constexpr (P::kVal) {
                if (mine) a = d_a[t];
            }
#pragma unroll
            for (int i0 = 0; i0 < E; i0 += kRegU) {
                int32_t c[kRegU];
                In v[kRegU];
#pragma unroll
                for (int u = 0; u < kRegU; ++u) {
                    c[u] = 0;
                    v[u] = In();
                    if (i0 + u < len) {
                        c[u] = ld_keep(ri.bcol + q0 + i0 + u, keep);
                        if constexpr (P::kVal) v[u] = ld_keep(ri.bval + q0 + i0 + u, keep);
                    }
                }
#pragma unroll
                for (int u = 0; u < kRegU; ++u) {
                    const int p = p0 + i0 + u;
                    if (i0 + u < len) {
                        key[i0 + u] = ((uint32_t)c[u] << SB) | (SB > 0 ? (uint32_t)p : 0u);
                        if constexpr (P::kVal) {
                            vals[p] = P::mul(a, v[u]);
                            lidx[p] = (uint16_t)t;
                        }
                    }
                }
            }
        } else {
            // position p = i * TPR + t
            int l = 0;
#pragma unroll
            for (int i0 = 0; i0 < E; i0 += kRegU) {
                if (!__any_sync(kFull, i0 * TPR < N)) break;
                int q[kRegU];
                In a[kRegU];
#pragma unroll
                for (int u = 0; u < kRegU; ++u) {
                    const int p = (i0 + u) * TPR + t;
                    q[u] = -1;
                    a[u] = In();
                    if (p < N) {
                        while (d_off[l + 1] <= p) ++l;
                        q[u] = d_q0[l] + (p - d_off[l]);
                        if constexpr (P::kVal) {
                            a[u] = d_a[l];
                            lidx[p] = (uint16_t)l;
                        }
                    }
                }
                int32_t c[kRegU];
                In v[kRegU];
#pragma unroll
                for (int u = 0; u < kRegU; ++u) {
                    c[u] = 0;
                    v[u] = In();
                    if (q[u] >= 0) {
                        c[u] = ld_keep(ri.bcol + q[u], keep);
                        if constexpr (P::kVal) v[u] = ld_keep(ri.bval + q[u], keep);
                    }
                }
#pragma unroll
                for (int u = 0; u < kRegU; ++u) {
                    const int p = (i0 + u) * TPR + t;
                    if (q[u] >= 0) {
                        key[i0 + u] = ((uint32_t)c[u] << SB) | (SB > 0 ? (uint32_t)p : 0u);
                        if constexpr (P::kVal) vals[p] = P::mul(a[u], v[u]);
                    }
                }
            }
        }

        // ---- accumulating phase: sort, then runs of equal columns -----------
        reg_bitonic_sort<TPR, E>(key, t, presorted);

        if constexpr (P::kPerm) {
            // symbolic, recording the order: thread t holds sorted positions
            // E t .. E t + E - 1; every entry gets its product's position and
            // the run marks (neighbours across threads by shuffles), and the
            // thread stores its E entries with 16-byte streaming stores (a
            // row's segment is padded to a multiple of 16 entries), which
            // keep B's columns in L2
            const uint32_t before = __shfl_up_sync(kFull, key[E - 1], 1, TPR);
            const uint32_t after = __shfl_down_sync(kFull, key[0], 1, TPR);
            uint32_t packed[E / 2];
            int cnt = 0;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const uint32_t c = key[i] >> SB;
                const uint32_t prv = (i == 0) ? before : key[i - 1];
                const uint32_t nxt = (i + 1 < E) ? key[i + 1] : ((t + 1 < TPR) ? after : kKeyPad);
                const bool real = key[i] != kKeyPad;
                const bool start = real && ((i == 0 && t == 0) || (prv >> SB) != c);
                const bool multi = start && nxt != kKeyPad && (nxt >> SB) == c;
                const uint32_t e = real ? ((key[i] & SMASK) | (start ? kPermStart : 0u) | (multi ? kPermMulti : 0u))
                                        : 0u;
                if (i & 1) packed[i >> 1] |= e << 16; else packed[i >> 1] = e;
                cnt += start ? 1 : 0;
            }
            if (has_row) {
                const int npad = (N + 15) & ~15;
                uint4 *dst = reinterpret_cast<uint4 *>(j.perm + j.perm_off[row] + E * t);
#pragma unroll
                for (int h = 0; h < E / 8; ++h)
                    if (E * t + 8 * h < npad)
                        __stcs(dst + h, make_uint4(packed[4 * h], packed[4 * h + 1], packed[4 * h + 2],
                                                   packed[4 * h + 3]));
            }
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
            if (has_row && t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = cnt;
        } else if constexpr (!P::kVal) {
            // symbolic: distinct columns of the row
            const uint32_t before = __shfl_up_sync(kFull, key[E - 1], 1, TPR);
            int cnt = 0;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const bool first = (i == 0) ? (t == 0 || key[0] != before) : (key[i] != key[i - 1]);
                cnt += (key[i] != kKeyPad && first) ? 1 : 0;
            }
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
            if (has_row && t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = cnt;
        } else {
            __syncwarp();   // every lane is done with the descriptors (same memory)
#pragma unroll
            for (int i = 0; i < E; ++i) stage[i * 33 + lane] = key[i];
            __syncwarp();
            const int64_t obase = has_row ? j.out_rp[row] : 0;
            // the row's slot: exactly nnz(C_i*) (Precise) or nprod_i (Upper)
            const int cap = has_row ? (int)(j.out_rp[row + 1] - obase) : 0;
            int32_t *ocol = j.out_col + obase;
            Out *oval = static_cast<Out *>(j.out_val) + obase;
            const unsigned gmask = (TPR == 32) ? kFull : (((1u << TPR) - 1u) << rowbase);
            const unsigned lt = (1u << lane) - 1u;
            int count = 0;
            // sorted position pos = jj * TPR + t: consecutive threads write
            // consecutive elements of the row
            for (int jj = 0; __any_sync(kFull, jj * TPR < N); ++jj) {
                const int pos = jj * TPR + t;
                bool live = false;
                uint32_t kk = kKeyPad;
                if (pos < N) {
                    kk = reg_sorted_key<E>(stage, rowbase, pos);
                    live = pos == 0 || (reg_sorted_key<E>(stage, rowbase, pos - 1) >> SB) != (kk >> SB);
                }
                const unsigned msk = __ballot_sync(kFull, live) & gmask;
                if (live) {
                    const int w = count + __popc(msk & lt);
                    const uint32_t c = kk >> SB;
                    T v;
                    if (pos + 1 >= N || (reg_sorted_key<E>(stage, rowbase, pos + 1) >> SB) != c)
                        v = vals[kk & SMASK];
                    else
                        v = reg_tree_reduce<P, SB, E>(stage, rowbase, pos, N, vals, lidx);
                    if (w < cap) {
                        __stcs(ocol + w, (int32_t)c);
                        __stcs(oval + w, P::fin(v));
                    }
                }
                count += __popc(msk);
            }
            if (has_row) {
                if (t == 0 && (count > cap || (j.exact && count != cap))) atomicOr(j.err, 1u);
                if (t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = count;
            }
        }
        __syncwarp();   // the tile and the parked products are reused by the next rows
    }
}

// ---------------------------------------------------------------------------
// Symbolic pass of the register bins by hashing (option symbolic_hash), as the
// paper's BRMerge-Precise does its symbolic step (Section III-D-2; on GB300
// the register sort is faster): every column of the row's lists is
// inserted into a shared-memory open-addressing table of 2 * CAP slots
// (multiplicative hash, linear probing, load factor <= 1/2) and the row's
// nnz is the number of first insertions.  The count is an integer, so the
// method of counting does not change the result.
// ---------------------------------------------------------------------------
template <int E>
__host__ __device__ constexpr size_t hash_warp_bytes() {
    return reg_stage_bytes(E) + (size_t)2 * 32 * E * sizeof(int32_t);
}

template <int TPR, int E>
__global__ void __launch_bounds__(256) k_sym_hash(RowJob j) {
    using Cf = RegCfg<TPR, E>;
    constexpr int HS = 2 * Cf::CAP;                   // table slots per row
    constexpr int HB = ilog2_c(HS);
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rho = lane / TPR, t = lane % TPR;
    unsigned char *wb = smem + (size_t)wid * hash_warp_bytes<E>();
    unsigned char *desc = wb + (size_t)rho * Cf::DESC;
    int32_t *d_q0 = reinterpret_cast<int32_t *>(desc + 8 * Cf::LCAP);
    int32_t *d_off = reinterpret_cast<int32_t *>(desc + 12 * Cf::LCAP);
    int32_t *tab = reinterpret_cast<int32_t *>(wb + reg_stage_bytes(E)) + rho * HS;
    const uint64_t keep = l2_keep_policy();
    const int stride = gridDim.x * nwarps * Cf::RPW;

    for (int r0 = (blockIdx.x * nwarps + wid) * Cf::RPW; r0 < j.count; r0 += stride) {
        const int slot = r0 + rho;
        const bool has_row = slot < j.count;
        const int row = has_row ? j.rows[slot] : 0;
        RowIn<float> ri{};
        if (has_row) ri = row_in<float>(j, row);
        const int L = has_row ? ri.L : 0;
        int carry = 0;
        for (int c0 = 0; __any_sync(kFull, c0 < L); c0 += TPR) {
            const int l = c0 + t;
            int len = 0;
            if (l < L) {
                const int k = ri.acol[l];
                const int q0 = ri.brp[k];
                len = ri.brp[k + 1] - q0;
                d_q0[l] = q0;
            }
            int incl = len;
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) {
                const int u = __shfl_up_sync(kFull, incl, d, TPR);
                if (t >= d) incl += u;
            }
            if (l < L) d_off[l + 1] = carry + incl;
            carry += __shfl_sync(kFull, incl, TPR - 1, TPR);
        }
        if (t == 0) d_off[0] = 0;
        const int N = carry;
#pragma unroll 4
        for (int x = t; x < HS; x += TPR) tab[x] = -1;
        __syncwarp();
        // all of this thread's columns in flight at once
        int32_t c[E];
        {
            int l = 0;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int p = i * TPR + t;
                c[i] = -1;
                if (p < N) {
                    while (d_off[l + 1] <= p) ++l;
                    c[i] = ld_keep(ri.bcol + d_q0[l] + (p - d_off[l]), keep);
                }
            }
        }
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            if (c[i] >= 0) {
                unsigned h = ((uint32_t)c[i] * 0x9E3779B1u) >> (32 - HB);
                while (true) {
                    const int old = atomicCAS(tab + h, -1, c[i]);
                    if (old == -1) { ++cnt; break; }
                    if (old == c[i]) break;
                    h = (h + 1) & (HS - 1);
                }
            }
        }
#pragma unroll
        for (int d = 1; d < TPR; d <<= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
        if (has_row && t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = cnt;
        __syncwarp();   // the table and the descriptors are reused by the next rows
    }
}

template <int TPR, int E>
cudaError_t launch_sym_hash_t(const RowJob &j, cudaStream_t st, int sms, int warps) {
    const size_t sm = (size_t)warps * hash_warp_bytes<E>();
    auto kern = k_sym_hash<TPR, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm);
    if (e != cudaSuccess) return e;
    const int rows_per_block = warps * RegCfg<TPR, E>::RPW;
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, warps * 32, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Numeric pass of the register bins from a recorded order (BRMerge-Precise,
// whose symbolic pass sorted every row already): the products are formed in
// list order and parked at their positions, then read in the recorded order;
// a run of one is its product, a longer run is reduced in the tree order of
// Algorithm 1 (list indices of its elements, as in reg_tree_reduce).  The
// result is the one of the sorting kernel, without sorting again.
// ---------------------------------------------------------------------------
template <int E, class P>
__host__ __device__ constexpr size_t perm_warp_bytes() {
    return reg_stage_bytes(E) + (sizeof(typename P::T) + sizeof(int32_t) + sizeof(uint8_t)) * 32 * (size_t)E;
}

// Asynchronous 4- and 8-byte copies global -> shared (cp.async), loaded under
// the L2 evict-last policy like the other gathers of B.
__device__ __forceinline__ void cp_async_4(void *dst, const void *src, uint64_t pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src, uint64_t pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "l"(pol)
                 : "memory");
}
template <class In>
__device__ __forceinline__ void cp_async_val(In *dst, const In *src, uint64_t pol) {
    if constexpr (sizeof(In) == 8) cp_async_8(dst, src, pol); else cp_async_4(dst, src, pol);
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class P>
__device__ __noinline__ typename P::T perm_tree_reduce(const uint16_t *pr, int P0, int N,
                                                       const typename P::T *vals, const uint8_t *lidx) {
    using T = typename P::T;
    T V[kRegMaxDepth];
    int G[kRegMaxDepth];
    int nv = 0, prev_l = 0;
    for (int pos = P0; pos < N; ++pos) {
        const uint32_t pe = pr[pos];
        if (pos > P0 && (pe & kPermStart)) break;
        const int p = (int)(pe & kPermPos);
        const int l = lidx[p];
        if (nv > 0) {
            const int d = 32 - __clz(prev_l ^ l);
            while (nv > 1 && G[nv - 1] < d) {
                V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
                --nv;
            }
            G[nv] = d;
        }
        if (nv == kRegMaxDepth) {   // only reachable with duplicate columns inside a B row (invalid input)
            V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
            --nv;
        }
        V[nv++] = vals[p];
        prev_l = l;
    }
    while (nv > 1) {
        V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
        --nv;
    }
    return V[0];
}

template <class P, int TPR, int E>
__global__ void __launch_bounds__(256) k_rows_perm(RowJob j) {
    using Cf = RegCfg<TPR, E>;
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rho = lane / TPR, t = lane % TPR, rowbase = rho * TPR;
    unsigned char *wb = smem + (size_t)wid * perm_warp_bytes<E, P>();
    unsigned char *desc = wb + (size_t)rho * Cf::DESC;
    In *d_a = reinterpret_cast<In *>(desc);
    int32_t *d_q0 = reinterpret_cast<int32_t *>(desc + 8 * Cf::LCAP);
    int32_t *d_off = reinterpret_cast<int32_t *>(desc + 12 * Cf::LCAP);
    // one slot per product: the copied B value, then (in place) the product
    T *vals = reinterpret_cast<T *>(wb + reg_stage_bytes(E)) + rho * Cf::CAP;
    int32_t *cols = reinterpret_cast<int32_t *>(wb + reg_stage_bytes(E) + sizeof(T) * 32 * E) + rho * Cf::CAP;
    uint8_t *lidx = reinterpret_cast<uint8_t *>(wb + reg_stage_bytes(E) + (sizeof(T) + 4) * 32 * E) + rho * Cf::CAP;
    const uint64_t keep = l2_keep_policy();
    const int stride = gridDim.x * nwarps * Cf::RPW;

    for (int r0 = (blockIdx.x * nwarps + wid) * Cf::RPW; r0 < j.count; r0 += stride) {
        const int slot = r0 + rho;
        const bool has_row = slot < j.count;
        const int row = has_row ? j.rows[slot] : 0;
        RowIn<In> ri{};
        if (has_row) ri = row_in<In>(j, row);
        const int L = has_row ? ri.L : 0;
        const uint16_t *pr = j.perm + (has_row ? j.perm_off[row] : 0);

        int carry = 0;
        for (int c0 = 0; __any_sync(kFull, c0 < L); c0 += TPR) {
            const int l = c0 + t;
            int len = 0;
            if (l < L) {
                const int k = ri.acol[l];
                const int q0 = ri.brp[k];
                len = ri.brp[k + 1] - q0;
                d_q0[l] = q0;
                d_a[l] = ri.aval[l];
            }
            int incl = len;
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) {
                const int u = __shfl_up_sync(kFull, incl, d, TPR);
                if (t >= d) incl += u;
            }
            if (l < L) d_off[l + 1] = carry + incl;
            carry += __shfl_sync(kFull, incl, TPR - 1, TPR);
        }
        if (t == 0) d_off[0] = 0;
        const int N = carry;
        // this thread's recorded entries (output positions jj * TPR + t),
        // in flight while the products are gathered
        uint16_t pe[E];
#pragma unroll
        for (int jj = 0; jj < E; ++jj) {
            const int pos = jj * TPR + t;
            pe[jj] = pos < N ? __ldcs(pr + pos) : (uint16_t)0;
        }
        __syncwarp();

        // multiplying phase: every product's column and B value copied
        // asynchronously to its position p = i * TPR + t (list order)
        {
            int l = 0;
            uint8_t li[E];
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int p = i * TPR + t;
                li[i] = 0;
                if (p < N) {
                    while (d_off[l + 1] <= p) ++l;
                    const int q = d_q0[l] + (p - d_off[l]);
                    li[i] = (uint8_t)l;
                    lidx[p] = (uint8_t)l;
                    cp_async_4(cols + p, ri.bcol + q, keep);
                    cp_async_val(reinterpret_cast<In *>(vals + p), ri.bval + q, keep);
                }
            }
            cp_async_wait_all();
            // the products, each rounded, in place of the copied B values
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int p = i * TPR + t;
                if (p < N) vals[p] = P::mul(d_a[li[i]], *reinterpret_cast<const In *>(vals + p));
            }
        }
        __syncwarp();

        // accumulating phase in the recorded order
        const int64_t obase = has_row ? j.out_rp[row] : 0;
        const int cap = has_row ? (int)(j.out_rp[row + 1] - obase) : 0;
        int32_t *ocol = j.out_col + obase;
        Out *oval = static_cast<Out *>(j.out_val) + obase;
        const unsigned gmask = (TPR == 32) ? kFull : (((1u << TPR) - 1u) << rowbase);
        const unsigned lt = (1u << lane) - 1u;
        int count = 0;
#pragma unroll
        for (int jj = 0; jj < E; ++jj) {
            if (!__any_sync(kFull, jj * TPR < N)) break;
            const uint32_t e = pe[jj];
            const bool start = (e & kPermStart) != 0;
            const unsigned msk = __ballot_sync(kFull, start) & gmask;
            if (start) {
                const int w = count + __popc(msk & lt);
                const int p0 = (int)(e & kPermPos);
                T v;
                if (!(e & kPermMulti)) v = vals[p0];
                else v = perm_tree_reduce<P>(pr, jj * TPR + t, N, vals, lidx);
                if (w < cap) {
                    __stcs(ocol + w, cols[p0]);
                    __stcs(oval + w, P::fin(v));
                }
            }
            count += __popc(msk);
        }
        if (has_row) {
            if (t == 0 && (count > cap || (j.exact && count != cap))) atomicOr(j.err, 1u);
            if (t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = count;
        }
        __syncwarp();   // descriptors and copied products are reused by the next rows
    }
}

// The same numeric pass from a recorded order without staging the products:
// every run start reads its products straight from B (list index from a
// per-row table of the positions' lists, B position, column and value), four
// output positions at a time so that their loads are in flight together.
// Only the list descriptors and that table use shared memory, so many more
// warps fit an SM; used for the rows of 32-key bins, whose staged form is
// limited by shared memory.
template <class P>
__device__ __noinline__ typename P::T perm_tree_reduce_direct(const uint16_t *pr, int P0, int N, const int32_t *d_off,
                                                              const int32_t *d_q0, const typename P::In *d_a,
                                                              const uint8_t *ltab, const typename P::In *bval) {
    using T = typename P::T;
    T V[kRegMaxDepth];
    int G[kRegMaxDepth];
    int nv = 0, prev_l = 0;
    for (int pos = P0; pos < N; ++pos) {
        const uint32_t pe = pr[pos];
        if (pos > P0 && (pe & kPermStart)) break;
        const int p = (int)(pe & kPermPos);
        const int l = ltab[p];
        if (nv > 0) {
            const int d = 32 - __clz(prev_l ^ l);
            while (nv > 1 && G[nv - 1] < d) {
                V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
                --nv;
            }
            G[nv] = d;
        }
        if (nv == kRegMaxDepth) {   // only reachable with duplicate columns inside a B row (invalid input)
            V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
            --nv;
        }
        V[nv++] = P::mul(d_a[l], bval[d_q0[l] + (p - d_off[l])]);
        prev_l = l;
    }
    while (nv > 1) {
        V[nv - 2] = P::add(V[nv - 2], V[nv - 1]);
        --nv;
    }
    return V[0];
}

template <class P, int TPR, int E>
__global__ void __launch_bounds__(256, 4) k_rows_perm_direct(RowJob j) {
    using Cf = RegCfg<TPR, E>;
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    constexpr unsigned kFull = 0xffffffffu;
    // output positions whose loads are issued together: four, so that the
    // kernel fits 64 registers and four blocks of 8 warps an SM (eight
    // positions took 98 registers and two blocks; the batched mix's numeric
    // pass went from 49.2 to 44.9 ms)
    constexpr int NB = 4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int rho = lane / TPR, t = lane % TPR, rowbase = rho * TPR;
    unsigned char *desc = smem + (size_t)wid * reg_stage_bytes(E) + (size_t)rho * Cf::DESC;
    In *d_a = reinterpret_cast<In *>(desc);
    int32_t *d_q0 = reinterpret_cast<int32_t *>(desc + 8 * Cf::LCAP);
    int32_t *d_off = reinterpret_cast<int32_t *>(desc + 12 * Cf::LCAP);
    // the list of every product position of the row (at most 256 lists)
    uint8_t *ltab = smem + (size_t)nwarps * reg_stage_bytes(E) + (size_t)wid * 32 * E + (size_t)rho * Cf::CAP;
    const uint64_t keep = l2_keep_policy();
    const int stride = gridDim.x * nwarps * Cf::RPW;
    static_assert(Cf::LCAP <= 256, "list indices must fit a byte");

    for (int r0 = (blockIdx.x * nwarps + wid) * Cf::RPW; r0 < j.count; r0 += stride) {
        const int slot = r0 + rho;
        const bool has_row = slot < j.count;
        const int row = has_row ? j.rows[slot] : 0;
        RowIn<In> ri{};
        if (has_row) ri = row_in<In>(j, row);
        const int L = has_row ? ri.L : 0;
        const uint16_t *pr = j.perm + (has_row ? j.perm_off[row] : 0);

        int carry = 0;
        for (int c0 = 0; __any_sync(kFull, c0 < L); c0 += TPR) {
            const int l = c0 + t;
            int len = 0;
            if (l < L) {
                const int k = ri.acol[l];
                const int q0 = ri.brp[k];
                len = ri.brp[k + 1] - q0;
                d_q0[l] = q0;
                d_a[l] = ri.aval[l];
            }
            int incl = len;
#pragma unroll
            for (int d = 1; d < TPR; d <<= 1) {
                const int u = __shfl_up_sync(kFull, incl, d, TPR);
                if (t >= d) incl += u;
            }
            if (l < L) d_off[l + 1] = carry + incl;
            carry += __shfl_sync(kFull, incl, TPR - 1, TPR);
        }
        if (t == 0) d_off[0] = 0;
        const int N = carry;
        __syncwarp();
        {
            int l = 0;
#pragma unroll 4
            for (int i = 0; i < E; ++i) {
                const int p = i * TPR + t;
                if (p < N) {
                    while (d_off[l + 1] <= p) ++l;
                    ltab[p] = (uint8_t)l;
                }
            }
        }
        __syncwarp();

        const int64_t obase = has_row ? j.out_rp[row] : 0;
        const int cap = has_row ? (int)(j.out_rp[row + 1] - obase) : 0;
        int32_t *ocol = j.out_col + obase;
        Out *oval = static_cast<Out *>(j.out_val) + obase;
        const unsigned gmask = (TPR == 32) ? kFull : (((1u << TPR) - 1u) << rowbase);
        const unsigned lt = (1u << lane) - 1u;
        int count = 0;
        // the recorded entries of the next batch are loaded while this one is
        // processed
        uint32_t en[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int pos = b * TPR + t;
            en[b] = pos < N ? __ldcs(pr + pos) : 0u;
        }
        for (int j0 = 0; __any_sync(kFull, j0 * TPR < N); j0 += NB) {
            uint32_t e[NB];
            int q[NB], l[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                e[b] = en[b];
                const int pos = (j0 + NB + b) * TPR + t;
                en[b] = pos < N ? __ldcs(pr + pos) : 0u;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                l[b] = 0;
                q[b] = 0;
                if (e[b] & kPermStart) {
                    const int p0 = (int)(e[b] & kPermPos);
                    l[b] = ltab[p0];
                    q[b] = d_q0[l[b]] + (p0 - d_off[l[b]]);
                }
            }
            int32_t c[NB];
            In v[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                c[b] = 0;
                v[b] = In();
                if (e[b] & kPermStart) {
                    c[b] = ld_keep(ri.bcol + q[b], keep);
                    v[b] = ld_keep(ri.bval + q[b], keep);
                }
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const bool start = (e[b] & kPermStart) != 0;
                const unsigned msk = __ballot_sync(kFull, start) & gmask;
                if (start) {
                    const int w = count + __popc(msk & lt);
                    T val;
                    if (!(e[b] & kPermMulti)) val = P::mul(d_a[l[b]], v[b]);
                    else val = perm_tree_reduce_direct<P>(pr, (j0 + b) * TPR + t, N, d_off, d_q0, d_a, ltab, ri.bval);
                    if (w < cap) {
                        __stcs(ocol + w, c[b]);
                        __stcs(oval + w, P::fin(val));
                    }
                }
                count += __popc(msk);
            }
        }
        if (has_row) {
            if (t == 0 && (count > cap || (j.exact && count != cap))) atomicOr(j.err, 1u);
            if (t == 0 && j.out_cnt != nullptr) j.out_cnt[row] = count;
        }
        __syncwarp();   // the descriptors are reused by the next rows
    }
}

template <class P, int TPR, int E>
cudaError_t launch_perm_direct_t(const RowJob &j, cudaStream_t st, int sms, int warps) {
    const size_t sm = (size_t)warps * (reg_stage_bytes(E) + 32 * (size_t)E);
    auto kern = k_rows_perm_direct<P, TPR, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm);
    if (e != cudaSuccess) return e;
    const int rows_per_block = warps * RegCfg<TPR, E>::RPW;
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, warps * 32, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <class P, int TPR, int E>
cudaError_t launch_perm_t(const RowJob &j, cudaStream_t st, int sms, int warps) {
    const size_t sm = (size_t)warps * perm_warp_bytes<E, P>();
    auto kern = k_rows_perm<P, TPR, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm);
    if (e != cudaSuccess) return e;
    const int rows_per_block = warps * RegCfg<TPR, E>::RPW;
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, warps * 32, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <class P, int TPR, int E>
cudaError_t launch_reg_t(const RowJob &j, cudaStream_t st, int sms, int warps) {
    if constexpr (!P::kVal && !P::kPerm) {
        if (j.perm != nullptr) return launch_reg_t<PPerm, TPR, E>(j, st, sms, warps);
        if (j.sym_hash) return launch_sym_hash_t<TPR, E>(j, st, sms, warps);
    }
    if constexpr (P::kVal) {
        if (j.perm != nullptr) {
            // the same rows with twice the threads of half the keys (same
            // products and lists per row): more warps in flight for the gathers
            if constexpr (TPR <= 16 && E >= 16)
                if (j.num_half) return launch_perm_t<P, 2 * TPR, E / 2>(j, st, sms, warps);
            if constexpr (E >= 32)
                if (j.num_direct) return launch_perm_direct_t<P, TPR, E>(j, st, sms, warps);
            return launch_perm_t<P, TPR, E>(j, st, sms, warps);
        }
    }
    const size_t sm = (size_t)warps * reg_warp_bytes<P>(E);
    auto kern = k_rows_reg<P, TPR, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm);
    if (e != cudaSuccess) return e;
    const int rows_per_block = warps * RegCfg<TPR, E>::RPW;
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, warps * 32, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <class P, int E>
cudaError_t launch_reg_e(int tpr, const RowJob &j, cudaStream_t st, int sms, int warps) {
    switch (tpr) {
        case 1: return launch_reg_t<P, 1, E>(j, st, sms, warps);
        case 2: return launch_reg_t<P, 2, E>(j, st, sms, warps);
        case 4: return launch_reg_t<P, 4, E>(j, st, sms, warps);
        case 8: return launch_reg_t<P, 8, E>(j, st, sms, warps);
        case 16: return launch_reg_t<P, 16, E>(j, st, sms, warps);
        default: return launch_reg_t<P, 32, E>(j, st, sms, warps);
    }
}

// Register bin `tpr` with `keys` (8, 16 or 32) keys per thread and `warps`
// warps per block.
template <class P>
cudaError_t launch_reg_rows(int tpr, const RowJob &j, cudaStream_t st, int sms) {
    const int warps = (j.reg_warps >= 1 && j.reg_warps <= 8) ? j.reg_warps : 4;
    if (j.reg_keys == 8) return launch_reg_e<P, 8>(tpr, j, st, sms, warps);
    if (j.reg_keys == 16) return launch_reg_e<P, 16>(tpr, j, st, sms, warps);
    return launch_reg_e<P, 32>(tpr, j, st, sms, warps);
}

}  // namespace brm
