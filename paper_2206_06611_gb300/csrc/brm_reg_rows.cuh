// Register-resident BRMerge rows: nprod_i <= 32 * TPR and L_i <= 8 * TPR for
// TPR = 1, 2, 4, ..., 32 threads per row.
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
//      threads x 32 keys; stages across threads exchange keys by warp
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

constexpr int kRegWarps = 4;                 // warps per block
constexpr int kRegU = 8;                     // products gathered per thread at a time
constexpr uint32_t kKeyPad = 0xffffffffu;    // sorts after every real key
// Per warp: a 32 x 33-word tile for the sorted keys (padded against bank
// conflicts), which also holds the rows' list descriptors during the gather.
constexpr size_t kRegStageBytes = 32 * 33 * 4 + 128;
constexpr int kRegMaxDepth = 12;             // tree stack: log2(256 lists) + 1 levels suffice

__host__ __device__ constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x >> 1); }

template <int TPR>
struct RegCfg {
    static constexpr int CAP = kRegE * TPR;                 // products per row
    static constexpr int LCAP = kRegListsPerThread * TPR;   // lists per row
    static constexpr int SB = 5 + ilog2_c(TPR);             // bits of the position in a key
    static constexpr int RPW = 32 / TPR;                    // rows per warp
    static constexpr size_t DESC = 16 * (size_t)LCAP + 8;   // descriptor bytes per row
    static_assert(RPW * DESC <= kRegStageBytes, "list descriptors must fit the staging tile");
};

// Shared memory of one warp: staging tile, then (numeric passes) the parked
// products and their list indices for the warp's 32 * 32 positions.
template <class P>
__host__ __device__ constexpr size_t reg_warp_bytes() {
    return kRegStageBytes + (P::kVal ? (sizeof(typename P::T) + sizeof(uint16_t)) * 32 * kRegE : 0);
}

__device__ __forceinline__ void cmpswap(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Ascending bitonic sort of the CAP = 32 * TPR keys of a row; thread t of the
// row holds sorted positions 32 t .. 32 t + 31 in key[0..31] afterwards.  Each
// merge stage k starts with a "flip" (position x against x ^ (k - 1)) and
// continues with half cleaners (x against x ^ j), the smaller key always to
// the lower position.
template <int TPR>
__device__ __forceinline__ void reg_bitonic_sort(uint32_t (&key)[kRegE], int t) {
    constexpr int E = kRegE, CAP = E * TPR;
    constexpr unsigned kFull = 0xffffffffu;
#pragma unroll
    for (int k = 2; k <= CAP; k <<= 1) {
        if (k <= E) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int ip = i ^ (k - 1);
                if (ip > i) cmpswap(key[i], key[ip]);
            }
        } else {
            // partner: element E-1-i of thread t ^ m
            const int m = (k - 1) >> 5;
            const bool lower = (t & (k >> 6)) == 0;
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
                const int m = jj >> 5;
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

__device__ __forceinline__ uint32_t reg_sorted_key(const uint32_t *stage, int rowbase, int pos) {
    return stage[(pos & 31) * 33 + rowbase + (pos >> 5)];
}

// Tree-order sum of a run of equal columns starting at sorted position P0:
// leaves in list order, two neighbours meet at the level bitlen(l1 ^ l2); a
// stack of partial sums whose separating levels strictly decrease is reduced
// whenever the next leaf is separated by a higher level.
template <class P, int SB>
__device__ __noinline__ typename P::T reg_tree_reduce(const uint32_t *stage, int rowbase, int P0, int N,
                                                      const typename P::T *vals, const uint16_t *lidx) {
    using T = typename P::T;
    constexpr uint32_t SMASK = (1u << SB) - 1u;
    T V[kRegMaxDepth];
    int G[kRegMaxDepth];
    const uint32_t c = reg_sorted_key(stage, rowbase, P0) >> SB;
    int nv = 0, prev_l = 0;
    for (int pos = P0; pos < N; ++pos) {
        const uint32_t kk = reg_sorted_key(stage, rowbase, pos);
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

template <class P, int TPR>
__global__ void __launch_bounds__(kRegWarps * 32) k_rows_reg(RowJob j) {
    using Cf = RegCfg<TPR>;
    using In = typename P::In;
    using T = typename P::T;
    using Out = typename P::Out;
    constexpr int E = kRegE;
    constexpr int SB = P::kVal ? Cf::SB : 0;   // the symbolic pass sorts bare columns
    constexpr uint32_t SMASK = (1u << Cf::SB) - 1u;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int rho = lane / TPR, t = lane % TPR, rowbase = rho * TPR;
    unsigned char *wb = smem + (size_t)wid * reg_warp_bytes<P>();
    uint32_t *stage = reinterpret_cast<uint32_t *>(wb);
    unsigned char *desc = wb + (size_t)rho * Cf::DESC;
    In *d_a = reinterpret_cast<In *>(desc);
    int32_t *d_q0 = reinterpret_cast<int32_t *>(desc + 8 * Cf::LCAP);
    int32_t *d_off = reinterpret_cast<int32_t *>(desc + 12 * Cf::LCAP);
    T *vals = nullptr;
    uint16_t *lidx = nullptr;
    if constexpr (P::kVal) {
        vals = reinterpret_cast<T *>(wb + kRegStageBytes) + rho * Cf::CAP;
        lidx = reinterpret_cast<uint16_t *>(wb + kRegStageBytes + sizeof(T) * 32 * E) + rho * Cf::CAP;
    }
    const In *aval = static_cast<const In *>(j.aval);
    const In *bval = static_cast<const In *>(j.bval);
    const int stride = gridDim.x * kRegWarps * Cf::RPW;

    for (int r0 = (blockIdx.x * kRegWarps + wid) * Cf::RPW; r0 < j.count; r0 += stride) {
        const int slot = r0 + rho;
        const bool has_row = slot < j.count;
        const int row = has_row ? j.rows[slot] : 0;
        const int a0 = has_row ? j.arp[row] : 0;
        const int L = has_row ? j.arp[row + 1] - a0 : 0;

        // ---- list descriptors: start of B_k*, A_ik, and the list ends ------
        int carry = 0;
        for (int c0 = 0; __any_sync(kFull, c0 < L); c0 += TPR) {
            const int l = c0 + t;
            int len = 0;
            if (l < L) {
                const int k = j.acol[a0 + l];
                const int q0 = j.brp[k];
                len = j.brp[k + 1] - q0;
                d_q0[l] = q0;
                if constexpr (P::kVal) d_a[l] = aval[a0 + l];
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

        // ---- multiplying phase: position p = i * TPR + t ---------------------
        uint32_t key[E];
#pragma unroll
        for (int i = 0; i < E; ++i) key[i] = kKeyPad;
        {
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
                        c[u] = __ldg(j.bcol + q[u]);
                        if constexpr (P::kVal) v[u] = __ldg(bval + q[u]);
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
        reg_bitonic_sort<TPR>(key, t);

        if constexpr (!P::kVal) {
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
            for (int jj = 0; __any_sync(kFull, jj * TPR < N); ++jj) {
                const int pos = jj * TPR + t;
                bool live = false;
                uint32_t kk = kKeyPad;
                if (pos < N) {
                    kk = reg_sorted_key(stage, rowbase, pos);
                    live = pos == 0 || (reg_sorted_key(stage, rowbase, pos - 1) >> SB) != (kk >> SB);
                }
                const unsigned msk = __ballot_sync(kFull, live) & gmask;
                if (live) {
                    const int w = count + __popc(msk & lt);
                    const uint32_t c = kk >> SB;
                    T v;
                    if (pos + 1 >= N || (reg_sorted_key(stage, rowbase, pos + 1) >> SB) != c)
                        v = vals[kk & SMASK];
                    else
                        v = reg_tree_reduce<P, SB>(stage, rowbase, pos, N, vals, lidx);
                    if (w < cap) {
                        ocol[w] = (int32_t)c;
                        oval[w] = P::fin(v);
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

template <class P, int TPR>
cudaError_t launch_reg_t(const RowJob &j, cudaStream_t st, int sms) {
    const size_t sm = kRegWarps * reg_warp_bytes<P>();
    auto kern = k_rows_reg<P, TPR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRegWarps * 32, sm);
    if (e != cudaSuccess) return e;
    const int rows_per_block = kRegWarps * RegCfg<TPR>::RPW;
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, kRegWarps * 32, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_reg_rows(int tpr, const RowJob &j, cudaStream_t st, int sms) {
    switch (tpr) {
        case 1: return launch_reg_t<P, 1>(j, st, sms);
        case 2: return launch_reg_t<P, 2>(j, st, sms);
        case 4: return launch_reg_t<P, 4>(j, st, sms);
        case 8: return launch_reg_t<P, 8>(j, st, sms);
        case 16: return launch_reg_t<P, 16>(j, st, sms);
        default: return launch_reg_t<P, 32>(j, st, sms);
    }
}

}  // namespace brm
