// Row kernels of the row bins, built on the BRMerge row engine.
//
//   register bins  rows of at most 1024 products: brm_reg_rows.cuh.
//   warp bin   0 < nprod_i <= WCAP, L_i <= WCAP: one warp per row, ping-pong
//              buffers and list offsets in the warp's slice of shared memory.
//   block bin  nprod_i <= BCAP, L_i <= BLCAP: one thread block per row,
//              buffers in shared memory.
//   long bin   everything else: one thread block per row; by column buckets
//              (brm_long_rows.cuh) or by merge rounds in a device-memory
//              arena slice given per row by the host (this file), each round
//              tile by tile through shared memory (merge_round_tiled).
// Rows are taken from the bin's row list in a grid-stride loop.
#pragma once

#include "brm_engine.cuh"
#include "brm_internal.h"
#include "brm_long_rows.cuh"
#include "brm_long_tiles.cuh"
#include "brm_reg_rows.cuh"

namespace brm {

constexpr int kWarpK = 8;        // diagonals per thread per tile, warp kernel
constexpr int kWarpUnr = 4;      // products gathered per thread at a time
constexpr int kWarpsPerBlock = 8;
constexpr int kBlockThreads = 256;
constexpr int kBlockK = 8;
constexpr int kLongThreads = 512;
// diagonals per thread in the long-row kernel: the value passes use 4 (so
// that two 512-thread blocks fit an SM), the index-only symbolic pass 8
template <class P>
__host__ __device__ constexpr int long_k() { return P::kVal ? 4 : 8; }

// Shared-memory bytes of one row buffer pair holding `cap` elements and
// `lcap` lists: two value arrays, two column arrays, two offset arrays.  The
// bins guarantee L <= lcap <= cap, so the spare value array can hold one A
// value per list during the multiplying phase.
template <class P>
__host__ __device__ constexpr size_t pair_bytes(int cap, int lcap) {
    return (P::kVal ? align_up(2 * sizeof(typename P::T) * (size_t)cap, 16) : 0) +
           align_up(2 * sizeof(int32_t) * (size_t)cap, 16) + align_up(2 * sizeof(int32_t) * (size_t)(lcap + 1), 16);
}

template <class P>
__device__ __forceinline__ void carve(unsigned char *p, int cap, int lcap, Buf<P> &b0, Buf<P> &b1) {
    using T = typename P::T;
    if constexpr (P::kVal) {
        b0.val = reinterpret_cast<T *>(p);
        b1.val = b0.val + cap;
        p += align_up(2 * sizeof(T) * (size_t)cap, 16);
    } else {
        b0.val = nullptr;
        b1.val = nullptr;
    }
    b0.col = reinterpret_cast<int32_t *>(p);
    b1.col = b0.col + cap;
    p += align_up(2 * sizeof(int32_t) * (size_t)cap, 16);
    b0.off = reinterpret_cast<int32_t *>(p);
    b1.off = b0.off + (lcap + 1);
}

static_assert(kBlockLCap <= kBlockCap, "block bin: list capacity must not exceed element capacity");

template <class P, int WCAP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 3) k_rows_warp(RowJob j) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5;
    Buf<P> b0, b1;
    carve<P>(smem + (size_t)wid * pair_bytes<P>(WCAP, WCAP), WCAP, WCAP, b0, b1);
    const WarpGrp g;
    for (int r = blockIdx.x * kWarpsPerBlock + wid; r < j.count; r += gridDim.x * kWarpsPerBlock)
        brm_row<P, WarpGrp, kWarpK, kWarpUnr>(g, j.rows[r], j, b0, b1);
}

template <class P, int BCAP, int BLCAP>
__global__ void __launch_bounds__(kBlockThreads, 2) k_rows_block(RowJob j) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ws[kBlockThreads / 32 + 1];
    Buf<P> b0, b1;
    carve<P>(smem, BCAP, BLCAP, b0, b1);
    BlockGrp<kBlockThreads> g;
    g.ws = ws;
    for (int r = blockIdx.x; r < j.count; r += gridDim.x)
        brm_row<P, BlockGrp<kBlockThreads>, kBlockK, 4>(g, j.rows[r], j, b0, b1);
}

// ---------------------------------------------------------------------------
// Symbolic pass of the warp and block bins by hashing (option symbolic_hash),
// the paper's symbolic step (Section III-D-2, step 3): every column of the
// row's lists goes into a shared-memory open-addressing table of twice the
// bin's product capacity (multiplicative hash, linear probing, load factor
// <= 1/2); the row's nnz is the number of first insertions.  The products
// are spread evenly over the group: the list ends are prefix-summed first
// and every thread finds the list of each of its positions.  (Long rows count
// their columns in a bitmap: a table whose hash is the column itself and that
// never collides.)
// ---------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ int hash_count_row(const G &g, const RowIn<float> &ri, int32_t *tab, int hs_bits,
                                              int32_t *q0s, int32_t *offs) {
    const int L = ri.L;
    int carry = 0;
    if (g.rank() == 0) offs[0] = 0;
    for (int base = 0; base < L; base += G::N) {
        const int t = base + g.rank();
        int len = 0;
        if (t < L) {
            const int k = ri.acol[t];
            const int q0 = ri.brp[k];
            len = ri.brp[k + 1] - q0;
            q0s[t] = q0;
        }
        int tot;
        const int ex = g.scan_excl(len, tot);
        if (t < L) offs[t + 1] = carry + ex + len;
        carry += tot;
    }
    const int hs = 1 << hs_bits;
    for (int x = g.rank(); x < hs; x += G::N) tab[x] = -1;
    g.sync();
    const int N = carry;
    int cnt = 0;
    for (int p = g.rank(); p < N; p += G::N) {
        const int t = find_last_le(offs, L, p);
        const int32_t c = __ldg(ri.bcol + q0s[t] + (p - offs[t]));
        unsigned h = ((uint32_t)c * 0x9E3779B1u) >> (32 - hs_bits);
        while (true) {
            const int old = atomicCAS(tab + h, -1, c);
            if (old == -1) { ++cnt; break; }
            if (old == c) break;
            h = (h + 1) & (unsigned)(hs - 1);
        }
    }
    int total;
    g.scan_excl(cnt, total);
    return total;
}

constexpr int kHashWarpBits = 9;     // 512 slots: twice the warp bin's 256 products
constexpr int kHashBlockBits = 13;   // 8192 slots: twice the block bin's 4096 products
static_assert((1 << kHashWarpBits) >= 2 * kWarpCap && (1 << kHashBlockBits) >= 2 * kBlockCap, "load <= 1/2");

__host__ __device__ constexpr size_t hash_grp_bytes(int bits, int lcap) {
    return sizeof(int32_t) * ((size_t)(1 << bits) + 2 * (size_t)lcap + 1);
}

template <class P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_sym_hash_warp(RowJob j) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wid = threadIdx.x >> 5;
    int32_t *tab = reinterpret_cast<int32_t *>(smem + (size_t)wid * hash_grp_bytes(kHashWarpBits, kWarpCap));
    int32_t *q0s = tab + (1 << kHashWarpBits);
    int32_t *offs = q0s + kWarpCap;
    const WarpGrp g;
    for (int r = blockIdx.x * kWarpsPerBlock + wid; r < j.count; r += gridDim.x * kWarpsPerBlock) {
        const int row = j.rows[r];
        const int n = hash_count_row(g, row_in<float>(j, row), tab, kHashWarpBits, q0s, offs);
        if (g.rank() == 0 && j.out_cnt != nullptr) j.out_cnt[row] = n;
        __syncwarp();
    }
}

template <class P>
__global__ void __launch_bounds__(kBlockThreads) k_sym_hash_block(RowJob j) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ws[kBlockThreads / 32 + 1];
    int32_t *tab = reinterpret_cast<int32_t *>(smem);
    int32_t *q0s = tab + (1 << kHashBlockBits);
    int32_t *offs = q0s + kBlockLCap;
    BlockGrp<kBlockThreads> g;
    g.ws = ws;
    for (int r = blockIdx.x; r < j.count; r += gridDim.x) {
        const int row = j.rows[r];
        const int n = hash_count_row(g, row_in<float>(j, row), tab, kHashBlockBits, q0s, offs);
        if (threadIdx.x == 0 && j.out_cnt != nullptr) j.out_cnt[row] = n;
        __syncthreads();
    }
}

template <class K>
cudaError_t launch_grp_kernel(K kern, int threads, size_t sm, int rows_per_block, const RowJob &j, cudaStream_t st,
                              int sms) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, sm);
    const int need = (j.count + rows_per_block - 1) / rows_per_block;
    const int grid = max(1, min(need, sms * max(occ, 1)));
    kern<<<grid, threads, sm, st>>>(j);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// Arena layout of one long row with n products and L lists; host and device
// both use it.  The value arrays hold max(n, L) entries because the
// multiplying phase parks one A value per list in the spare buffer (a row may
// have more lists than products when many B rows are empty).
struct LongLayout {
    size_t val1, col0, col1, off0, off1, total;
};

template <class P>
__host__ __device__ constexpr LongLayout long_layout(int64_t n, int64_t L) {
    const size_t nv = (size_t)(n > L ? n : L);
    const size_t vb = P::kVal ? align_up(sizeof(typename P::T) * nv, 256) : 0;
    const size_t cb = align_up(sizeof(int32_t) * (size_t)n, 256);
    const size_t ob = align_up(sizeof(int32_t) * (size_t)(L + 1), 256);
    return LongLayout{vb, 2 * vb, 2 * vb + cb, 2 * vb + 2 * cb, 2 * vb + 2 * cb + ob, 2 * vb + 2 * cb + 2 * ob};
}

template <class P>
__host__ __device__ constexpr size_t long_row_bytes(int64_t n, int64_t L) { return long_layout<P>(n, L).total; }

template <class P>
__global__ void __launch_bounds__(kLongThreads, 2) k_rows_long(RowJob j) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ int ws[kLongThreads / 32 + 1];
    __shared__ int s_next;
    BlockGrp<kLongThreads> g;
    g.ws = ws;
    using T = typename P::T;
    // persistent blocks (long_grid > 0): slot blockIdx.x first, then slots
    // from the counter, all in this block's arena; else one slot per block
    const bool pers = j.long_grid > 0;
    unsigned char *p = reinterpret_cast<unsigned char *>(j.arena) + j.arena_off[blockIdx.x];
    for (int r = blockIdx.x; r < j.count;) {
        const int row = j.rows[r];
        const int64_t n = j.slot_nprod[r];
        const int L = row_in<typename P::In>(j, row).L;
        const LongLayout lay = long_layout<P>(n, L);
        Buf<P> b0, b1;
        if constexpr (P::kVal) {
            b0.val = reinterpret_cast<T *>(p);
            b1.val = reinterpret_cast<T *>(p + lay.val1);
        } else {
            b0.val = nullptr;
            b1.val = nullptr;
        }
        b0.col = reinterpret_cast<int32_t *>(p + lay.col0);
        b1.col = reinterpret_cast<int32_t *>(p + lay.col1);
        b0.off = reinterpret_cast<int32_t *>(p + lay.off0);
        b1.off = reinterpret_cast<int32_t *>(p + lay.off1);
        brm_row<P, BlockGrp<kLongThreads>, long_k<P>(), 4, true>(g, row, j, b0, b1, tsm);
        if (!pers) break;
        if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(j.long_ctr, 1);
        __syncthreads();
        r = s_next;
        __syncthreads();   // s_next is rewritten only after every thread has read it
    }
}

// ---------------------------------------------------------------------------
// Launchers (grid sized to the SM count times the resident blocks per SM).
// ---------------------------------------------------------------------------
template <class P>
cudaError_t launch_rows_t(int bin, const RowJob &j, cudaStream_t st) {
    if (j.count <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (bin == kBinRegTop) {
        RowJob jt = j;
        jt.reg_keys = 2 * j.reg_keys;
        return launch_reg_rows<P>(32, jt, st, sms);
    }
    if (bin >= kBinReg0 && bin < kBinReg0 + kNumRegBins) return launch_reg_rows<P>(reg_bin_tpr(bin), j, st, sms);
    if constexpr (!P::kVal && !P::kPerm) {
        // symbolic pass by hashing, on request
        if (j.sym_hash && bin == kBinWarp)
            return launch_grp_kernel(k_sym_hash_warp<PIdx>, kWarpsPerBlock * 32,
                                     kWarpsPerBlock * hash_grp_bytes(kHashWarpBits, kWarpCap), kWarpsPerBlock, j, st,
                                     sms);
        if (j.sym_hash && bin == kBinBlock)
            return launch_grp_kernel(k_sym_hash_block<PIdx>, kBlockThreads, hash_grp_bytes(kHashBlockBits, kBlockLCap), 1, j,
                                     st, sms);
    }
    if (bin == kBinWarp) {
        const size_t sm = kWarpsPerBlock * pair_bytes<P>(kWarpCap, kWarpCap);
        auto kern = k_rows_warp<P, kWarpCap>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarpsPerBlock * 32, sm);
        const int need = (j.count + kWarpsPerBlock - 1) / kWarpsPerBlock;
        const int grid = max(1, min(need, sms * max(occ, 1)));
        kern<<<grid, kWarpsPerBlock * 32, sm, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return cudaGetLastError();
    }
    if (bin == kBinBlock) {
        const size_t sm = pair_bytes<P>(kBlockCap, kBlockLCap);
        auto kern = k_rows_block<P, kBlockCap, kBlockLCap>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlockThreads, sm);
        const int grid = max(1, min(j.count, sms * max(occ, 1)));
        kern<<<grid, kBlockThreads, sm, st>>>(j);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return cudaGetLastError();
    }
    // long rows: by column tiles, by column buckets, or one block per row
    if (j.tiles != nullptr) return launch_long_tiles<P>(j, st);
    if (j.long_bucket) return launch_long_bucket<P>(j, st);
    {
        const size_t sm = TiledRoundSmem<P, kLongThreads, long_k<P>()>::kBytes;
        cudaError_t e = cudaFuncSetAttribute(k_rows_long<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        const int grid = j.long_grid > 0 ? min(j.long_grid, j.count) : j.count;
        k_rows_long<P><<<grid, kLongThreads, sm, st>>>(j);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// Arena bytes of one long row: the bucket kernels (the symbolic one needs
// none) or the merge rounds.
template <class P>
size_t long_bytes_t(int64_t n, int64_t L, bool bucket) {
    if (bucket) return P::kVal ? lb_layout<P>(n).total : 256;
    return long_row_bytes<P>(n, L);
}

}  // namespace brm
