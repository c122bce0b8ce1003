// Binning, validation, prefix sums and the Upper compaction copy.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "brm_engine.cuh"
#include "brm_internal.h"

namespace brm {

std::atomic<long long> g_launches{0};

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// ---------------------------------------------------------------------------
// Step 1 of both libraries (Section III-D; the buffer sizing that opens
// Algorithm 1): per row the intermediate-product count
// nprod_i = sum over k in A_i* of |B_k*| and the list count L_i = |A_i*|.  The paper then splits rows statically into p
// groups of equal nprod for p CPU threads (Section III-D); on the GPU rows are
// instead sorted into bins by size, each bin served by a kernel whose thread
// group and buffer location fit that size.  This pass classifies the rows and
// counts the bins (warp-aggregated atomics); k_bin_scatter then lists them.
// ---------------------------------------------------------------------------
__global__ void k_bin(BinArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int L = 0, bin = -1;
    int64_t np = 0;
    // short rows: one thread per row; a warp with a row of more than 64
    // entries instead takes its 32 rows one after another, each row's entries
    // spread over the lanes, lane r keeping row r's sum (rows of power-law
    // matrices differ by orders of magnitude in length)
    const int32_t *arp_i = a.arp, *acol_i = a.acol, *brp_i = a.brp;
    int s_i = 0, e_i = 0;
    if (i < a.m) {
        int64_t li = i;
        if (a.prods != nullptr) {
            const ProdDesc &d = a.prods[a.prod_of[i]];
            arp_i = d.arp; acol_i = d.acol; brp_i = d.brp;
            li = i - d.row0;
        }
        s_i = arp_i[li];
        e_i = arp_i[li + 1];
    }
    if (!__any_sync(kFull, e_i - s_i > 64)) {
        L = e_i - s_i;
#pragma unroll 4
        for (int p = s_i; p < e_i; ++p) {
            const int k = acol_i[p];
            np += brp_i[k + 1] - brp_i[k];
        }
    } else {
        const int64_t wbase = i - lane;
        for (int r = 0; r < 32; ++r) {
            const int64_t ir = wbase + r;
            if (ir >= a.m) break;
            const int32_t *arp = a.arp, *acol = a.acol, *brp = a.brp;
            int64_t li = ir;
            if (a.prods != nullptr) {
                const ProdDesc &d = a.prods[a.prod_of[ir]];
                arp = d.arp; acol = d.acol; brp = d.brp;
                li = ir - d.row0;
            }
            const int s = arp[li], e = arp[li + 1];
            int64_t part = 0;
            for (int p = s + lane; p < e; p += 32) {
                const int k = acol[p];
                part += brp[k + 1] - brp[k];
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(kFull, part, d);
            if (lane == r) {
                np = part;
                L = e - s;
            }
        }
    }
    if (i < a.m) {
        // threads per row a register bin would need: enough for the products
        // (E per thread) and for the lists (E/4 per thread)
        const int E = a.reg_keys, EL = a.reg_keys / kRegKeysPerList;
        const int64_t need = max((np + E - 1) / E, (int64_t)(L + EL - 1) / EL);
        if (np == 0) bin = kBinEmpty;
        else if (need <= a.reg_max_tpr) bin = kBinReg0 + (need <= 1 ? 0 : 32 - __clz((int)need - 1));
        else if (a.reg_top && np <= 64 * E && L <= 16 * E) bin = kBinRegTop;
        else if (np <= a.warp_cap && L <= a.warp_cap) bin = kBinWarp;
        else if (np <= a.block_cap && L <= a.block_lcap) bin = kBinBlock;
        else bin = kBinLong;
        if (a.nprod) a.nprod[i] = np;
        if (a.bin_of) a.bin_of[i] = (uint8_t)bin;
        if (bin == kBinEmpty && a.row_cnt) a.row_cnt[i] = 0;
        // a given output row pointer must leave an empty row an empty slot
        if (bin == kBinEmpty && a.out_rp && a.out_rp[i + 1] != a.out_rp[i]) atomicOr(a.out_err, 1u);
    }
#pragma unroll
    for (int b = 0; b < kNumBins; ++b) {
        const unsigned mask = __ballot_sync(kFull, bin == b);
        if (mask != 0u && lane == __ffs(mask) - 1) atomicAdd(&a.st->count[b], (unsigned long long)__popc(mask));
    }
    unsigned long long sum = (unsigned long long)np, mx = (unsigned long long)np, ml = (unsigned long long)L;
    unsigned long long rs = (bin >= kBinReg0 && bin < kBinReg0 + kNumRegBins) ? (unsigned long long)np : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        sum += __shfl_down_sync(kFull, sum, d);
        rs += __shfl_down_sync(kFull, rs, d);
        mx = max(mx, (unsigned long long)__shfl_down_sync(kFull, mx, d));
        ml = max(ml, (unsigned long long)__shfl_down_sync(kFull, ml, d));
    }
    if (lane == 0) {
        if (sum) atomicAdd(&a.st->total_nprod, sum);
        if (rs) atomicAdd(&a.st->reg_nprod, rs);
        atomicMax(&a.st->max_nprod, mx);
        atomicMax(&a.st->max_L, ml);
    }
}

__global__ void k_reg_nprod(int64_t m, const uint8_t *bin_of, const int64_t *nprod, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        const int b = bin_of[i];
        // a row's recorded order is padded to a multiple of 16 entries (one
        // 32-byte sector), so that every sector is written whole
        out[i] = (b >= kBinReg0 && b < kBinReg0 + kNumRegBins) ? ((nprod[i] + 15) & ~int64_t(15)) : 0;
    }
}

// Second pass: every non-empty row appends itself to its bin's segment of
// a.rows (warp-aggregated atomics on the bin's cursor).
__global__ void k_bin_scatter(BinArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int bin = i < a.m ? (int)a.bin_of[i] : -1;
#pragma unroll
    for (int b = kBinReg0; b < kNumBins; ++b) {
        const unsigned mask = __ballot_sync(kFull, bin == b);
        if (mask == 0u) continue;
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&a.st->cursor[b], (unsigned long long)__popc(mask));
        base = __shfl_sync(kFull, base, leader);
        if (bin == b) {
            const int64_t slot = (int64_t)base + __popc(mask & lanemask_lt());
            a.rows[a.base[b] + slot] = (int32_t)i;
            if (b == kBinLong && a.long_nprod) {
                const int32_t *arp = a.arp;
                int64_t li = i;
                if (a.prods != nullptr) {
                    const ProdDesc &d = a.prods[a.prod_of[i]];
                    arp = d.arp;
                    li = i - d.row0;
                }
                a.long_nprod[slot] = a.nprod[i];
                a.long_L[slot] = arp[li + 1] - arp[li];
            }
        }
    }
}

// Batched products: every stacked row learns its product.
__global__ void k_fill_prod_of(const ProdDesc *prods, const int64_t *rows_of, int32_t *prod_of) {
    const int p = blockIdx.x;
    const int64_t r0 = prods[p].row0, n = rows_of[p];
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) prod_of[r0 + r] = p;
}

// Input check (CSR with strictly ascending in-range columns per row).
__global__ void k_validate(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                           BinStats *st) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (i == 0) bad |= (rp[0] != 0) || ((int64_t)rp[rows] != nnz);
    if (i < rows) {
        const int64_t s = rp[i], e = rp[i + 1];
        if (s < 0 || s > e || e > nnz) {
            bad = true;
        } else {
            for (int64_t p = s; p < e; ++p) {
                const int32_t c = col[p];
                if (c < 0 || c >= cols || (p > s && col[p - 1] >= c)) { bad = true; break; }
            }
        }
    }
    if (bad) atomicOr(&st->bad, 1ull);
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of int64 (three passes: tile sums, scan of the tile
// sums in one block, tile scans with their offsets).
// ---------------------------------------------------------------------------
constexpr int kScanT = 256, kScanV = 8, kScanTile = kScanT * kScanV;

template <int NT>
__device__ __forceinline__ long long block_excl_scan(long long x, long long *ws, long long &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    long long v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long u = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += u;
    }
    if (lane == 31) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < NW ? ws[lane] : 0;
        const long long w0 = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long u = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += u;
        }
        if (lane < NW) ws[lane] = w - w0;
        if (lane == NW - 1) ws[NW] = w;
    }
    __syncthreads();
    const long long r = ws[wid] + v - x;
    total = ws[NW];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanT) k_scan_sums(const int64_t *in, int64_t n, long long *sums) {
    __shared__ long long ws[kScanT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int v = 0; v < kScanV; ++v) {
        const int64_t idx = base + (int64_t)v * kScanT + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    long long tot;
    block_excl_scan<kScanT>(s, ws, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long *sums, int64_t nb) {
    __shared__ long long ws[1024 / 32 + 1];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t b = b0 + threadIdx.x;
        const long long x = b < nb ? sums[b] : 0;
        long long tot;
        const long long ex = block_excl_scan<1024>(x, ws, tot);
        if (b < nb) sums[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanT) k_scan_apply(const int64_t *in, int64_t *out, int64_t n,
                                                       const long long *sums, int64_t nb) {
    __shared__ long long ws[kScanT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanV;
    long long x[kScanV];
    long long s = 0;
#pragma unroll
    for (int v = 0; v < kScanV; ++v) {
        const int64_t idx = base + v;
        x[v] = idx < n ? in[idx] : 0;
        s += x[v];
    }
    long long tot;
    long long run = block_excl_scan<kScanT>(s, ws, tot) + sums[blockIdx.x];
#pragma unroll
    for (int v = 0; v < kScanV; ++v) {
        const int64_t idx = base + v;
        if (idx < n) out[idx] = run;
        run += x[v];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

// ---------------------------------------------------------------------------
// BRMerge-Upper step 6: copy each row of C_bar to its place in C.
// ---------------------------------------------------------------------------
template <class V>
__global__ void k_compact(int64_t m, const int64_t *cbar_off, const int64_t *rp, const int32_t *ccol,
                          const V *cval, int32_t *col, V *val) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += nw) {
        const int64_t src = cbar_off[r], dst = rp[r], len = rp[r + 1] - dst;
        for (int64_t p = lane; p < len; p += 32) {
            col[dst + p] = ccol[src + p];
            val[dst + p] = cval[src + p];
        }
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

cudaError_t launch_bin(const BinArgs &a, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    const int T = 256;
    const int64_t grid = (a.m + T - 1) / T;
    k_bin<<<(unsigned)grid, T, 0, st>>>(a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_fill_prod_of(const ProdDesc *prods, const int64_t *rows_of, int32_t count, int32_t *prod_of,
                                cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_fill_prod_of<<<count, 256, 0, st>>>(prods, rows_of, prod_of);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const BinArgs &a, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    const int T = 256;
    const int64_t grid = (a.m + T - 1) / T;
    k_bin_scatter<<<(unsigned)grid, T, 0, st>>>(a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_reg_nprod(int64_t m, const uint8_t *bin_of, const int64_t *nprod, int64_t *out, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int T = 256;
    k_reg_nprod<<<(unsigned)((m + T - 1) / T), T, 0, st>>>(m, bin_of, nprod, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_validate(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                            BinStats *st, cudaStream_t stream) {
    const int T = 256;
    const int64_t grid = (rows + T) / T;   // at least one thread for the rp[0] check
    k_validate<<<(unsigned)grid, T, 0, stream>>>(rows, cols, nnz, rp, col, st);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

size_t scan_tmp_bytes(int64_t n) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(nb + 1) * sizeof(long long);
}

cudaError_t launch_scan(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    long long *sums = static_cast<long long *>(tmp);
    k_scan_sums<<<(unsigned)nb, kScanT, 0, st>>>(in, n, sums);
    k_scan_top<<<1, 1024, 0, st>>>(sums, nb);
    k_scan_apply<<<(unsigned)nb, kScanT, 0, st>>>(in, out, n, sums, nb);
    g_launches.fetch_add(3, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_compact(int64_t m, const int64_t *cbar_off, const int64_t *rp, const int32_t *cbar_col,
                           const void *cbar_val, int32_t *col, void *val, size_t vbytes, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int T = 256;
    const int64_t want = (m + (T / 32) - 1) / (T / 32);
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count() * 8);
    if (vbytes == 8)
        k_compact<double><<<grid, T, 0, st>>>(m, cbar_off, rp, cbar_col, static_cast<const double *>(cbar_val), col,
                                              static_cast<double *>(val));
    else
        k_compact<float><<<grid, T, 0, st>>>(m, cbar_off, rp, cbar_col, static_cast<const float *>(cbar_val), col,
                                             static_cast<float *>(val));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

extern cudaError_t launch_rows_f64(int bin, const RowJob &j, cudaStream_t st);
extern cudaError_t launch_rows_f32(int bin, const RowJob &j, cudaStream_t st);
extern cudaError_t launch_rows_f32c(int bin, const RowJob &j, cudaStream_t st);
extern cudaError_t launch_rows_idx(int bin, const RowJob &j, cudaStream_t st);
extern size_t long_bytes_f64(int64_t n, int64_t L, bool bucket);
extern size_t long_bytes_f32(int64_t n, int64_t L, bool bucket);
extern size_t long_bytes_f32c(int64_t n, int64_t L, bool bucket);
extern size_t long_bytes_idx(int64_t n, int64_t L, bool bucket);
extern int tile_grid_f64();
extern int tile_grid_f32();
extern int tile_grid_f32c();

cudaError_t launch_rows(VKind v, int bin, const RowJob &j, cudaStream_t st) {
    switch (v) {
        case kF64: return launch_rows_f64(bin, j, st);
        case kF32: return launch_rows_f32(bin, j, st);
        case kF32C: return launch_rows_f32c(bin, j, st);
        default: return launch_rows_idx(bin, j, st);
    }
}

size_t long_row_bytes_for(VKind v, int64_t n, int64_t L, bool bucket) {
    switch (v) {
        case kF64: return long_bytes_f64(n, L, bucket);
        case kF32: return long_bytes_f32(n, L, bucket);
        case kF32C: return long_bytes_f32c(n, L, bucket);
        default: return long_bytes_idx(n, L, bucket);
    }
}

int long_tile_grid(VKind v) {
    switch (v) {
        case kF64: return tile_grid_f64();
        case kF32: return tile_grid_f32();
        case kF32C: return tile_grid_f32c();
        default: return 0;
    }
}

// The static split of Section III-D: bounds[p] = the first row whose
// exclusive product prefix reaches floor(p * total / parts), bounds[parts] = m.
__global__ void k_row_split(const int64_t *excl, int64_t m, int32_t parts, int64_t *bounds) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > parts) return;
    if (p == parts) {
        bounds[p] = m;
        return;
    }
    const int64_t total = excl[m];
    const int64_t target = (int64_t)(((__int128)total * p) / parts);
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (excl[mid] < target) lo = mid + 1; else hi = mid;
    }
    bounds[p] = lo;
}

cudaError_t launch_row_split(const int64_t *excl, int64_t m, int32_t parts, int64_t *bounds, cudaStream_t st) {
    const int T = 256;
    k_row_split<<<(parts + T) / T, T, 0, st>>>(excl, m, parts, bounds);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace brm
