// Internal interfaces between the translation units of libbrm.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace brm {

struct RowJob;

// row bins (by intermediate products nprod_i and list count L_i of a row)
enum { kBinEmpty = 0, kBinWarp = 1, kBinBlock = 2, kBinLong = 3, kNumBins = 4 };

// Capacities of the shared-memory bins.
constexpr int kWarpCap = 256;     // warp bin: nprod_i <= 256 and L_i <= 256
constexpr int kBlockCap = 4096;   // block bin: nprod_i <= 4096 ...
constexpr int kBlockLCap = 1024;  // ... and L_i <= 1024

// Kernel phases recorded by the tracer (brm_trace_*).
enum Phase {
    kPhValidate = 0, kPhBin, kPhSymWarp, kPhSymBlock, kPhSymLong, kPhScan,
    kPhNumWarp, kPhNumBlock, kPhNumLong, kPhCompact, kNumPhases
};

// Kernel launches made by the library so far (all threads).
extern std::atomic<long long> g_launches;

// value kinds of a pass
enum VKind { kIdx = 0, kF64 = 1, kF32 = 2, kF32C = 3 };

cudaError_t launch_rows(VKind v, int bin, const RowJob &j, cudaStream_t st);
size_t long_row_bytes_for(VKind v, int64_t nprod, int64_t L);

// Statistics written by the binning kernel.
struct BinStats {
    unsigned long long count[kNumBins];
    unsigned long long total_nprod;
    unsigned long long max_nprod;
    unsigned long long max_L;
    unsigned long long bad;   // validation: nonzero if an input is malformed
};

struct BinArgs {
    int64_t m;
    const int32_t *arp, *acol, *brp;
    int32_t warp_cap, block_cap, block_lcap;
    int64_t *nprod;        // optional, per row
    int32_t *bin_rows[kNumBins];   // per bin row lists (bins 1..3), optional
    int64_t *long_nprod;   // per long-bin slot: nprod_i
    int32_t *long_L;       // per long-bin slot: L_i
    int64_t *row_cnt;      // optional: rows of the empty bin get 0
    BinStats *st;
};

cudaError_t launch_bin(const BinArgs &a, cudaStream_t st);
cudaError_t launch_validate(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                            BinStats *st, cudaStream_t stream);
// exclusive scan of in[0..n) into out[0..n] (out[n] = total); tmp needs
// scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_scan(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t st);
// Upper: copy rows of C_bar (at cbar_off[i], row_size[i] long) to C at rp[i]
cudaError_t launch_compact(int64_t m, const int64_t *cbar_off, const int64_t *rp, const int32_t *cbar_col,
                           const void *cbar_val, int32_t *col, void *val, size_t vbytes, cudaStream_t st);

}  // namespace brm
