// Internal interfaces between the translation units of libbrm.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace brm {

struct RowJob;
struct ProdDesc;

// Row bins (by intermediate products nprod_i and list count L_i of a row):
//   empty           nprod_i = 0 (the row of C is empty);
//   register r=0..5 TPR = 2^r threads per row holding E keys each (E = 8, 16
//                   or 32): nprod_i <= E * TPR and L_i <= E/4 * TPR, keys sorted
//                   in registers (brm_reg_rows.cuh);
//   warp            one warp per row, shared-memory ping-pong (brm_rows.cuh);
//   block           one thread block per row, shared-memory ping-pong;
//   long            one thread block per row, device-memory ping-pong arena.
//   register top    (only when E < 32) 32 threads holding 2E keys each, for
//                   rows just above the largest register bin;
enum {
    kBinEmpty = 0, kBinReg0 = 1, kNumRegBins = 7, kBinRegTop = kBinReg0 + 6, kBinWarp = kBinReg0 + kNumRegBins,
    kBinBlock, kBinLong, kNumBins
};
__host__ __device__ constexpr int reg_bin_tpr(int bin) { return bin == kBinRegTop ? 32 : 1 << (bin - kBinReg0); }

// Register bins: keys per thread (E), lists per key, threads per row.
constexpr int kRegKeysDefault = 16;
constexpr int kRegKeysPerList = 4;    // a row may have up to E/4 lists per thread
constexpr int kRegMaxTpr = 32;
constexpr int kRegMaxNprod = 32 * kRegMaxTpr;   // 1024 (E = 32; 512 with E = 16)
constexpr int kRegWarpsDefault = 4;   // warps per block

// Most columns B may have for a register bin of `tpr` threads x `keys` keys:
// a 32-bit key holds the column above the product's position in the row
// (log2(tpr * keys) bits) and must stay below the all-ones padding key.
__host__ __device__ constexpr int64_t reg_col_limit(int tpr, int keys) {
    int b = 0;
    for (int x = tpr * keys; x > 1; x >>= 1) ++b;
    return (int64_t(1) << (32 - b)) - 1;
}

// Capacities of the shared-memory bins.
constexpr int kWarpCap = 256;     // warp bin: nprod_i <= 256 and L_i <= 256
constexpr int kBlockCap = 4096;   // block bin: nprod_i <= 4096 ...
constexpr int kBlockLCap = 1024;  // ... and L_i <= 1024

// Limits of the column-bucket long-row kernels (brm_long_rows.cuh): lists of
// a row (a 16-bit list index that never forms the all-ones padding key) and
// columns of B (at most 4096 cells of at most 4096 columns each).
constexpr int kLbMaxL = 65535;
constexpr int64_t kLbMaxCols = (int64_t)1 << 24;
// The numeric bucket kernels' work list (hot cells and giant columns, each of
// more than kLbUnit products: at most n / (kLbUnit + 1) + 1 records for a row
// of n products, kLbWorkBytes each) and the value slots of a giant column
// (kLbSlots per block of the work-list kernel, kLbHotPerSm blocks per SM).
constexpr int kLbUnit = 256;
constexpr size_t kLbWorkBytes = 32;
constexpr int kLbSlots = 65536;
constexpr int kLbHotPerSm = 2;
__host__ __device__ constexpr int64_t lb_work_cap(int64_t n) { return n / (kLbUnit + 1) + 1; }

// Long rows by column tiles (brm_long_tiles.cuh): a tile holds at most kTileP
// products (one thread block of kTileThreads sorts them) unless it is a single
// cell of at most kTileCellMax columns (a "hot" tile, taken in chunks); the
// plan cuts pieces every kTilePiece products and packs them into tiles; at most
// kTileCells cells per bitmap window of kTileBitmapCols columns; rows of at most
// kTileMaxL lists and at least kTileMinNprod products (others keep the merge
// rounds); spans of at least
// max(kTileSpanMin, kTileSpanPerList * L) products.
constexpr int kTileP = 2048;
constexpr int kTilePBits = 11;
constexpr int kTileThreads = 256;
constexpr int kTileMaxL = 65535;     // 16-bit list index
constexpr int kTileSmemL = 2048;     // lists whose cursors fit shared memory (more: device memory)
// long rows of fewer products keep the merge rounds (measured faster there)
constexpr int64_t kTileMinNprod = 65536;
constexpr int kTilePiece = 256;
constexpr int64_t kTileBitmapCols = (int64_t)1 << 20;
constexpr int kTileCells = 8192;
constexpr int kTileCellMax = (int)(kTileBitmapCols / kTileCells);
constexpr int64_t kTileSpanMin = 32768;
constexpr int kTileSpanPerList = 16;
static_assert((1 << kTilePBits) == kTileP, "a tile position fits the key's low bits");
static_assert(kTileSmemL <= kTileP, "a tile that fits one sort has at most kTileP segments");
static_assert(kTileCellMax == 128, "cells are at most 128 columns wide");
static_assert((((kTileBitmapCols - 1) << kTilePBits) | (kTileP - 1)) <= 0xffffffffLL, "key = column offset and position");

// One tile of a long row: first column, products, and the number of the
// row's distinct columns before it (its output offset inside the row).
struct TileRec {
    int32_t c0;
    int32_t np;
    int64_t off;
};
static_assert(sizeof(TileRec) == 16, "tile record size");

// Tiles a row of n products can produce over B's columns (ncols): every
// bitmap window holds at most 3 n_w / kTilePiece + 1 pieces (and tiles), and
// never more than its cells.
__host__ __device__ constexpr int64_t tile_cap(int64_t n, int64_t ncols) {
    const int64_t nbw = ncols > 0 ? (ncols + kTileBitmapCols - 1) / kTileBitmapCols : 1;
    const int64_t a = 3 * ((n + kTilePiece - 1) / kTilePiece) + nbw;
    const int64_t b = nbw * kTileCells;
    return a < b ? a : b;
}

// Spans a row of n products can produce: at most 2 n / kTileSpanMin + 2.
__host__ __device__ constexpr int64_t tile_span_cap(int64_t n) { return 2 * (n / kTileSpanMin) + 2; }

// Kernel phases recorded by the tracer (brm_trace_*).
enum Phase {
    kPhValidate = 0, kPhBin, kPhSymReg, kPhSymWarp, kPhSymBlock, kPhSymLong, kPhScan,
    kPhNumReg, kPhNumWarp, kPhNumBlock, kPhNumLong, kPhCompact, kPhBackward, kPhSymTile, kPhNumTile, kNumPhases
};

// Kernel launches made by the library so far (all threads).
extern std::atomic<long long> g_launches;

// value kinds of a pass
enum VKind { kIdx = 0, kF64 = 1, kF32 = 2, kF32C = 3 };

cudaError_t launch_rows(VKind v, int bin, const RowJob &j, cudaStream_t st);
size_t long_row_bytes_for(VKind v, int64_t nprod, int64_t L, bool bucket);
// blocks of the long-row tile kernel of a value kind (0 for kIdx)
int long_tile_grid(VKind v);

// Statistics written by the binning kernels.
struct BinStats {
    unsigned long long count[kNumBins];
    unsigned long long total_nprod;
    unsigned long long max_nprod;
    unsigned long long max_L;
    unsigned long long bad;   // validation: nonzero if an input is malformed
    unsigned long long cursor[kNumBins];   // fill level of each bin during the scatter
    unsigned long long reg_nprod;          // products of the rows in register bins
};

// Binning in two passes: k_bin classifies every row (bin_of, counts); after
// the host has read the counts, k_bin_scatter lists the rows of every bin b
// contiguously at rows[base[b] ...] (order inside a bin is unspecified).
struct BinArgs {
    int64_t m;
    const int32_t *arp, *acol, *brp;
    const ProdDesc *prods;     // batched products (null: one product, arp/acol/brp)
    const int32_t *prod_of;    // batched: product of every stacked row
    int32_t reg_max_tpr;   // largest register-bin TPR allowed (0: none)
    int32_t reg_keys;      // keys per thread of the register bins (8, 16 or 32)
    int32_t reg_top;       // 1: the top register bin (32 threads x 2 reg_keys) is allowed
    int32_t warp_cap, block_cap, block_lcap;
    int64_t *nprod;        // optional, per row
    uint8_t *bin_of;       // optional, per row: its bin
    int64_t *row_cnt;      // optional: rows of the empty bin get 0
    const int64_t *out_rp; // optional: C's row pointer; an empty row with a slot sets *out_err
    unsigned int *out_err;
    BinStats *st;
    // scatter pass
    int64_t base[kNumBins];
    int32_t *rows;         // m entries
    int64_t *long_nprod;   // optional, per long-bin slot: nprod_i (needs nprod)
    int32_t *long_L;       // optional, per long-bin slot: L_i
};

cudaError_t launch_bin(const BinArgs &a, cudaStream_t st);
// batched products: prod_of[row0[p] .. row0[p] + rows[p]) = p
cudaError_t launch_fill_prod_of(const ProdDesc *prods, const int64_t *rows_of, int32_t count, int32_t *prod_of,
                                cudaStream_t st);
cudaError_t launch_bin_scatter(const BinArgs &a, cudaStream_t st);
// out[i] = nprod[i] rounded up to a multiple of 16 if row i is in a register
// bin, else 0
cudaError_t launch_reg_nprod(int64_t m, const uint8_t *bin_of, const int64_t *nprod, int64_t *out, cudaStream_t st);
cudaError_t launch_validate(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rp, const int32_t *col,
                            BinStats *st, cudaStream_t stream);
// exclusive scan of in[0..n) into out[0..n] (out[n] = total); tmp needs
// scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_scan(const int64_t *in, int64_t *out, int64_t n, void *tmp, cudaStream_t st);
// bounds[0 .. parts] of the static nprod-balanced row split from the
// exclusive product prefix excl[0 .. m]
cudaError_t launch_row_split(const int64_t *excl, int64_t m, int32_t parts, int64_t *bounds, cudaStream_t st);
// Upper: copy rows of C_bar (at cbar_off[i], row_size[i] long) to C at rp[i]
cudaError_t launch_compact(int64_t m, const int64_t *cbar_off, const int64_t *rp, const int32_t *cbar_col,
                           const void *cbar_val, int32_t *col, void *val, size_t vbytes, cudaStream_t st);

// Backward pass of C = A * B (brm_backward.cu).
struct BackwardArgs {
    int64_t m, nnz_a;
    int64_t ka, kb, nnz_b;    // A's columns (= B's rows), B's rows, B's entries
    const int32_t *arp, *acol; const void *aval;
    const int32_t *brp, *bcol; const void *bval;
    const int64_t *crp; const int32_t *ccol; const void *dC;
    void *dA, *dB;            // either may be null
    unsigned int *err;        // set when C's pattern lacks a column of some B_k*
    // dB workspace: bucket sizes / cursors (ka), bucket starts (ka + 1), the
    // scans' temporaries, entry indices and rows (nnz_a), every entry's first
    // product (nnz_a + 1) and every product's G_ij (nprod values)
    int64_t *ws_cnt, *ws_colptr;
    void *ws_scan, *ws_scan2;
    int32_t *ws_ent, *ws_row;
    int64_t *ws_plen, *ws_poff;
    void *ws_gp;
};
cudaError_t launch_backward(const BackwardArgs &a, bool f64, cudaStream_t st);

}  // namespace brm
