/*
 * brm.h -- C ABI of libbrm, BRMerge row-wise sparse matrix multiplication
 * C = A * B on CSR matrices for one NVIDIA GB300 (sm_103a).
 *
 * The method is the BRMerge accumulation of Du et al., "Accelerating CPU-Based
 * Sparse General Matrix Multiplication With Binary Row Merging" (IEEE Access
 * 2022): for every output row the scaled rows A_ik * B_k* are gathered into a
 * ping-pong buffer (the multiplying phase) and merged two lists at a time in a
 * binary tree, adjacent pairs (0,1), (2,3), ..., a last odd list copied, equal
 * columns added (the accumulating phase); Section III-A/B, Algorithm 1,
 * Fig. 2.  C is sized either from the intermediate-product upper bound and
 * compacted afterwards (BRMerge-Upper, Section III-D-1) or from a symbolic
 * pass that counts each row's nonzeros first (BRMerge-Precise, Section
 * III-D-2, allocation methods of Section II-B).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices: CSR.  Input row pointers and column indices are int32; columns
 *   must be strictly ascending inside each row (Section II-A: sorted CSR; the
 *   sortedness of every generated list relies on it, Section III-B).  The
 *   output row pointer is int64 because nnz(C) may exceed 2^31.
 * - All array pointers in brm_csr / brm_csr_out are DEVICE pointers on the
 *   current CUDA device unless a call says otherwise.  Inputs are owned by the
 *   caller and only read.
 * - Values: dtype BRM_F64 (double) or BRM_F32 (float); A and B must agree and
 *   C gets the same dtype.  Products are rounded before they are added and no
 *   multiply-add is fused, so a row's value is fixed by the merge tree alone.
 * - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every kernel of a call runs on it.  Calls that must size an output read a
 *   few scalars back to the host and therefore synchronise the stream (each
 *   call's comment says how many times).
 * - Memory: C's arrays and all temporary workspace are obtained through the
 *   brm_allocator callbacks (for example PyTorch's caching allocator); with a
 *   NULL allocator the library uses cudaMallocAsync/cudaFreeAsync on the
 *   stream.  Workspace is released before the call returns.  On error every
 *   allocation made by the call is released and *C is zeroed.
 * - Return value: BRM_OK (0) or one of the negative brm_status codes; nothing
 *   is thrown across the ABI.  brm_last_error() gives a message for the last
 *   failing call on the calling host thread.
 */
#ifndef BRM_H_
#define BRM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BRM_OK = 0,
    BRM_ERR_INVALID = -1,   /* malformed CSR (row_ptr, column range/order) or bad argument */
    BRM_ERR_SHAPE = -2,     /* A.cols != B.rows, or inconsistent sizes */
    BRM_ERR_DTYPE = -3,     /* unknown dtype, or A and B differ */
    BRM_ERR_OOM = -4,       /* the allocator returned NULL */
    BRM_ERR_OVERFLOW = -5,  /* a count exceeds what the index types can hold */
    BRM_ERR_CUDA = -6,      /* a CUDA runtime call failed (message has the CUDA error) */
    BRM_ERR_TIMEOUT = -7    /* a bounded device-side wait ran out */
} brm_status;

typedef enum { BRM_F32 = 0, BRM_F64 = 1 } brm_dtype;

/* Input matrix (rows x cols, nnz entries): row_ptr[rows+1], col_idx[nnz],
 * val[nnz] of the given dtype.  All device pointers, caller-owned, read only.
 * val may be NULL only for brm_spgemm_symbolic. */
typedef struct {
    int64_t rows, cols, nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;
    int32_t dtype;
} brm_csr;

/* Output matrix filled by the library: row_ptr[rows+1] (int64), col_idx[nnz],
 * val[nnz].  The arrays come from the brm_allocator of the call and belong to
 * the caller afterwards (free them with the same allocator). */
typedef struct {
    int64_t rows, cols, nnz;
    int64_t *row_ptr;
    int32_t *col_idx;
    void *val;
    int32_t dtype;
} brm_csr_out;

/* Device-memory callbacks.  alloc(bytes, ctx) returns a device pointer
 * aligned to at least 256 bytes, or NULL when out of memory; release(p, ctx)
 * frees it (p may be NULL).  Memory must be usable by work queued on the
 * call's stream. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*release)(void *p, void *ctx);
    void *ctx;
} brm_allocator;

/* Tuning and checking options; brm_options_default() fills the defaults
 * (start from it: a zeroed struct is valid too, but switches reg_top,
 * reg_perm, reg_num_half and reg_num_direct off and takes the other
 * defaults).
 *   validate       1: check both inputs on the device first (row_ptr starts at
 *                  0, is non-decreasing and ends at nnz; columns in range and
 *                  strictly ascending per row) and return BRM_ERR_INVALID.
 *   compensated    BRM_F32 only, 1: every addition of two equal-column
 *                  elements in the merge tree is TwoSum-compensated (Knuth,
 *                  TAOCP vol. 2, 4.2.2): each element carries a float
 *                  running error, the stored value is sum + error.
 *   reg_max_nprod  rows with 0 < nprod <= this (at most 32 * reg_keys;
 *                  0 = that maximum, negative = none) are merged with their
 *                  keys in registers by 1..32 threads per row, each holding
 *                  reg_keys products and at most reg_keys/4 lists, when B
 *                  has few enough columns to pack a column and a position
 *                  into 32 bits (2^32 / (threads * reg_keys) - 1);
 *   reg_keys       8, 16 or 32 (default 16; other values give 16);
 *   reg_warps      warps per block of the register-bin kernels, 1..8
 *                  (default 4);
 *   reg_top        1 (default): with reg_keys < 32, rows of up to
 *                  64 * reg_keys products (and 16 * reg_keys lists) beyond
 *                  the register bins still take a register kernel, with 32
 *                  threads of 2 * reg_keys keys; 0: they take the shared-
 *                  memory kernels;
 *   reg_perm       1 (default): in BRMerge-Precise (and prepared batches)
 *                  the symbolic pass of the register bins records every
 *                  row's merge order (2 bytes per product, temporary) and the
 *                  numeric pass applies it instead of sorting again; the
 *                  result is the same; 0: the numeric pass sorts by itself;
 *   reg_num_half   1 (default): with reg_perm, the numeric pass runs each
 *                  register row with twice the threads and half the keys of
 *                  its bin where it can (rows of <= 16 threads, >= 16 keys);
 *   reg_num_direct 1 (default): with reg_perm, rows of 32-key register bins
 *                  (the top bin among them) read their products from B at
 *                  output time instead of staging them in shared memory;
 *   symbolic_hash  the symbolic pass counts a row's distinct columns by
 *                  sorting (register bins: the numeric pass's sorting
 *                  network on bare columns; warp and block bins: merge
 *                  rounds on column indices) (0, default), or by hashing
 *                  every column into a shared-memory open-addressing table of
 *                  twice the bin's capacity (1, the paper's symbolic method,
 *                  Section III-D-2); long rows always count their columns in a
 *                  bitmap (a table whose hash is the column itself); the
 *                  counts are identical;
 *   warp_max_nprod other rows with 0 < nprod <= this (and <= as many lists)
 *                  are merged by one warp in shared memory (at most 256).
 *   block_max_nprod rows up to this many products are merged by one thread
 *                  block in shared memory; longer rows use the device-memory
 *                  ping-pong arena (bounded by the kernel's shared memory).
 *   long_bucket    1: rows beyond block_max_nprod are merged by column
 *                  buckets in the numeric pass -- their products are
 *                  scattered to column cells in the arena and every column is
 *                  reduced in the merge tree's order (the same values as the
 *                  merge rounds) -- when every such row has at most 65535
 *                  lists and B at most 2^24 columns; 0 (default): merge rounds
 *                  through the device-memory arena.  (The symbolic pass always
 *                  counts those rows' columns in a shared-memory bitmap when B
 *                  has at most 2^24 columns.)
 *   arena_bytes    budget of the device-memory arena for long rows (0 = the
 *                  library picks 1/4 of free memory, at most 64 GiB, for the
 *                  merge rounds -- persistent blocks, each holding one row's
 *                  buffers at a time -- or 1/8, at most 32 GiB, for the
 *                  column-bucket batches; always at least enough for the
 *                  longest row; BRMerge-Upper in row chunks: 1/8, at most
 *                  32 GiB, per chunk).  A smaller budget runs fewer
 *                  persistent blocks (merge rounds) or more batches (column
 *                  buckets).
 *   long_window    how rows beyond block_max_nprod are merged when
 *                  long_bucket is 0 and B has at most 2^24 columns.  1
 *                  (default): rows of at most 2048 lists and at least 65536
 *                  products are cut into column tiles of at most 2048
 *                  products (the symbolic pass plans them from a column
 *                  bitmap and a per-cell product histogram), each tile's
 *                  products sorted by column in shared memory and summed by
 *                  Algorithm 1's merge rounds on the sorted positions, one
 *                  thread block per tile (the same values as the merge rounds
 *                  in the arena); the other long rows take the arena merge
 *                  rounds in the same pass.  2: every long row of
 *                  at most 65535 lists takes the tiles.  0: every long row
 *                  takes the arena merge rounds.  BRMerge-Upper in row chunks
 *                  always takes the arena merge rounds.
 *   upper_chunk_bytes  BRMerge-Upper: the largest C_bar (nprod * (4 +
 *                  sizeof value) bytes) processed at once; a larger product
 *                  is processed in row chunks of at most this size, each
 *                  compacted on its own, and C assembled from them (peak
 *                  about twice C plus one chunk).  0 = the whole C_bar when it
 *                  can be allocated, else chunks of a quarter of free memory.
 */
typedef struct {
    int32_t validate;
    int32_t compensated;
    int32_t warp_max_nprod;
    int32_t block_max_nprod;
    int32_t reg_max_nprod;
    int32_t reg_keys;
    int32_t reg_warps;
    int32_t symbolic_hash;
    int32_t reg_top;
    int32_t reg_perm;
    int32_t reg_num_half;
    int32_t reg_num_direct;
    int32_t long_bucket;
    size_t arena_bytes;
    size_t upper_chunk_bytes;
    int32_t long_window;
} brm_options;

void brm_options_default(brm_options *opts);

/* Message of the last failing call on this host thread ("" if none). */
const char *brm_last_error(void);

/* Library version string. */
const char *brm_version(void);

/*
 * Symbolic phase of BRMerge-Precise (Section II-B precise allocation, step 3
 * of Section III-D-2): the number of nonzeros of every row of C = A * B,
 * computed from the column indices alone, then its prefix sum.
 *   A, B        inputs (values not read; val may be NULL).
 *   C_row_ptr   device int64[A.rows + 1], caller-allocated; receives the
 *               exclusive prefix sum of the row counts (C_row_ptr[0] = 0).
 *   nnz_C       host int64*, receives nnz(C) = C_row_ptr[A.rows].
 * Synchronises the stream twice (product counts and bins; nnz(C)), plus once
 * more when some rows need the device-memory arena (their sizes are read).
 */
int brm_spgemm_symbolic(const brm_csr *A, const brm_csr *B, int64_t *C_row_ptr, int64_t *nnz_C,
                        const brm_options *opts, const brm_allocator *alloc, void *stream);

/*
 * BRMerge-Precise (Section III-D-2): product counts and binning, the symbolic
 * pass, the prefix sum into C.row_ptr, exact allocation of C, then the
 * numeric BRMerge pass (Algorithm 1) writing every row straight into C.
 * Columns of C are strictly ascending per row; structural zeros (exact
 * cancellations, stored zeros) are kept.
 *   C   host struct; receives the allocated device arrays and sizes.
 * Synchronises the stream three times (bins, nnz(C), a final check that every
 * numeric row filled exactly its symbolic slot), once more with long rows.
 */
int brm_spgemm_precise(const brm_csr *A, const brm_csr *B, brm_csr_out *C,
                       const brm_options *opts, const brm_allocator *alloc, void *stream);

/*
 * BRMerge-Upper (Section III-D-1): product counts, the prefix sum of the
 * upper bounds nprod_i into a temporary C_bar (nprod columns and values),
 * the numeric BRMerge pass writing each row and its size into C_bar, the
 * prefix sum of the row sizes into C.row_ptr, allocation of C and the copy of
 * C_bar into C.  Same result as brm_spgemm_precise, bit for bit.  C_bar needs
 * total_nprod * (4 + sizeof(value)) bytes; when that is more than
 * opts->upper_chunk_bytes (or cannot be allocated) the rows are processed in
 * chunks (see brm_options).
 * Synchronises the stream three times (bins, nnz(C), final check), once more
 * with long rows.
 */
int brm_spgemm_upper(const brm_csr *A, const brm_csr *B, brm_csr_out *C,
                     const brm_options *opts, const brm_allocator *alloc, void *stream);

/*
 * Numeric pass of BRMerge-Precise that allocates no device memory.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or an allocator of their own -- an application that has given
 * all device memory to its own pool, a latency-bound loop that must not take
 * the implicit synchronisation of an allocation, or a plug-in that may only
 * touch the buffers it is handed.  The caller passes C's row pointer (for
 * example from brm_spgemm_symbolic on the same A and B) and C's column and
 * value arrays, sized C_row_ptr[A.rows] entries; every row of C is written
 * into its slot, columns strictly ascending, with the same values as
 * brm_spgemm_precise gives.
 *   A, B        inputs as for brm_spgemm_precise (values required).
 *   C_row_ptr   device int64[A.rows + 1], read only; must be the exact row
 *               pointer of A * B (a row whose length -- zero for a row
 *               without products -- differs from its slot makes the call fail
 *               with BRM_ERR_INVALID, and nothing is written outside the
 *               slots).
 *   C_col_idx   device int32[nnz(C)], written.
 *   C_val       device float/double[nnz(C)] (A's dtype), written.
 *   opts        validate, compensated, warp_max_nprod and block_max_nprod as
 *               elsewhere; arena_bytes is ignored.
 * Limits: A.rows <= 2^20, and every row must fit a shared-memory bin
 * (nprod_i <= block_max_nprod and at most 1024 lists); otherwise the call
 * returns BRM_ERR_OVERFLOW with a message and writes nothing into C.
 * Workspace: a fixed 5 MiB device array inside the library (held on every
 * GPU that loads it until the process exits) instead of allocations.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress)
 * with the device current and keeps it for the life of the process, so make
 * the first call on each device before any stream capture starts, and do not
 * call this entry point again after cudaDeviceReset (the kept address would
 * belong to the destroyed context).  Every call reuses the same array and clears the
 * parts that must start at zero; calls that overlap on the GPU (on different
 * streams or from different host threads) race on it and must be avoided.
 * Synchronises the stream twice (bins; the row-length check), three times
 * with validate.
 */
int brm_spgemm_numeric_noalloc(const brm_csr *A, const brm_csr *B, const int64_t *C_row_ptr, int32_t *C_col_idx,
                               void *C_val, const brm_options *opts, void *stream);

/*
 * Backward pass of C = A * B for a scalar loss with dLoss/dC = G given on C's
 * pattern (the differentiable form; the paper's method is the forward pass,
 * Eq. 2):
 *   dA_ik = sum_{j in B_k*} G_ij * B_kj           for every stored (i, k) of A,
 *   dB_kj = sum_{i : k in A_i*} A_ik * G_ij      for every stored (k, j) of B,
 * i.e. (G * B^T) masked to A's pattern and (A^T * G) masked to B's pattern.
 *   A, B         the forward inputs (values required, same dtype).
 *   C_row_ptr,   device int64[A.rows + 1] and int32[nnz(C)]: the pattern of C
 *   C_col_idx    as returned by brm_spgemm_precise / brm_spgemm_upper (every
 *                column of every B_k*, k in A_i*, must be present in row i).
 *   dC           device values of G on C's pattern (A's dtype).
 *   dA_val       device, A.nnz values, written (NULL: not computed).
 *   dB_val       device, B.nnz values, overwritten (NULL: not computed).
 * Both are deterministic sums in a fixed order, each product rounded before
 * it is added: dA_ik over B_k* in column order (one GPU thread per entry of
 * A), dB_kj over the rows i in increasing order (one thread per entry of B,
 * after A's entries are bucketed by column and every bucket is sorted).
 * Returns BRM_ERR_INVALID if C's pattern misses a column.  Synchronises the
 * stream twice when dB is computed (the product count sizes its workspace),
 * else once.  opts is unused (may be NULL); alloc provides a 4-byte flag
 * and, when dB is computed, about 16 * A.cols + 32 * A.nnz bytes plus one
 * value per intermediate product (every product's G_ij, kept by the dA pass
 * for the dB sums) of workspace.
 */
int brm_spgemm_backward(const brm_csr *A, const brm_csr *B, const int64_t *C_row_ptr, const int32_t *C_col_idx,
                        const void *dC, void *dA_val, void *dB_val, const brm_options *opts,
                        const brm_allocator *alloc, void *stream);

/*
 * Batched products (the batching pattern added to the paper's method): count
 * independent products C_p = A_p * B_p of uneven sizes processed as one
 * problem -- one binning over all their rows, one launch per row bin for the
 * symbolic pass and one for the numeric pass (BRMerge-Precise, Section
 * III-D-2), whatever the number of products.  The result is the vertical
 * stack of the C_p: one CSR whose rows row_offset[p] .. row_offset[p+1]-1 are
 * the rows of C_p, with C_p's own column indices (C.cols = the largest
 * B_p.cols).  All products must have the same dtype.
 *   A, B        host arrays of count input descriptors (device arrays inside).
 *   C           receives the stacked result (arrays from alloc).
 *   row_offset  host int64[count + 1] or NULL: the first row of every C_p.
 * Synchronises the stream as brm_spgemm_precise does, plus once to set up
 * the product table.
 */
int brm_spgemm_batched(int32_t count, const brm_csr *A, const brm_csr *B, brm_csr_out *C, int64_t *row_offset,
                       const brm_options *opts, const brm_allocator *alloc, void *stream);

/*
 * Prepared batches: brm_batch_create runs everything of brm_spgemm_batched
 * up to the numeric pass (product table, bins, symbolic pass, allocation of
 * C, the long-row arena) and keeps it; the numeric pass can then be run again
 * and again on new VALUES of the same input arrays (same patterns, same
 * pointers) -- the structure reuse of repeated products -- without any host
 * synchronisation or allocation:
 *   brm_batch_numeric       launches the numeric pass on stream.
 *   brm_batch_graph_launch  the same, as a CUDA graph: the first call captures
 *                           the launches (on a private stream) and
 *                           instantiates the graph, every call launches it
 *                           on stream.  The batch must not be modified while
 *                           a graph launch is in flight.
 *   brm_batch_check         synchronises stream and reports BRM_ERR_INVALID
 *                           if a numeric row did not fill its symbolic slot.
 *   brm_batch_result        the stacked C (arrays still owned by the batch).
 *   brm_batch_take          the same, and the caller becomes the owner (free
 *                           with brm_csr_out_free and the batch's allocator).
 *   brm_batch_destroy       frees what the batch still owns.
 * The allocator struct is copied; its callbacks and context must stay valid
 * until brm_batch_destroy.  A batch is used by one host thread at a time.
 */
typedef struct brm_batch brm_batch;
int brm_batch_create(int32_t count, const brm_csr *A, const brm_csr *B, const brm_options *opts,
                     const brm_allocator *alloc, void *stream, brm_batch **out);
int brm_batch_numeric(brm_batch *batch, void *stream);
int brm_batch_graph_launch(brm_batch *batch, void *stream);
int brm_batch_check(brm_batch *batch, void *stream);
int brm_batch_result(const brm_batch *batch, brm_csr_out *C, int64_t *row_offset);
int brm_batch_take(brm_batch *batch, brm_csr_out *C, int64_t *row_offset);
void brm_batch_destroy(brm_batch *batch);

/*
 * Autotuner of the row bins: times brm_batch_create + brm_batch_numeric +
 * brm_batch_check (wall clock; each candidate runs once to warm up and twice
 * timed, the minimum counts) on the given products, first for every shape of
 * the register bins (reg_keys 8, 16, 32 x reg_warps 2, 4, 8, each with its
 * full register range), then for the bin thresholds one at a time from the
 * best so far: reg_max_nprod at 1/2 and 1/4 of that range, reg_top switched,
 * warp_max_nprod 128 and 64, block_max_nprod 2048 and 1024 (the other fields
 * are taken from base).  Writes the fastest options to best (and its time in
 * milliseconds to best_ms, if not NULL).  Synchronises the stream many times.
 */
int brm_autotune(int32_t count, const brm_csr *A, const brm_csr *B, const brm_options *base, brm_options *best,
                 double *best_ms, const brm_allocator *alloc, void *stream);

/* Frees the arrays of a brm_csr_out with the given allocator and zeroes it. */
void brm_csr_out_free(brm_csr_out *C, const brm_allocator *alloc, void *stream);

/*
 * Per-row statistics used by the binning (step 1 of both libraries, Section
 * III-D; the buffer sizing that opens Algorithm 1): nprod_i = sum over k in A_i* of |B_k*|.
 *   row_nprod   device int64[A.rows], caller-allocated, or NULL (only the
 *               totals below are wanted).
 *   total_nprod, max_row_nprod, max_row_nnz_A: host int64*, may be NULL.
 * Synchronises the stream once.
 */
int brm_row_nprod(const brm_csr *A, const brm_csr *B, int64_t *row_nprod, int64_t *total_nprod,
                  int64_t *max_row_nprod, int64_t *max_row_nnz_A, void *stream);

/*
 * The static split of the rows (Section III-D: the rows are cut into
 * contiguous groups of about equal intermediate products, one per worker),
 * used to shard one product over several GPUs: every GPU holds B, computes
 * the rows bounds[p] .. bounds[p+1]-1 of C with its own call on that slice of
 * A's rows, and one exchange of the parts' nnz places its rows in the global
 * row pointer.
 *   parts   number of parts (>= 1).
 *   bounds  host int64[parts + 1], written: bounds[0] = 0, bounds[parts] =
 *           A.rows, non-decreasing; part p starts at the first row whose
 *           products before it reach floor(p * total_nprod / parts).
 * Workspace (nprod per row, its prefix sum) comes from alloc.  Synchronises
 * the stream once.
 */
int brm_row_split(const brm_csr *A, const brm_csr *B, int32_t parts, int64_t *bounds, const brm_allocator *alloc,
                  void *stream);

/*
 * Tracing (the measurement side of the paper's evaluation, Section IV-A: the
 * time of each part of the computation).  With tracing on, every later call
 * records CUDA events on its stream around each kernel phase; the elapsed
 * device times are added per phase when the call returns.  Phases, in order:
 * validate, bin, symbolic_reg, symbolic_warp, symbolic_block, symbolic_long,
 * scan, numeric_reg, numeric_warp, numeric_block, numeric_long (the long
 * rows' merge rounds), compact, backward, symbolic_tile and numeric_tile (the
 * column tiles of the long rows, option long_window).  Not thread-safe across
 * concurrent calls from several host threads.
 *   brm_trace_enable      on != 0 enables; returns the previous setting.
 *   brm_trace_reset       zeroes the accumulated times and launch counts.
 *   brm_trace_read        copies up to n per-phase totals (milliseconds of
 *                         device time, kernel launches) into host arrays
 *                         (either may be NULL); returns the number of phases.
 *   brm_trace_phase_name  name of phase i ("" if out of range).
 *   brm_kernel_launches   kernel launches made by the library since loading
 *                         (counted whether tracing is on or not).
 */
int brm_trace_enable(int on);
void brm_trace_reset(void);
int brm_trace_read(double *ms, int64_t *launches, int n);
const char *brm_trace_phase_name(int i);
int64_t brm_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* BRM_H_ */
