// Host side of libbrm: argument checks, the BRMerge-Upper / BRMerge-Precise
// pipelines (Section III-D), workspace through the caller's allocator, and the
// extern "C" entry points declared in include/brm.h.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "brm.h"
#include "brm_engine.cuh"
#include "brm_internal.h"

namespace brm {
namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// ---------------------------------------------------------------------------
// Tracer: when enabled, CUDA events are recorded on the call's stream around
// every kernel phase; their elapsed times are added up per phase once the
// call has synchronised.  Meant for one host thread at a time.
// ---------------------------------------------------------------------------
struct Trace {
    bool on = false;
    double ms[kNumPhases] = {};
    long long launches[kNumPhases] = {};
    std::vector<cudaEvent_t> pool;
    struct Rec { int ph; long long nl; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::mutex mu;

    cudaEvent_t event() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return e;
    }
    void flush() {
        std::lock_guard<std::mutex> lk(mu);
        for (const Rec &r : pending) {
            float t = 0.0f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.ph] += t;
                launches[r.ph] += r.nl;
            } else {
                cudaGetLastError();
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
};
Trace g_trace;

struct PhaseScope {
    int ph;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    long long n0;
    PhaseScope(int phase, cudaStream_t s) : ph(phase), st(s), n0(g_launches.load()) {
        if (g_trace.on && phase >= 0) {
            std::lock_guard<std::mutex> lk(g_trace.mu);
            a = g_trace.event();
            if (a) cudaEventRecord(a, st);
        }
    }
    ~PhaseScope() {
        if (!a) return;
        std::lock_guard<std::mutex> lk(g_trace.mu);
        cudaEvent_t b = g_trace.event();
        if (!b) { g_trace.pool.push_back(a); return; }
        cudaEventRecord(b, st);
        g_trace.pending.push_back({ph, g_launches.load() - n0, a, b});
    }
};

#define BRM_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(BRM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Device memory of one call.  Everything still owned at destruction (error
// paths, workspace) is released; arrays handed to the caller are detached.
//
// Workspace of a known size can be reserved up front as one block (reserve):
// later get() calls are carved from it, so a call makes one allocator call
// for its workspace instead of one per array.  Arrays handed to the caller
// always come from get_direct().
struct Mem {
    const brm_allocator *al;
    cudaStream_t st;
    std::vector<void *> owned;
    char *slab = nullptr;
    size_t slab_size = 0, slab_used = 0;

    Mem(const brm_allocator *a, cudaStream_t s) : al(a), st(s) {}
    ~Mem() { release_all(); }

    void *get_direct(size_t bytes) {
        if (bytes == 0) bytes = 256;
        void *p = nullptr;
        if (al && al->alloc) {
            p = al->alloc(bytes, al->ctx);
        } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) owned.push_back(p);
        return p;
    }
    void reserve(size_t bytes) {
        if (slab) return;
        slab = static_cast<char *>(get_direct(bytes));
        slab_size = slab ? bytes : 0;
        slab_used = 0;
    }
    bool in_slab(const void *p) const {
        return slab && p >= slab && static_cast<const char *>(p) < slab + slab_size;
    }
    void *get(size_t bytes) {
        const size_t b = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
        if (slab && slab_used + b <= slab_size) {
            void *p = slab + slab_used;
            slab_used += b;
            return p;
        }
        return get_direct(bytes);
    }
    void free_one(void *p) {
        if (!p || in_slab(p)) return;   // carved workspace goes with the block
        auto it = std::find(owned.begin(), owned.end(), p);
        if (it != owned.end()) owned.erase(it);
        release(p);
    }
    void release(void *p) {
        if (al && al->release) al->release(p, al->ctx);
        else if (!al || !al->alloc) cudaFreeAsync(p, st);
    }
    void detach(void *p) {
        auto it = std::find(owned.begin(), owned.end(), p);
        if (it != owned.end()) owned.erase(it);
    }
    void release_all() {
        for (void *p : owned) release(p);
        owned.clear();
    }
};

template <class T>
int get(Mem &mem, T *&p, size_t count, const char *what) {
    p = static_cast<T *>(mem.get(count * sizeof(T)));
    if (!p) return fail(BRM_ERR_OOM, "allocation of %zu bytes for %s failed", count * sizeof(T), what);
    return BRM_OK;
}

// An array that is handed to the caller (never carved from the workspace).
template <class T>
int get_own(Mem &mem, T *&p, size_t count, const char *what) {
    p = static_cast<T *>(mem.get_direct(count * sizeof(T)));
    if (!p) return fail(BRM_ERR_OOM, "allocation of %zu bytes for %s failed", count * sizeof(T), what);
    return BRM_OK;
}

// Workspace bytes that a Precise / symbolic / Upper call over m rows needs
// before its first synchronisation (bins, counts, scans, offsets).
size_t row_workspace_bytes(int64_t m);

int check_csr(const brm_csr *M, const char *name, bool need_val) {
    if (!M) return fail(BRM_ERR_INVALID, "%s is NULL", name);
    if (M->rows < 0 || M->cols < 0 || M->nnz < 0) return fail(BRM_ERR_INVALID, "%s has a negative size", name);
    if (M->rows >= INT32_MAX || M->cols >= INT32_MAX || M->nnz > INT32_MAX)
        return fail(BRM_ERR_OVERFLOW, "%s exceeds the int32 index range", name);
    if (!M->row_ptr) return fail(BRM_ERR_INVALID, "%s.row_ptr is NULL", name);
    if (M->nnz > 0 && !M->col_idx) return fail(BRM_ERR_INVALID, "%s.col_idx is NULL", name);
    if (need_val && M->nnz > 0 && !M->val) return fail(BRM_ERR_INVALID, "%s.val is NULL", name);
    if (M->dtype != BRM_F32 && M->dtype != BRM_F64) return fail(BRM_ERR_DTYPE, "%s has unknown dtype %d", name, M->dtype);
    return BRM_OK;
}

int check_pair(const brm_csr *A, const brm_csr *B, bool need_val) {
    int rc = check_csr(A, "A", need_val);
    if (rc) return rc;
    if ((rc = check_csr(B, "B", need_val))) return rc;
    if (A->cols != B->rows)
        return fail(BRM_ERR_SHAPE, "A is %lld x %lld but B is %lld x %lld", (long long)A->rows, (long long)A->cols,
                    (long long)B->rows, (long long)B->cols);
    if (need_val && A->dtype != B->dtype) return fail(BRM_ERR_DTYPE, "A and B have different dtypes");
    return BRM_OK;
}

// The inputs of one pass: one product A * B, or a batch of products whose
// rows are stacked (row r of the stack is row r - row0[p] of product p).
struct Src {
    int64_t m = 0;           // rows of C (stacked rows for a batch)
    int64_t bcols = 0;       // columns of B (the largest over a batch)
    int32_t dtype = BRM_F64;
    const int32_t *arp = nullptr, *acol = nullptr, *brp = nullptr, *bcol = nullptr;
    const void *aval = nullptr, *bval = nullptr;
    const ProdDesc *prods = nullptr;   // batch: device table of the products
    const int32_t *prod_of = nullptr;  // batch: product of every stacked row
};

Src src_of(const brm_csr *A, const brm_csr *B) {
    Src s;
    s.m = A->rows;
    s.bcols = B->cols;
    s.dtype = A->dtype;
    s.arp = A->row_ptr;
    s.acol = A->col_idx;
    s.aval = A->val;
    s.brp = B->row_ptr;
    s.bcol = B->col_idx;
    s.bval = B->val;
    return s;
}

brm_options resolve(const brm_options *o) {
    brm_options r;
    brm_options_default(&r);
    if (o) r = *o;
    if (r.warp_max_nprod <= 0 || r.warp_max_nprod > kWarpCap) r.warp_max_nprod = kWarpCap;
    if (r.block_max_nprod <= 0 || r.block_max_nprod > kBlockCap) r.block_max_nprod = kBlockCap;
    if (r.block_max_nprod < r.warp_max_nprod) r.block_max_nprod = r.warp_max_nprod;
    if (r.reg_keys != 8 && r.reg_keys != 16 && r.reg_keys != 32) r.reg_keys = kRegKeysDefault;
    if (r.reg_warps < 1 || r.reg_warps > 8) r.reg_warps = kRegWarpsDefault;
    if (r.reg_max_nprod == 0 || r.reg_max_nprod > r.reg_keys * kRegMaxTpr) r.reg_max_nprod = r.reg_keys * kRegMaxTpr;
    r.reg_top = r.reg_top != 0 ? 1 : 0;
    r.reg_perm = r.reg_perm != 0 ? 1 : 0;
    r.reg_num_half = r.reg_num_half != 0 ? 1 : 0;
    r.reg_num_direct = r.reg_num_direct != 0 ? 1 : 0;
    r.long_bucket = r.long_bucket != 0 ? 1 : 0;
    r.long_window = r.long_window < 0 || r.long_window > 2 ? 1 : r.long_window;
    if (r.reg_max_nprod < 0) r.reg_max_nprod = 0;
    return r;
}

// Largest threads-per-row of a register bin usable for this product: its
// capacity within reg_max_nprod and B's column count packable into its keys.
int reg_max_tpr(const brm_options &o, int64_t bcols) {
    int best = 0;
    for (int tpr = 1; tpr <= kRegMaxTpr; tpr <<= 1)
        if (o.reg_keys * tpr <= o.reg_max_nprod && bcols <= reg_col_limit(tpr, o.reg_keys)) best = tpr;
    return best;
}

// The top register bin (32 threads x 2 reg_keys keys): only below 32 keys, when
// the other register bins are all usable and reg_max_nprod was not lowered.
int reg_top_ok(const brm_options &o, int64_t bcols) {
    return o.reg_keys < 32 && reg_max_tpr(o, bcols) == kRegMaxTpr && o.reg_max_nprod >= 32 * o.reg_keys &&
           o.reg_top && bcols <= reg_col_limit(32, 2 * o.reg_keys);
}

size_t row_workspace_bytes(int64_t m) {
    const size_t m1 = (size_t)std::max<int64_t>(m, 1) + 1;
    // statistics and flags; per row: bin (1), row list (4), nprod (8), counts
    // (8), order sizes (8), order offsets (8); two scan workspaces
    return 8 * 256 + m1 * (1 + 4 + 8 + 8 + 8 + 8) + 2 * scan_tmp_bytes(m) + 8 * 256;
}

// Result of the binning step.
struct Plan {
    BinStats stats{};
    uint8_t *bin_of = nullptr;          // device: the bin of every row
    int64_t *nprod = nullptr;           // device: nprod_i of every row
    int32_t *rows = nullptr;            // device: the rows of every bin, bin after bin
    int64_t base[kNumBins] = {};        // where bin b starts in rows
    int64_t *long_nprod = nullptr;      // device, per long slot (binning order)
    int32_t *long_L = nullptr;
    int32_t *long_rows_s = nullptr;     // device, long rows sorted by nprod (descending)
    int64_t *long_nprod_s = nullptr;
    std::vector<int32_t> long_rows_h;   // host copies, same order
    std::vector<int64_t> long_nprod_h;
    std::vector<int32_t> long_L_h;
    // with column tiles: the long slots [0, long_split) keep the merge rounds
    // (rows of more than kTileMaxL lists), the others take the tiles
    int64_t long_split = 0;
};

// Whether the long rows of a product take the column tiles (brm_long_tiles.cuh):
// the option is on, the bucket option off, and B has at most 2^24 columns.
bool tiles_apply(const brm_options &o, int64_t bcols) {
    return o.long_window && !o.long_bucket && bcols <= kLbMaxCols;
}

int validate_inputs(Mem &mem, const brm_csr *A, const brm_csr *B) {
    BinStats *st;
    int rc = get(mem, st, 1, "validation flag");
    if (rc) return rc;
    BRM_CUDA(cudaMemsetAsync(st, 0, sizeof(BinStats), mem.st));
    {
        PhaseScope ps(kPhValidate, mem.st);
        BRM_CUDA(launch_validate(A->rows, A->cols, A->nnz, A->row_ptr, A->col_idx, st, mem.st));
        BRM_CUDA(launch_validate(B->rows, B->cols, B->nnz, B->row_ptr, B->col_idx, st, mem.st));
    }
    BinStats h{};
    BRM_CUDA(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    mem.free_one(st);
    if (h.bad) return fail(BRM_ERR_INVALID, "malformed CSR input (row_ptr or column order/range)");
    return BRM_OK;
}

// Step 1 (+ the GPU form of step 2): product counts, bins, long-row order.
int make_plan(Mem &mem, const Src &src, const brm_options &o, Plan &pl, int64_t *nprod, int64_t *row_cnt) {
    const int64_t m = src.m;
    const size_t m1 = (size_t)std::max<int64_t>(m, 1);
    BinStats *st;
    int rc = get(mem, st, 1, "bin statistics");
    if (rc) return rc;
    BRM_CUDA(cudaMemsetAsync(st, 0, sizeof(BinStats), mem.st));
    uint8_t *bin_of;
    if ((rc = get(mem, bin_of, m1, "row bins"))) return rc;
    if ((rc = get(mem, pl.rows, m1, "bin row lists"))) return rc;
    if (!nprod && (rc = get(mem, nprod, m1, "row nprod"))) return rc;
    pl.bin_of = bin_of;
    pl.nprod = nprod;
    BinArgs a{};
    a.m = m;
    a.arp = src.arp;
    a.acol = src.acol;
    a.brp = src.brp;
    a.prods = src.prods;
    a.prod_of = src.prod_of;
    a.reg_max_tpr = reg_max_tpr(o, src.bcols);
    a.reg_keys = o.reg_keys;
    a.reg_top = reg_top_ok(o, src.bcols);
    a.warp_cap = o.warp_max_nprod;
    a.block_cap = o.block_max_nprod;
    a.block_lcap = kBlockLCap;
    a.nprod = nprod;
    a.bin_of = bin_of;
    a.row_cnt = row_cnt;
    a.st = st;
    a.rows = pl.rows;
    {
        PhaseScope ps(kPhBin, mem.st);
        BRM_CUDA(launch_bin(a, mem.st));
    }
    BRM_CUDA(cudaMemcpyAsync(&pl.stats, st, sizeof(BinStats), cudaMemcpyDeviceToHost, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    if (pl.stats.max_nprod >= (unsigned long long)INT32_MAX)
        return fail(BRM_ERR_OVERFLOW, "a row has %llu intermediate products (limit 2^31-1)", pl.stats.max_nprod);
    int64_t off = 0;
    for (int b = 0; b < kNumBins; ++b) {
        pl.base[b] = a.base[b] = off;
        if (b != kBinEmpty) off += (int64_t)pl.stats.count[b];
    }
    const int64_t nl = (int64_t)pl.stats.count[kBinLong];
    if (nl > 0) {
        if ((rc = get(mem, pl.long_nprod, nl, "long-row sizes"))) return rc;
        if ((rc = get(mem, pl.long_L, nl, "long-row list counts"))) return rc;
        a.long_nprod = pl.long_nprod;
        a.long_L = pl.long_L;
    }
    {
        PhaseScope ps(kPhBin, mem.st);
        BRM_CUDA(launch_bin_scatter(a, mem.st));
    }
    mem.free_one(st);   // stream-ordered: released after the scatter
    if (nl > 0) {
        std::vector<int32_t> rows(nl), Ls(nl);
        std::vector<int64_t> np(nl);
        BRM_CUDA(cudaMemcpyAsync(rows.data(), pl.rows + pl.base[kBinLong], nl * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, mem.st));
        BRM_CUDA(cudaMemcpyAsync(np.data(), pl.long_nprod, nl * sizeof(int64_t), cudaMemcpyDeviceToHost, mem.st));
        BRM_CUDA(cudaMemcpyAsync(Ls.data(), pl.long_L, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, mem.st));
        BRM_CUDA(cudaStreamSynchronize(mem.st));
        // largest rows first, so that the longest merges start earliest; with
        // column tiles, the rows that keep the merge rounds before the others:
        // long_window 1, rows of more than kTileSmemL lists or fewer than
        // kTileMinNprod products (measured faster there); long_window 2, rows
        // of more than kTileMaxL lists
        const bool tiles = tiles_apply(o, src.bcols);
        const int64_t tmin = o.long_window == 1 ? kTileMinNprod : 0;
        const int64_t tmaxl = o.long_window == 1 ? kTileSmemL : kTileMaxL;
        auto rounds = [&](int64_t x) { return !tiles || Ls[x] > tmaxl || np[x] < tmin; };
        std::vector<int64_t> idx(nl);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
            const bool rx = rounds(x), ry = rounds(y);
            if (rx != ry) return rx;
            return np[x] > np[y];
        });
        pl.long_split = 0;
        for (int64_t s = 0; s < nl; ++s) pl.long_split += rounds(s) ? 1 : 0;
        pl.long_rows_h.resize(nl);
        pl.long_nprod_h.resize(nl);
        pl.long_L_h.resize(nl);
        for (int64_t s = 0; s < nl; ++s) {
            pl.long_rows_h[s] = rows[idx[s]];
            pl.long_nprod_h[s] = np[idx[s]];
            pl.long_L_h[s] = Ls[idx[s]];
        }
        if ((rc = get(mem, pl.long_rows_s, nl, "long rows"))) return rc;
        if ((rc = get(mem, pl.long_nprod_s, nl, "long-row sizes"))) return rc;
        BRM_CUDA(cudaMemcpyAsync(pl.long_rows_s, pl.long_rows_h.data(), nl * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 mem.st));
        BRM_CUDA(cudaMemcpyAsync(pl.long_nprod_s, pl.long_nprod_h.data(), nl * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, mem.st));
        BRM_CUDA(cudaStreamSynchronize(mem.st));   // host vectors must outlive the copies
    }
    return BRM_OK;
}

// Device-memory arena of the long rows of one pass: the long slots (longest
// first) cut into batches whose ping-pong slices fit the budget.
struct LongPlan {
    bool bucket = false;            // column-bucket kernels (else merge rounds)
    std::vector<int64_t> starts;    // batch boundaries over the long slots
    // numeric bucket kernels, per batch: where its work list starts in the
    // arena (after its rows), and its capacity in records
    std::vector<int64_t> work_off, work_cap;
    int64_t slots_bytes = 0, work_bytes_max = 0;
    int64_t *off_d = nullptr;       // device: arena offset of every long slot (merge rounds: of every block)
    char *arena = nullptr;
    // merge rounds: one launch of `grid` persistent blocks; block b takes
    // slot b, then the next slot from the counter; its arena holds the
    // largest of the slots it can get
    int32_t grid = 0;
    int32_t *ctr = nullptr;
};

// Long rows by column tiles (brm_long_tiles.cuh): the plan's arrays, kept from
// the pass that computes them (the symbolic pass of BRMerge-Precise and of
// prepared batches; the numeric pass itself in BRMerge-Upper) to the numeric
// pass.  They cover the long slots [long_split, count).
struct TilePlan {
    bool on = false;
    bool planned = false;          // a pass has launched the plan kernel
    TileRec *rec = nullptr;
    int64_t *base = nullptr;
    int32_t *n = nullptr, *nws = nullptr;
    int64_t *rownnz = nullptr;
    int2 *spans = nullptr;
    unsigned long long *ctr = nullptr;
    int32_t *cur = nullptr;        // per block: cursors of rows of more than kTileSmemL lists
    int32_t maxL = 0;
    int32_t grid = 0;
};

// The tiles' arrays, when the long rows of these passes take them.
int plan_tiles(Mem &mem, const Plan &pl, const brm_options &o, int64_t bcols, VKind vnum, TilePlan &wp) {
    wp = TilePlan{};
    const int64_t nl = (int64_t)pl.long_rows_h.size(), s0 = pl.long_split;
    if (nl == s0 || !tiles_apply(o, bcols)) return BRM_OK;
    const int64_t nt = nl - s0;
    std::vector<int64_t> base((size_t)nt + 1, 0);
    int64_t spans = 0, maxL = 0;
    for (int64_t s = 0; s < nt; ++s) {
        base[s + 1] = base[s] + tile_cap(pl.long_nprod_h[s0 + s], bcols);
        spans += tile_span_cap(pl.long_nprod_h[s0 + s]);
        maxL = std::max<int64_t>(maxL, pl.long_L_h[s0 + s]);
    }
    wp.grid = long_tile_grid(vnum == kIdx ? kF64 : vnum);
    int rc;
    if ((rc = get(mem, wp.base, (size_t)nt + 1, "tile offsets"))) return rc;
    if ((rc = get(mem, wp.rec, (size_t)std::max<int64_t>(base[nt], 1), "tiles"))) return rc;
    if ((rc = get(mem, wp.n, (size_t)nt, "tile counts"))) return rc;
    if ((rc = get(mem, wp.nws, (size_t)nt, "tiles per span"))) return rc;
    if ((rc = get(mem, wp.rownnz, (size_t)nt, "long-row lengths"))) return rc;
    if ((rc = get(mem, wp.spans, (size_t)std::max<int64_t>(spans, 1), "tile spans"))) return rc;
    if ((rc = get(mem, wp.ctr, 2, "span counters"))) return rc;
    if (maxL > kTileSmemL && vnum != kIdx) {
        wp.maxL = (int32_t)maxL;
        if ((rc = get(mem, wp.cur, (size_t)wp.grid * 3 * (size_t)maxL, "list cursors"))) return rc;
    }
    BRM_CUDA(cudaMemcpyAsync(wp.base, base.data(), base.size() * sizeof(int64_t), cudaMemcpyHostToDevice, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));   // the host offsets must outlive the copy
    wp.on = true;
    return BRM_OK;
}

// The tile fields of a long-row job.
void tile_job(RowJob &jb, const TilePlan &wp, bool plan_here) {
    jb.tiles = wp.rec;
    jb.tile_base = wp.base;
    jb.tile_n = wp.n;
    jb.tile_nws = wp.nws;
    jb.tile_rownnz = wp.rownnz;
    jb.tile_spans = wp.spans;
    jb.tile_ctr = wp.ctr;
    jb.tile_cur = wp.cur;
    jb.tile_maxL = wp.maxL;
    jb.tile_grid = wp.grid;
    jb.tile_plan = plan_here ? 1 : 0;
}

int plan_long(Mem &mem, VKind v, const Plan &pl, const brm_options &o, int64_t bcols, LongPlan &lp,
              bool persistent = true, const TilePlan *wp = nullptr) {
    // with column tiles, only the slots before long_split merge in rounds
    const int64_t nl = (wp && wp->on) ? pl.long_split : (int64_t)pl.long_rows_h.size();
    lp.starts.clear();
    if (nl == 0) return BRM_OK;
    // the symbolic pass counts long rows with the column bitmap whenever B has
    // at most 2^24 columns; the numeric pass uses column buckets on request
    // (they pack a list index into 16 bits and cut B's columns into at most
    // 4096 cells of at most 4096 columns)
    int64_t maxL = 0;
    for (int64_t s = 0; s < nl; ++s) maxL = std::max<int64_t>(maxL, pl.long_L_h[s]);
    lp.bucket = bcols <= kLbMaxCols && (v == kIdx || (o.long_bucket && maxL <= kLbMaxL));
    std::vector<int64_t> need(nl);
    size_t biggest = 0;
    for (int64_t s = 0; s < nl; ++s) {
        need[s] = (int64_t)long_row_bytes_for(v, pl.long_nprod_h[s], pl.long_L_h[s], lp.bucket);
        biggest = std::max(biggest, (size_t)need[s]);
    }
    size_t budget = o.arena_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = (size_t)8 << 30; }
        budget = (lp.bucket || !persistent) ? std::min<size_t>(fr / 8, (size_t)32 << 30)
                                            : std::min<size_t>(fr / 4, (size_t)64 << 30);
    }
    budget = std::max(budget, biggest);
    std::vector<int64_t> off(nl);
    size_t maxbatch = 0;
    lp.grid = 0;
    if (!lp.bucket && persistent) {
        // merge rounds: the slots are sorted by product count, largest first.
        // Block b < R merges slot b and then slots R, R + 1, ... from a
        // counter; its arena holds max(need[b], the largest need after R).
        // R is the resident block count (two 512-thread blocks of the arena
        // kernel per SM), lowered until the arena fits the budget.
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        std::vector<int64_t> tailmax(nl + 1, 0);
        for (int64_t s = nl - 1; s >= 0; --s) tailmax[s] = std::max(tailmax[s + 1], need[s]);
        int64_t R = std::min<int64_t>(nl, 2 * (int64_t)std::max(sms, 1));
        for (;; --R) {
            size_t sum = 0;
            for (int64_t b = 0; b < R; ++b) sum += (size_t)std::max(need[b], tailmax[R]);
            if (sum <= budget || R == 1) break;
        }
        size_t cur = 0;
        for (int64_t b = 0; b < R; ++b) {
            off[b] = (int64_t)cur;
            cur += (size_t)std::max(need[b], tailmax[R]);
        }
        maxbatch = cur;
        lp.grid = (int32_t)R;
        lp.starts.push_back(0);
    } else {
        size_t cur = 0;
        for (int64_t s = 0; s < nl; ++s) {
            if (s == 0 || cur + (size_t)need[s] > budget) {
                lp.starts.push_back(s);
                cur = 0;
            }
            off[s] = (int64_t)cur;
            cur += (size_t)need[s];
            maxbatch = std::max(maxbatch, cur);
        }
    }
    lp.starts.push_back(nl);
    lp.work_off.clear();
    lp.work_cap.clear();
    if (lp.bucket && v != kIdx) {
        // after each batch's rows: its work list, two counters, and the value
        // slots of the work-list kernel's blocks
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t vb = v == kF32 ? 4 : 8;
        lp.slots_bytes = (int64_t)align_up((size_t)kLbHotPerSm * std::max(sms, 1) * kLbSlots * vb, 256);
        maxbatch = 0;
        for (size_t b = 0; b + 1 < lp.starts.size(); ++b) {
            int64_t cap = 0, rows = 0;
            for (int64_t s = lp.starts[b]; s < lp.starts[b + 1]; ++s) {
                cap += lb_work_cap(pl.long_nprod_h[s]);
                rows = off[s] + need[s];
            }
            const int64_t wo = (int64_t)align_up((size_t)rows, 256);
            lp.work_off.push_back(wo);
            lp.work_cap.push_back(cap);
            const size_t wb = align_up((size_t)cap * kLbWorkBytes, 256) + 256;
            maxbatch = std::max(maxbatch, (size_t)wo + wb + (size_t)lp.slots_bytes);
        }
    }
    int rc = get(mem, lp.off_d, nl, "arena offsets");
    if (rc) return rc;
    if ((rc = get(mem, lp.arena, maxbatch, "long-row arena"))) return rc;
    if (lp.grid > 0 && (rc = get(mem, lp.ctr, 1, "long-row counter"))) return rc;
    BRM_CUDA(cudaMemcpyAsync(lp.off_d, off.data(), nl * sizeof(int64_t), cudaMemcpyHostToDevice, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));   // the host offsets must outlive the copy
    return BRM_OK;
}

// Kernel launches of one pass over every bin (no host synchronisation, no
// allocation: a numeric pass of a prepared plan can be captured in a graph).
int launch_pass(VKind v, const Plan &pl, const LongPlan &lp, const RowJob &j, cudaStream_t st, bool trace,
                const TilePlan *wp = nullptr) {
    for (int b = kBinReg0; b <= kBinBlock; ++b) {
        RowJob jb = j;
        jb.rows = pl.rows + pl.base[b];
        jb.count = (int32_t)pl.stats.count[b];
        if (jb.count == 0) continue;
        const int ph = b < kBinWarp ? kPhSymReg : kPhSymWarp + (b - kBinWarp);
        PhaseScope ps(trace ? (v == kIdx ? ph : ph + (kPhNumReg - kPhSymReg)) : -1, st);
        BRM_CUDA(launch_rows(v, b, jb, st));
    }
    if (wp && wp->on) {
        // the tiled long rows in one launch (two with the plan)
        RowJob jb = j;
        jb.rows = pl.long_rows_s + pl.long_split;
        jb.count = (int32_t)((int64_t)pl.long_rows_h.size() - pl.long_split);
        jb.slot_nprod = pl.long_nprod_s + pl.long_split;
        tile_job(jb, *wp, v == kIdx || !wp->planned);
        PhaseScope ps(trace ? (v == kIdx ? kPhSymTile : kPhNumTile) : -1, st);
        BRM_CUDA(launch_rows(v, kBinLong, jb, st));
    }
    if (lp.starts.size() < 2) return BRM_OK;
    PhaseScope ps(trace ? (v == kIdx ? kPhSymLong : kPhNumLong) : -1, st);
    for (size_t bi = 0; bi + 1 < lp.starts.size(); ++bi) {
        RowJob jb = j;
        jb.rows = pl.long_rows_s + lp.starts[bi];
        jb.count = (int32_t)(lp.starts[bi + 1] - lp.starts[bi]);
        jb.long_bucket = lp.bucket ? 1 : 0;
        jb.arena = lp.arena;
        jb.arena_off = lp.off_d + lp.starts[bi];
        if (bi < lp.work_off.size()) {
            char *w = lp.arena + lp.work_off[bi];
            const size_t wb = align_up((size_t)lp.work_cap[bi] * kLbWorkBytes, 256);
            jb.lb_work = w;
            jb.lb_ctr = reinterpret_cast<int32_t *>(w + wb);
            jb.lb_slots = w + wb + 256;
            jb.lb_cap = lp.work_cap[bi];
        }
        jb.slot_nprod = pl.long_nprod_s + lp.starts[bi];
        if (lp.grid > 0) {
            jb.long_grid = lp.grid;
            jb.long_ctr = lp.ctr;
            BRM_CUDA(cudaMemsetAsync(lp.ctr, 0, sizeof(int32_t), st));
        }
        BRM_CUDA(launch_rows(v, kBinLong, jb, st));
    }
    return BRM_OK;
}

// One BRMerge pass (symbolic or numeric) over all bins.
int run_pass(Mem &mem, VKind v, const Plan &pl, const brm_options &o, RowJob j, bool persistent = true,
             TilePlan *wp = nullptr) {
    LongPlan lp;
    int rc = plan_long(mem, v, pl, o, j.bcols, lp, persistent, wp);
    if (rc) return rc;
    if ((rc = launch_pass(v, pl, lp, j, mem.st, true, wp))) return rc;
    if (wp && wp->on) wp->planned = true;
    if (lp.arena) {
        mem.free_one(lp.arena);   // stream-ordered release after the launches
        mem.free_one(lp.off_d);
        mem.free_one(lp.ctr);
    }
    return BRM_OK;
}

// Reads the row-length flag of a numeric pass (synchronises the stream).
int check_flag(Mem &mem, const unsigned int *err) {
    unsigned int h = 0;
    BRM_CUDA(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    if (h) return fail(BRM_ERR_INVALID, "a numeric row length disagrees with its symbolic count");
    return BRM_OK;
}

RowJob base_job(const Src &src, const brm_options &o) {
    RowJob j{};
    j.prods = src.prods;
    j.prod_of = src.prod_of;
    j.reg_keys = o.reg_keys;
    j.reg_warps = o.reg_warps;
    j.sym_hash = o.symbolic_hash ? 1 : 0;
    j.num_half = o.reg_num_half ? 1 : 0;
    j.num_direct = o.reg_num_direct ? 1 : 0;
    j.bcols = src.bcols;
    j.arp = src.arp;
    j.acol = src.acol;
    j.aval = src.aval;
    j.brp = src.brp;
    j.bcol = src.bcol;
    j.bval = src.bval;
    return j;
}

VKind value_kind(int32_t dtype, const brm_options &o) {
    if (dtype == BRM_F64) return kF64;
    return o.compensated ? kF32C : kF32;
}

size_t value_bytes(int32_t dtype) { return dtype == BRM_F64 ? 8 : 4; }

// Symbolic phase into row_ptr (m+1, device); returns nnz(C) on the host.
// The recorded orders of the register-bin rows (written by the symbolic
// pass, read by the numeric pass): one 16-bit entry per product, row i's
// entries at perm_off[i].
struct PermBuf {
    uint16_t *perm = nullptr;
    int64_t *perm_off = nullptr;
};

int symbolic_into(Mem &mem, const Src &src, const brm_options &o, Plan &pl, int64_t *row_ptr, int64_t *nnz,
                  PermBuf *pb = nullptr, TilePlan *wp = nullptr) {
    const int64_t m = src.m;
    int64_t *row_nnz;
    int rc = get(mem, row_nnz, (size_t)std::max<int64_t>(m, 1), "row counts");
    if (rc) return rc;
    if ((rc = make_plan(mem, src, o, pl, nullptr, row_nnz))) return rc;
    if (wp && (rc = plan_tiles(mem, pl, o, src.bcols, value_kind(src.dtype, o), *wp))) return rc;
    void *tmp;
    if (!(tmp = mem.get(scan_tmp_bytes(m)))) return fail(BRM_ERR_OOM, "scan workspace");
    RowJob j = base_job(src, o);
    j.out_cnt = row_nnz;
    if (pb && o.reg_perm && !o.symbolic_hash && pl.stats.reg_nprod > 0) {
        int64_t *masked;
        if ((rc = get(mem, masked, (size_t)std::max<int64_t>(m, 1), "register-row products"))) return rc;
        if ((rc = get(mem, pb->perm_off, (size_t)m + 1, "recorded-order offsets"))) return rc;
        size_t reg_rows = 0;
        for (int b = kBinReg0; b < kBinReg0 + kNumRegBins; ++b) reg_rows += (size_t)pl.stats.count[b];
        // every row's segment padded to a multiple of 16 entries
        if ((rc = get(mem, pb->perm, (size_t)pl.stats.reg_nprod + 15 * reg_rows, "recorded orders"))) return rc;
        {
            PhaseScope ps(kPhScan, mem.st);
            BRM_CUDA(launch_reg_nprod(m, pl.bin_of, pl.nprod, masked, mem.st));
            BRM_CUDA(launch_scan(masked, pb->perm_off, m, tmp, mem.st));
        }
        mem.free_one(masked);
        j.perm = pb->perm;
        j.perm_off = pb->perm_off;
    }
    if ((rc = run_pass(mem, kIdx, pl, o, j, true, wp))) return rc;
    {
        PhaseScope ps(kPhScan, mem.st);
        BRM_CUDA(launch_scan(row_nnz, row_ptr, m, tmp, mem.st));
    }
    BRM_CUDA(cudaMemcpyAsync(nnz, row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    mem.free_one(tmp);
    mem.free_one(row_nnz);
    return BRM_OK;
}

int precise(const brm_csr *A, const brm_csr *B, brm_csr_out *C, const brm_options *opts, const brm_allocator *al,
            cudaStream_t st) {
    if (!C) return fail(BRM_ERR_INVALID, "C is NULL");
    std::memset(C, 0, sizeof *C);
    int rc = check_pair(A, B, true);
    if (rc) return rc;
    const brm_options o = resolve(opts);
    Mem mem(al, st);
    if (o.validate && (rc = validate_inputs(mem, A, B))) return rc;
    const int64_t m = A->rows;
    int64_t *rp;
    if ((rc = get_own(mem, rp, (size_t)m + 1, "C.row_ptr"))) return rc;
    mem.reserve(row_workspace_bytes(m));
    Plan pl;
    int64_t nnz = 0;
    const Src src = src_of(A, B);
    PermBuf pb;
    TilePlan wp;
    if ((rc = symbolic_into(mem, src, o, pl, rp, &nnz, &pb, &wp))) return rc;
    int32_t *col;
    if ((rc = get_own(mem, col, (size_t)std::max<int64_t>(nnz, 1), "C.col_idx"))) return rc;
    void *val = mem.get_direct((size_t)std::max<int64_t>(nnz, 1) * value_bytes(A->dtype));
    if (!val) return fail(BRM_ERR_OOM, "allocation of C.val failed");
    RowJob j = base_job(src, o);
    j.out_rp = rp;
    j.out_col = col;
    j.out_val = val;
    j.perm = pb.perm;
    j.perm_off = pb.perm_off;
    unsigned int *err;
    if ((rc = get(mem, err, 1, "error flag"))) return rc;
    BRM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), mem.st));
    j.err = err;
    j.exact = 1;
    if ((rc = run_pass(mem, value_kind(A->dtype, o), pl, o, j, true, &wp))) return rc;
    if ((rc = check_flag(mem, err))) return rc;
    mem.detach(rp);
    mem.detach(col);
    mem.detach(val);
    C->rows = m;
    C->cols = B->cols;
    C->nnz = nnz;
    C->row_ptr = rp;
    C->col_idx = col;
    C->val = val;
    C->dtype = A->dtype;
    return BRM_OK;
}

// BRMerge-Upper in row chunks whose C_bar fits `budget` bytes (the paper's
// Upper allocates C_bar in per-thread parts, Section III-D-1; here the parts
// are processed one after another so that C_bar never exceeds the budget).
// Every chunk is merged into the reused C_bar and compacted into a buffer of
// its exact size; C is then allocated and the chunks copied into it in order.
// Peak memory: about twice C plus one chunk's C_bar.
int upper_chunked(Mem &mem, const brm_csr *A, const brm_csr *B, brm_csr_out *C, const brm_options &o,
                  const Src &src, int64_t *nprod, int64_t *row_size, const int64_t *cbar_off, void *tmp,
                  size_t budget) {
    const int64_t m = A->rows;
    const size_t vb = value_bytes(A->dtype), per = 4 + vb;
    std::vector<int64_t> off_h((size_t)m + 1);
    BRM_CUDA(cudaMemcpyAsync(off_h.data(), cbar_off, ((size_t)m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    const int64_t cap = std::max<int64_t>((int64_t)(budget / per), 1);
    std::vector<int64_t> bounds{0};
    int64_t biggest = 1;
    while (bounds.back() < m) {
        const int64_t r0 = bounds.back();
        // the most rows from r0 whose products fit the chunk (at least one row)
        int64_t r1 = (int64_t)(std::upper_bound(off_h.begin() + r0 + 1, off_h.end(), off_h[r0] + cap) -
                               off_h.begin()) - 1;
        r1 = std::max(r1, r0 + 1);
        biggest = std::max(biggest, off_h[r1] - off_h[r0]);
        bounds.push_back(r1);
    }
    int32_t *ccol;
    int rc = get(mem, ccol, (size_t)biggest, "C_bar chunk columns");
    if (rc) return rc;
    void *cval = mem.get((size_t)biggest * vb);
    if (!cval) return fail(BRM_ERR_OOM, "allocation of a C_bar chunk (%lld products) failed", (long long)biggest);
    int64_t maxrows = 1;
    for (size_t c = 0; c + 1 < bounds.size(); ++c) maxrows = std::max(maxrows, bounds[c + 1] - bounds[c]);
    int64_t *loc_off, *loc_rp;
    if ((rc = get(mem, loc_off, (size_t)maxrows + 1, "chunk C_bar offsets"))) return rc;
    if ((rc = get(mem, loc_rp, (size_t)maxrows + 1, "chunk row pointer"))) return rc;
    unsigned int *err;
    if ((rc = get(mem, err, 1, "error flag"))) return rc;
    BRM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), mem.st));
    struct Piece { int32_t *col; void *val; int64_t nnz; };
    std::vector<Piece> pieces;
    const VKind v = value_kind(A->dtype, o);
    for (size_t c = 0; c + 1 < bounds.size(); ++c) {
        const int64_t r0 = bounds[c], rows = bounds[c + 1] - bounds[c];
        Src sub = src;
        sub.m = rows;
        sub.arp = A->row_ptr + r0;
        Plan pc;
        if ((rc = make_plan(mem, sub, o, pc, nprod + r0, row_size + r0))) return rc;
        {
            PhaseScope ps(kPhScan, mem.st);
            BRM_CUDA(launch_scan(nprod + r0, loc_off, rows, tmp, mem.st));
        }
        RowJob j = base_job(sub, o);
        j.out_rp = loc_off;
        j.out_col = ccol;
        j.out_val = cval;
        j.out_cnt = row_size + r0;
        j.err = err;
        // long rows in arena-sized batches of one block per row, an eighth of
        // what is free at a time: the compacted chunks pile up to the size of
        // C, and persistent blocks with a larger arena left the caller's
        // allocator no room for C at the end (R-MAT scale 20)
        if ((rc = run_pass(mem, v, pc, o, j, false))) return rc;
        {
            PhaseScope ps(kPhScan, mem.st);
            BRM_CUDA(launch_scan(row_size + r0, loc_rp, rows, tmp, mem.st));
        }
        Piece pc_out{nullptr, nullptr, 0};
        BRM_CUDA(cudaMemcpyAsync(&pc_out.nnz, loc_rp + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, mem.st));
        BRM_CUDA(cudaStreamSynchronize(mem.st));
        if ((rc = get_own(mem, pc_out.col, (size_t)std::max<int64_t>(pc_out.nnz, 1), "chunk columns"))) return rc;
        pc_out.val = mem.get_direct((size_t)std::max<int64_t>(pc_out.nnz, 1) * vb);
        if (!pc_out.val) return fail(BRM_ERR_OOM, "allocation of a compacted chunk failed");
        {
            PhaseScope ps(kPhCompact, mem.st);
            BRM_CUDA(launch_compact(rows, loc_off, loc_rp, ccol, cval, pc_out.col, pc_out.val, vb, mem.st));
        }
        pieces.push_back(pc_out);
    }
    mem.free_one(cval);
    mem.free_one(ccol);
    int64_t *rp;
    if ((rc = get_own(mem, rp, (size_t)m + 1, "C.row_ptr"))) return rc;
    {
        PhaseScope ps(kPhScan, mem.st);
        BRM_CUDA(launch_scan(row_size, rp, m, tmp, mem.st));
    }
    int64_t nnz = 0;
    for (const Piece &p : pieces) nnz += p.nnz;
    int32_t *col;
    if ((rc = get_own(mem, col, (size_t)std::max<int64_t>(nnz, 1), "C.col_idx"))) return rc;
    void *val = mem.get_direct((size_t)std::max<int64_t>(nnz, 1) * vb);
    if (!val) return fail(BRM_ERR_OOM, "allocation of C.val failed");
    int64_t at = 0;
    for (const Piece &p : pieces) {
        if (p.nnz > 0) {
            BRM_CUDA(cudaMemcpyAsync(col + at, p.col, (size_t)p.nnz * 4, cudaMemcpyDeviceToDevice, mem.st));
            BRM_CUDA(cudaMemcpyAsync(static_cast<char *>(val) + (size_t)at * vb, p.val, (size_t)p.nnz * vb,
                                     cudaMemcpyDeviceToDevice, mem.st));
        }
        at += p.nnz;
        mem.free_one(p.col);
        mem.free_one(p.val);
    }
    if ((rc = check_flag(mem, err))) return rc;
    mem.detach(rp);
    mem.detach(col);
    mem.detach(val);
    C->rows = m;
    C->cols = B->cols;
    C->nnz = nnz;
    C->row_ptr = rp;
    C->col_idx = col;
    C->val = val;
    C->dtype = A->dtype;
    return BRM_OK;
}

int upper(const brm_csr *A, const brm_csr *B, brm_csr_out *C, const brm_options *opts, const brm_allocator *al,
          cudaStream_t st) {
    if (!C) return fail(BRM_ERR_INVALID, "C is NULL");
    std::memset(C, 0, sizeof *C);
    int rc = check_pair(A, B, true);
    if (rc) return rc;
    const brm_options o = resolve(opts);
    Mem mem(al, st);
    if (o.validate && (rc = validate_inputs(mem, A, B))) return rc;
    const int64_t m = A->rows;
    const size_t vb = value_bytes(A->dtype);
    int64_t *nprod, *row_size, *cbar_off, *rp;
    mem.reserve(row_workspace_bytes(m));
    if ((rc = get(mem, nprod, (size_t)std::max<int64_t>(m, 1), "row nprod"))) return rc;
    if ((rc = get(mem, row_size, (size_t)std::max<int64_t>(m, 1), "row sizes"))) return rc;
    if ((rc = get(mem, cbar_off, (size_t)m + 1, "C_bar offsets"))) return rc;
    Plan pl;
    const Src src = src_of(A, B);
    if ((rc = make_plan(mem, src, o, pl, nprod, row_size))) return rc;
    void *tmp;
    if (!(tmp = mem.get(scan_tmp_bytes(m)))) return fail(BRM_ERR_OOM, "scan workspace");
    // steps 1 and 3: prefix sum of the upper bounds, temporary C_bar
    {
        PhaseScope ps(kPhScan, mem.st);
        BRM_CUDA(launch_scan(nprod, cbar_off, m, tmp, mem.st));
    }
    const int64_t total = (int64_t)pl.stats.total_nprod;
    const size_t per = 4 + vb;
    size_t budget = o.upper_chunk_bytes;
    int32_t *ccol = nullptr;
    void *cval = nullptr;
    if (budget == 0 || (size_t)std::max<int64_t>(total, 1) * per <= budget) {
        ccol = static_cast<int32_t *>(mem.get_direct((size_t)std::max<int64_t>(total, 1) * 4));
        if (ccol) cval = mem.get_direct((size_t)std::max<int64_t>(total, 1) * vb);
        if (!ccol || !cval) {
            // the whole C_bar does not fit: row chunks of a quarter of what is free
            mem.free_one(ccol);
            ccol = nullptr;
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = (size_t)4 << 30; }
            budget = std::max<size_t>(fr / 4, (size_t)1 << 20);
        }
    }
    if (!cval)
        return upper_chunked(mem, A, B, C, o, src, nprod, row_size, cbar_off, tmp, budget);
    // step 4: BRMerge into C_bar, recording the row sizes
    RowJob j = base_job(src, o);
    j.out_rp = cbar_off;
    j.out_col = ccol;
    j.out_val = cval;
    j.out_cnt = row_size;
    unsigned int *err;
    if ((rc = get(mem, err, 1, "error flag"))) return rc;
    BRM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), mem.st));
    j.err = err;
    TilePlan wp;
    if ((rc = plan_tiles(mem, pl, o, src.bcols, value_kind(A->dtype, o), wp))) return rc;
    if ((rc = run_pass(mem, value_kind(A->dtype, o), pl, o, j, true, &wp))) return rc;
    // step 5: prefix sum of the row sizes, allocation of C
    if ((rc = get_own(mem, rp, (size_t)m + 1, "C.row_ptr"))) return rc;
    {
        PhaseScope ps(kPhScan, mem.st);
        BRM_CUDA(launch_scan(row_size, rp, m, tmp, mem.st));
    }
    int64_t nnz = 0;
    BRM_CUDA(cudaMemcpyAsync(&nnz, rp + m, sizeof(int64_t), cudaMemcpyDeviceToHost, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));
    int32_t *col;
    if ((rc = get_own(mem, col, (size_t)std::max<int64_t>(nnz, 1), "C.col_idx"))) return rc;
    void *val = mem.get_direct((size_t)std::max<int64_t>(nnz, 1) * vb);
    if (!val) return fail(BRM_ERR_OOM, "allocation of C.val failed");
    // step 6: copy C_bar into C
    {
        PhaseScope ps(kPhCompact, mem.st);
        BRM_CUDA(launch_compact(m, cbar_off, rp, ccol, cval, col, val, vb, mem.st));
    }
    if ((rc = check_flag(mem, err))) return rc;
    mem.detach(rp);
    mem.detach(col);
    mem.detach(val);
    C->rows = m;
    C->cols = B->cols;
    C->nnz = nnz;
    C->row_ptr = rp;
    C->col_idx = col;
    C->val = val;
    C->dtype = A->dtype;
    return BRM_OK;
}

// ---------------------------------------------------------------------------
// Batched products: C_p = A_p * B_p for p = 0 .. count-1, processed as one
// stacked problem.  Row r of the stack is row r - row0[p] of product p; the
// kernels find each row's A and B through a device table of the products, so
// every bin of every product is served by one launch per bin, and the result
// is the vertical stack of the C_p (one int64 row pointer, columns in each
// product's own column space).
// ---------------------------------------------------------------------------
int batch_setup(Mem &mem, int32_t count, const brm_csr *A, const brm_csr *B, const brm_options &o, Src &src,
                std::vector<int64_t> &row0) {
    if (count < 0) return fail(BRM_ERR_INVALID, "count is negative");
    if (count > 0 && (!A || !B)) return fail(BRM_ERR_INVALID, "A and B must not be NULL");
    std::vector<ProdDesc> d((size_t)std::max(count, 1));
    std::vector<int64_t> rows_of((size_t)std::max(count, 1), 0);
    row0.assign((size_t)count + 1, 0);
    int64_t M = 0, bcols = 0;
    const int32_t dtype = count > 0 ? A[0].dtype : BRM_F64;
    for (int32_t p = 0; p < count; ++p) {
        int rc = check_pair(&A[p], &B[p], true);
        if (rc) return fail(rc, "product %d: %s", p, g_err.c_str());
        if (A[p].dtype != dtype) return fail(BRM_ERR_DTYPE, "product %d has another dtype than product 0", p);
        d[p] = ProdDesc{A[p].row_ptr, A[p].col_idx, A[p].val, B[p].row_ptr, B[p].col_idx, B[p].val, M};
        row0[p] = M;
        rows_of[p] = A[p].rows;
        M += A[p].rows;
        bcols = std::max<int64_t>(bcols, B[p].cols);
    }
    row0[count] = M;
    if (M >= INT32_MAX) return fail(BRM_ERR_OVERFLOW, "the batch has %lld rows (limit 2^31-1)", (long long)M);
    if (o.validate)
        for (int32_t p = 0; p < count; ++p) {
            int rc = validate_inputs(mem, &A[p], &B[p]);
            if (rc) return fail(rc, "product %d: %s", p, g_err.c_str());
        }
    ProdDesc *dd;
    int64_t *ro;
    int32_t *po;
    int rc = get(mem, dd, d.size(), "product table");
    if (rc) return rc;
    if ((rc = get(mem, ro, rows_of.size(), "product rows"))) return rc;
    if ((rc = get(mem, po, (size_t)std::max<int64_t>(M, 1), "row products"))) return rc;
    BRM_CUDA(cudaMemcpyAsync(dd, d.data(), d.size() * sizeof(ProdDesc), cudaMemcpyHostToDevice, mem.st));
    BRM_CUDA(cudaMemcpyAsync(ro, rows_of.data(), rows_of.size() * sizeof(int64_t), cudaMemcpyHostToDevice, mem.st));
    BRM_CUDA(launch_fill_prod_of(dd, ro, count, po, mem.st));
    BRM_CUDA(cudaStreamSynchronize(mem.st));   // the host tables must outlive the copies
    src = Src{};
    src.m = M;
    src.bcols = bcols;
    src.dtype = dtype;
    src.prods = dd;
    src.prod_of = po;
    return BRM_OK;
}

}  // namespace
}  // namespace brm

// A prepared batch (opaque in brm.h): the symbolic pass is done, C is
// allocated and the long-row arena is planned, so the numeric pass is kernel
// launches only and can be replayed (on new values of the same patterns) or
// captured in a CUDA graph.
struct brm_batch {
    brm_allocator al{};
    bool has_al = false;
    brm::Mem mem;
    brm_options o{};
    brm::Src src;
    brm::Plan pl;
    brm::LongPlan lp;
    brm::RowJob job{};
    brm::PermBuf pb;
    brm::TilePlan wp;
    brm::VKind v = brm::kF64;
    int32_t count = 0;
    int64_t nnz = 0;
    std::vector<int64_t> row0;
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    void *val = nullptr;
    unsigned int *err = nullptr;
    bool taken = false;
    cudaStream_t cap = nullptr;          // private stream for graph capture
    cudaGraphExec_t exec = nullptr;
    long long graph_launches = 0;        // kernels in the captured graph

    brm_batch(const brm_allocator *a, cudaStream_t s)
        : al(a ? *a : brm_allocator{}), has_al(a != nullptr), mem(has_al ? &al : nullptr, s) {}
    ~brm_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        if (taken) {
            mem.detach(rp);
            mem.detach(col);
            mem.detach(val);
        }
    }
};

namespace brm {
namespace {

int batch_create(int32_t count, const brm_csr *A, const brm_csr *B, const brm_options *opts,
                 const brm_allocator *al, cudaStream_t st, brm_batch **out) {
    if (!out) return fail(BRM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    brm_batch *b = new brm_batch(al, st);
    b->o = resolve(opts);
    b->count = count;
    int rc = batch_setup(b->mem, count, A, B, b->o, b->src, b->row0);
    const int64_t M = b->src.m;
    if (!rc) rc = get_own(b->mem, b->rp, (size_t)M + 1, "C.row_ptr");
    if (!rc) b->mem.reserve(row_workspace_bytes(M));
    if (!rc) rc = symbolic_into(b->mem, b->src, b->o, b->pl, b->rp, &b->nnz, &b->pb, &b->wp);
    if (!rc) rc = get_own(b->mem, b->col, (size_t)std::max<int64_t>(b->nnz, 1), "C.col_idx");
    if (!rc) {
        b->val = b->mem.get_direct((size_t)std::max<int64_t>(b->nnz, 1) * value_bytes(b->src.dtype));
        if (!b->val) rc = fail(BRM_ERR_OOM, "allocation of C.val failed");
    }
    if (!rc) rc = get(b->mem, b->err, 1, "error flag");
    b->v = value_kind(b->src.dtype, b->o);
    if (!rc) rc = plan_long(b->mem, b->v, b->pl, b->o, b->src.bcols, b->lp, true, &b->wp);
    if (rc) {
        delete b;
        return rc;
    }
    RowJob j = base_job(b->src, b->o);
    j.out_rp = b->rp;
    j.out_col = b->col;
    j.out_val = b->val;
    j.err = b->err;
    j.exact = 1;
    j.perm = b->pb.perm;
    j.perm_off = b->pb.perm_off;
    b->job = j;
    *out = b;
    return BRM_OK;
}

// The numeric pass of a prepared batch: launches only.
int batch_numeric(brm_batch *b, cudaStream_t st, bool trace) {
    BRM_CUDA(cudaMemsetAsync(b->err, 0, sizeof(unsigned int), st));
    return launch_pass(b->v, b->pl, b->lp, b->job, st, trace, &b->wp);
}

int batch_check(brm_batch *b, cudaStream_t st) {
    unsigned int h = 0;
    BRM_CUDA(cudaMemcpyAsync(&h, b->err, sizeof h, cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(BRM_ERR_INVALID, "a numeric row length disagrees with its symbolic count");
    return BRM_OK;
}

int batch_graph_launch(brm_batch *b, cudaStream_t st) {
    if (!b->exec) {
        if (!b->cap) BRM_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        // the batch's memory was made on the creation stream: order the
        // capture stream after it once
        BRM_CUDA(cudaStreamSynchronize(b->mem.st));
        const long long n0 = g_launches.load();
        BRM_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        const int rc = batch_numeric(b, b->cap, false);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        b->graph_launches = g_launches.load() - n0;
        g_launches.fetch_sub(b->graph_launches);   // counted when the graph runs
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(BRM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            b->exec = nullptr;
            return fail(BRM_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e2));
        }
    }
    BRM_CUDA(cudaGraphLaunch(b->exec, st));
    g_launches.fetch_add(b->graph_launches);
    return BRM_OK;
}

void batch_result(const brm_batch *b, brm_csr_out *C, int64_t *row_offset) {
    if (C) {
        C->rows = b->src.m;
        C->cols = b->src.bcols;
        C->nnz = b->nnz;
        C->row_ptr = b->rp;
        C->col_idx = b->col;
        C->val = b->val;
        C->dtype = b->src.dtype;
    }
    if (row_offset)
        for (size_t p = 0; p < b->row0.size(); ++p) row_offset[p] = b->row0[p];
}

}  // namespace
}  // namespace brm

using namespace brm;

extern "C" {

void brm_options_default(brm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->validate = 0;
    o->compensated = 0;
    o->warp_max_nprod = kWarpCap;
    o->block_max_nprod = kBlockCap;
    o->reg_max_nprod = kRegMaxNprod;
    o->reg_keys = kRegKeysDefault;
    o->reg_warps = kRegWarpsDefault;
    o->reg_top = 1;
    o->reg_perm = 1;
    o->reg_num_half = 1;
    o->reg_num_direct = 1;
    o->long_bucket = 0;
    o->symbolic_hash = 0;
    o->arena_bytes = 0;
    o->long_window = 1;
}

const char *brm_last_error(void) { return g_err.c_str(); }

const char *brm_version(void) { return "brm 0.1 (sm_103a)"; }

int brm_spgemm_precise(const brm_csr *A, const brm_csr *B, brm_csr_out *C, const brm_options *opts,
                       const brm_allocator *alloc, void *stream) {
    g_err.clear();
    const int rc = precise(A, B, C, opts, alloc, static_cast<cudaStream_t>(stream));
    g_trace.flush();
    return rc;
}

int brm_spgemm_upper(const brm_csr *A, const brm_csr *B, brm_csr_out *C, const brm_options *opts,
                     const brm_allocator *alloc, void *stream) {
    g_err.clear();
    const int rc = upper(A, B, C, opts, alloc, static_cast<cudaStream_t>(stream));
    g_trace.flush();
    return rc;
}

int brm_spgemm_symbolic(const brm_csr *A, const brm_csr *B, int64_t *C_row_ptr, int64_t *nnz_C,
                        const brm_options *opts, const brm_allocator *alloc, void *stream) {
    g_err.clear();
    int rc = check_pair(A, B, false);
    if (rc) return rc;
    if (!C_row_ptr || !nnz_C) return fail(BRM_ERR_INVALID, "C_row_ptr and nnz_C must not be NULL");
    const brm_options o = resolve(opts);
    Mem mem(alloc, static_cast<cudaStream_t>(stream));
    if (o.validate && (rc = validate_inputs(mem, A, B))) return rc;
    mem.reserve(row_workspace_bytes(A->rows));
    Plan pl;
    rc = symbolic_into(mem, src_of(A, B), o, pl, C_row_ptr, nnz_C);
    g_trace.flush();
    return rc;
}

int brm_spgemm_backward(const brm_csr *A, const brm_csr *B, const int64_t *C_row_ptr, const int32_t *C_col_idx,
                        const void *dC, void *dA_val, void *dB_val, const brm_options *opts,
                        const brm_allocator *alloc, void *stream) {
    g_err.clear();
    (void)opts;
    int rc = check_pair(A, B, true);
    if (rc) return rc;
    if (!C_row_ptr || (A->rows > 0 && (!C_col_idx || !dC)))
        return fail(BRM_ERR_INVALID, "C_row_ptr, C_col_idx and dC must not be NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Mem mem(alloc, st);
    unsigned int *err;
    if ((rc = get(mem, err, 1, "error flag"))) return rc;
    BRM_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    BackwardArgs a{};
    a.m = A->rows;
    a.nnz_a = A->nnz;
    a.ka = A->cols;
    a.kb = B->rows;
    a.nnz_b = B->nnz;
    if (dB_val && B->nnz > 0 && A->nnz > 0) {
        // A^T's rows for the ordered dB sums, and every product's G_ij
        int64_t nprod = 0;
        {
            BinStats *bs;
            if ((rc = get(mem, bs, 1, "statistics"))) return rc;
            BRM_CUDA(cudaMemsetAsync(bs, 0, sizeof(BinStats), st));
            BinArgs ba{};
            ba.m = A->rows;
            ba.arp = A->row_ptr;
            ba.acol = A->col_idx;
            ba.brp = B->row_ptr;
            ba.reg_keys = kRegKeysDefault;
            ba.warp_cap = kWarpCap;
            ba.block_cap = kBlockCap;
            ba.block_lcap = kBlockLCap;
            ba.st = bs;
            BRM_CUDA(launch_bin(ba, st));
            BinStats h{};
            BRM_CUDA(cudaMemcpyAsync(&h, bs, sizeof h, cudaMemcpyDeviceToHost, st));
            BRM_CUDA(cudaStreamSynchronize(st));
            nprod = (int64_t)h.total_nprod;
            mem.free_one(bs);
        }
        const size_t ka = (size_t)std::max<int64_t>(A->cols, 1);
        if ((rc = get(mem, a.ws_cnt, ka, "backward column counts"))) return rc;
        if ((rc = get(mem, a.ws_colptr, ka + 1, "backward column starts"))) return rc;
        if (!(a.ws_scan = mem.get(scan_tmp_bytes(A->cols)))) return fail(BRM_ERR_OOM, "backward scan workspace");
        if (!(a.ws_scan2 = mem.get(scan_tmp_bytes(A->nnz)))) return fail(BRM_ERR_OOM, "backward scan workspace");
        if ((rc = get(mem, a.ws_ent, (size_t)A->nnz, "backward column entries"))) return rc;
        if ((rc = get(mem, a.ws_row, (size_t)A->nnz, "backward entry rows"))) return rc;
        if ((rc = get(mem, a.ws_plen, (size_t)A->nnz, "backward product counts"))) return rc;
        if ((rc = get(mem, a.ws_poff, (size_t)A->nnz + 1, "backward product offsets"))) return rc;
        if (!(a.ws_gp = mem.get((size_t)std::max<int64_t>(nprod, 1) * value_bytes(A->dtype))))
            return fail(BRM_ERR_OOM, "backward per-product gradients (%lld values)", (long long)nprod);
    } else if (dB_val && B->nnz > 0) {
        BRM_CUDA(cudaMemsetAsync(dB_val, 0, (size_t)B->nnz * value_bytes(A->dtype), st));   // A has no entries
        dB_val = nullptr;
    }
    a.arp = A->row_ptr;
    a.acol = A->col_idx;
    a.aval = A->val;
    a.brp = B->row_ptr;
    a.bcol = B->col_idx;
    a.bval = B->val;
    a.crp = C_row_ptr;
    a.ccol = C_col_idx;
    a.dC = dC;
    a.dA = dA_val;
    a.dB = dB_val;
    a.err = err;
    {
        PhaseScope ps(kPhBackward, st);
        BRM_CUDA(launch_backward(a, A->dtype == BRM_F64, st));
    }
    unsigned int h = 0;
    BRM_CUDA(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    g_trace.flush();
    if (h) return fail(BRM_ERR_INVALID, "C's pattern does not contain every column of A * B");
    return BRM_OK;
}

void brm_csr_out_free(brm_csr_out *C, const brm_allocator *alloc, void *stream) {
    if (!C) return;
    Mem mem(alloc, static_cast<cudaStream_t>(stream));
    if (C->row_ptr) mem.release(C->row_ptr);
    if (C->col_idx) mem.release(C->col_idx);
    if (C->val) mem.release(C->val);
    std::memset(C, 0, sizeof *C);
}

int brm_row_nprod(const brm_csr *A, const brm_csr *B, int64_t *row_nprod, int64_t *total_nprod,
                  int64_t *max_row_nprod, int64_t *max_row_nnz_A, void *stream) {
    g_err.clear();
    int rc = check_pair(A, B, false);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Mem mem(nullptr, st);
    BinStats *bs;
    if ((rc = get(mem, bs, 1, "statistics"))) return rc;
    BRM_CUDA(cudaMemsetAsync(bs, 0, sizeof(BinStats), st));
    BinArgs a{};
    a.m = A->rows;
    a.arp = A->row_ptr;
    a.acol = A->col_idx;
    a.brp = B->row_ptr;
    a.reg_max_tpr = 0;
    a.reg_keys = kRegKeysDefault;
    a.warp_cap = kWarpCap;
    a.block_cap = kBlockCap;
    a.block_lcap = kBlockLCap;
    a.nprod = row_nprod;
    a.st = bs;
    {
        PhaseScope ps(kPhBin, st);
        BRM_CUDA(launch_bin(a, st));
    }
    BinStats h{};
    BRM_CUDA(cudaMemcpyAsync(&h, bs, sizeof h, cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    if (total_nprod) *total_nprod = (int64_t)h.total_nprod;
    if (max_row_nprod) *max_row_nprod = (int64_t)h.max_nprod;
    if (max_row_nnz_A) *max_row_nnz_A = (int64_t)h.max_L;
    g_trace.flush();
    return BRM_OK;
}

int brm_row_split(const brm_csr *A, const brm_csr *B, int32_t parts, int64_t *bounds, const brm_allocator *alloc,
                  void *stream) {
    g_err.clear();
    int rc = check_pair(A, B, false);
    if (rc) return rc;
    if (parts < 1) return fail(BRM_ERR_INVALID, "parts must be at least 1 (got %d)", parts);
    if (!bounds) return fail(BRM_ERR_INVALID, "bounds is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t m = A->rows;
    Mem mem(alloc, st);
    BinStats *bs;
    int64_t *nprod, *excl, *db;
    if ((rc = get(mem, bs, 1, "statistics"))) return rc;
    if ((rc = get(mem, nprod, (size_t)std::max<int64_t>(m, 1), "row nprod"))) return rc;
    if ((rc = get(mem, excl, (size_t)m + 1, "product prefix"))) return rc;
    if ((rc = get(mem, db, (size_t)parts + 1, "bounds"))) return rc;
    void *tmp = mem.get(scan_tmp_bytes(m));
    if (!tmp) return fail(BRM_ERR_OOM, "scan workspace");
    BRM_CUDA(cudaMemsetAsync(bs, 0, sizeof(BinStats), st));
    BinArgs a{};
    a.m = m;
    a.arp = A->row_ptr;
    a.acol = A->col_idx;
    a.brp = B->row_ptr;
    a.reg_keys = kRegKeysDefault;
    a.warp_cap = kWarpCap;
    a.block_cap = kBlockCap;
    a.block_lcap = kBlockLCap;
    a.nprod = nprod;
    a.st = bs;
    {
        PhaseScope ps(kPhBin, st);
        if (m > 0) BRM_CUDA(launch_bin(a, st));
        BRM_CUDA(launch_scan(nprod, excl, m, tmp, st));
        BRM_CUDA(launch_row_split(excl, m, parts, db, st));
    }
    BRM_CUDA(cudaMemcpyAsync(bounds, db, ((size_t)parts + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    for (int32_t p = 1; p <= parts; ++p) bounds[p] = std::max(bounds[p], bounds[p - 1]);
    g_trace.flush();
    return BRM_OK;
}

static const char *kPhaseNames[kNumPhases] = {
    "validate", "bin", "symbolic_reg", "symbolic_warp", "symbolic_block", "symbolic_long", "scan",
    "numeric_reg", "numeric_warp", "numeric_block", "numeric_long", "compact", "backward", "symbolic_tile",
    "numeric_tile"};

int brm_trace_enable(int on) {
    const int was = g_trace.on ? 1 : 0;
    g_trace.on = on != 0;
    return was;
}

void brm_trace_reset(void) {
    g_trace.flush();
    std::lock_guard<std::mutex> lk(g_trace.mu);
    for (int i = 0; i < kNumPhases; ++i) {
        g_trace.ms[i] = 0.0;
        g_trace.launches[i] = 0;
    }
}

int brm_trace_read(double *ms, int64_t *launches, int n) {
    g_trace.flush();
    std::lock_guard<std::mutex> lk(g_trace.mu);
    for (int i = 0; i < n && i < kNumPhases; ++i) {
        if (ms) ms[i] = g_trace.ms[i];
        if (launches) launches[i] = g_trace.launches[i];
    }
    return kNumPhases;
}

const char *brm_trace_phase_name(int i) { return (i >= 0 && i < kNumPhases) ? kPhaseNames[i] : ""; }

int64_t brm_kernel_launches(void) { return (int64_t)g_launches.load(); }

}  // extern "C"

extern "C" {

int brm_batch_create(int32_t count, const brm_csr *A, const brm_csr *B, const brm_options *opts,
                     const brm_allocator *alloc, void *stream, brm_batch **out) {
    g_err.clear();
    const int rc = batch_create(count, A, B, opts, alloc, static_cast<cudaStream_t>(stream), out);
    g_trace.flush();
    return rc;
}

int brm_batch_numeric(brm_batch *b, void *stream) {
    g_err.clear();
    if (!b) return fail(BRM_ERR_INVALID, "batch is NULL");
    const int rc = batch_numeric(b, static_cast<cudaStream_t>(stream), true);
    g_trace.flush();
    return rc;
}

int brm_batch_graph_launch(brm_batch *b, void *stream) {
    g_err.clear();
    if (!b) return fail(BRM_ERR_INVALID, "batch is NULL");
    return batch_graph_launch(b, static_cast<cudaStream_t>(stream));
}

int brm_batch_check(brm_batch *b, void *stream) {
    g_err.clear();
    if (!b) return fail(BRM_ERR_INVALID, "batch is NULL");
    return batch_check(b, static_cast<cudaStream_t>(stream));
}

int brm_batch_result(const brm_batch *b, brm_csr_out *C, int64_t *row_offset) {
    g_err.clear();
    if (!b) return fail(BRM_ERR_INVALID, "batch is NULL");
    batch_result(b, C, row_offset);
    return BRM_OK;
}

int brm_batch_take(brm_batch *b, brm_csr_out *C, int64_t *row_offset) {
    g_err.clear();
    if (!b) return fail(BRM_ERR_INVALID, "batch is NULL");
    if (b->taken) return fail(BRM_ERR_INVALID, "the result was already taken");
    batch_result(b, C, row_offset);
    b->taken = true;
    return BRM_OK;
}

void brm_batch_destroy(brm_batch *b) { delete b; }

int brm_autotune(int32_t count, const brm_csr *A, const brm_csr *B, const brm_options *base, brm_options *best,
                 double *best_ms, const brm_allocator *alloc, void *stream) {
    g_err.clear();
    if (!best) return fail(BRM_ERR_INVALID, "best is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const brm_options b0 = resolve(base);
    // wall time of create + numeric + check, the best of two runs after one
    auto measure = [&](const brm_options &o, double &ms) -> int {
        ms = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            BRM_CUDA(cudaStreamSynchronize(st));
            const auto t0 = std::chrono::steady_clock::now();
            brm_batch *b = nullptr;
            int rc = batch_create(count, A, B, &o, alloc, st, &b);
            if (!rc) rc = batch_numeric(b, st, false);
            if (!rc) rc = batch_check(b, st);
            const auto t1 = std::chrono::steady_clock::now();
            delete b;
            if (rc) return rc;
            if (rep > 0) ms = std::min(ms, std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        return BRM_OK;
    };
    double top = 1e300;
    brm_options win = b0;
    auto consider = [&](brm_options o) -> int {
        o = resolve(&o);
        double ms;
        const int rc = measure(o, ms);
        if (rc) return rc;
        if (ms < top) {
            top = ms;
            win = o;
        }
        return BRM_OK;
    };
    // 1. the register bins' shape: keys per thread x warps per block
    static const int kKeys[] = {8, 16, 32};
    static const int kWarps[] = {2, 4, 8};
    for (int keys : kKeys)
        for (int warps : kWarps) {
            brm_options o = b0;
            o.reg_keys = keys;
            o.reg_warps = warps;
            o.reg_max_nprod = 0;   // the full register range of this shape
            int rc = consider(o);
            if (rc) return rc;
        }
    // 2. the bin thresholds, one at a time from the best so far: how far the
    // register bins reach, the top register bin, the warp and block bins' sizes
    {
        const brm_options w = win;
        const int full = kRegMaxTpr * w.reg_keys;
        for (int cap : {full / 2, full / 4}) {
            brm_options o = w;
            o.reg_max_nprod = cap;
            int rc = consider(o);
            if (rc) return rc;
        }
    }
    {
        brm_options o = win;
        o.reg_top = o.reg_top ? 0 : 1;
        int rc = consider(o);
        if (rc) return rc;
    }
    {
        const brm_options w = win;
        for (int wcap : {128, 64}) {
            brm_options o = w;
            o.warp_max_nprod = wcap;
            int rc = consider(o);
            if (rc) return rc;
        }
    }
    {
        const brm_options w = win;
        for (int bcap : {2048, 1024}) {
            brm_options o = w;
            o.block_max_nprod = bcap;
            int rc = consider(o);
            if (rc) return rc;
        }
    }
    *best = win;
    if (best_ms) *best_ms = top;
    return BRM_OK;
}

int brm_spgemm_batched(int32_t count, const brm_csr *A, const brm_csr *B, brm_csr_out *C, int64_t *row_offset,
                       const brm_options *opts, const brm_allocator *alloc, void *stream) {
    g_err.clear();
    if (!C) return fail(BRM_ERR_INVALID, "C is NULL");
    std::memset(C, 0, sizeof *C);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    brm_batch *b = nullptr;
    int rc = batch_create(count, A, B, opts, alloc, st, &b);
    if (!rc) rc = batch_numeric(b, st, true);
    if (!rc) rc = batch_check(b, st);
    if (!rc) {
        batch_result(b, C, row_offset);
        b->taken = true;
    }
    delete b;
    g_trace.flush();
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Numeric phase without any device allocation.
//
// Some callers may not allocate device memory at all: a host application that
// has handed the whole GPU to its own memory pool, a real-time loop in which
// the implicit synchronisation of cudaMalloc/cudaFree is not acceptable, or a
// plug-in that runs inside someone else's process and may only touch the
// buffers it was given.  For them the numeric pass of BRMerge-Precise is
// offered with its workspace (the binning statistics, the per-bin row lists
// and the row-length flag) in the fixed array below instead of in allocated
// memory.  The array lives in every GPU that loads the library until the
// process exits; host code must not use its name as a device address and
// gets the address through cudaGetSymbolAddress once per device.
// ---------------------------------------------------------------------------
namespace brm {
namespace {

constexpr int64_t kNoallocMaxRows = int64_t(1) << 20;
constexpr size_t kNoallocHeader = 512;                      // BinStats, then the flag at 256
// header, then one bin byte per row, then the rows of all bins (int32 each)
constexpr size_t kNoallocBytes = kNoallocHeader + (1 + sizeof(int32_t)) * (size_t)kNoallocMaxRows;
static_assert(sizeof(BinStats) <= 256, "statistics must fit the first 256 bytes");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device, with that device current).
int noalloc_scratch(unsigned char **out) {
    int dev = 0;
    BRM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(BRM_ERR_INVALID, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        BRM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return BRM_OK;
}

int numeric_noalloc(const brm_csr *A, const brm_csr *B, const int64_t *C_row_ptr, int32_t *C_col, void *C_val,
                    const brm_options *opts, cudaStream_t st) {
    int rc = check_pair(A, B, true);
    if (rc) return rc;
    if (A->rows > kNoallocMaxRows)
        return fail(BRM_ERR_OVERFLOW, "A has %lld rows; brm_spgemm_numeric_noalloc handles at most %lld",
                    (long long)A->rows, (long long)kNoallocMaxRows);
    if (!C_row_ptr) return fail(BRM_ERR_INVALID, "C_row_ptr is NULL");
    const brm_options o = resolve(opts);
    const int64_t m = A->rows;
    unsigned char *scr = nullptr;
    if ((rc = noalloc_scratch(&scr))) return rc;
    BinStats *stats = reinterpret_cast<BinStats *>(scr);
    unsigned int *err = reinterpret_cast<unsigned int *>(scr + 256);
    uint8_t *bin_of = scr + kNoallocHeader;
    int32_t *rows = reinterpret_cast<int32_t *>(scr + kNoallocHeader + kNoallocMaxRows);
    // the array keeps the previous call's contents: zero what is accumulated
    BRM_CUDA(cudaMemsetAsync(scr, 0, kNoallocHeader, st));
    BinStats h{};
    if (o.validate) {
        BRM_CUDA(launch_validate(A->rows, A->cols, A->nnz, A->row_ptr, A->col_idx, stats, st));
        BRM_CUDA(launch_validate(B->rows, B->cols, B->nnz, B->row_ptr, B->col_idx, stats, st));
        BRM_CUDA(cudaMemcpyAsync(&h, stats, sizeof h, cudaMemcpyDeviceToHost, st));
        BRM_CUDA(cudaStreamSynchronize(st));
        if (h.bad) return fail(BRM_ERR_INVALID, "malformed CSR input (row_ptr or column order/range)");
    }
    if (m == 0) return BRM_OK;
    BinArgs a{};
    a.m = m;
    a.arp = A->row_ptr;
    a.acol = A->col_idx;
    a.brp = B->row_ptr;
    a.reg_max_tpr = reg_max_tpr(o, B->cols);
    a.reg_keys = o.reg_keys;
    a.reg_top = reg_top_ok(o, B->cols);
    a.warp_cap = o.warp_max_nprod;
    a.block_cap = o.block_max_nprod;
    a.block_lcap = kBlockLCap;
    a.bin_of = bin_of;
    a.st = stats;
    a.rows = rows;
    a.out_rp = C_row_ptr;
    a.out_err = err;
    BRM_CUDA(launch_bin(a, st));
    BRM_CUDA(cudaMemcpyAsync(&h, stats, sizeof h, cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    if (h.count[kBinLong] > 0)
        return fail(BRM_ERR_OVERFLOW,
                    "%llu rows have more than %d products or %d lists; brm_spgemm_numeric_noalloc only merges rows "
                    "that fit in shared memory",
                    h.count[kBinLong], o.block_max_nprod, kBlockLCap);
    int64_t off = 0;
    for (int b = 0; b < kNumBins; ++b) {
        a.base[b] = off;
        if (b != kBinEmpty) off += (int64_t)h.count[b];
    }
    BRM_CUDA(launch_bin_scatter(a, st));
    RowJob j = base_job(src_of(A, B), o);
    j.out_rp = C_row_ptr;
    j.out_col = C_col;
    j.out_val = C_val;
    j.err = err;
    j.exact = 1;
    const VKind v = value_kind(A->dtype, o);
    for (int b = kBinReg0; b <= kBinBlock; ++b) {
        RowJob jb = j;
        jb.rows = rows + a.base[b];
        jb.count = (int32_t)h.count[b];
        if (jb.count == 0) continue;
        BRM_CUDA(launch_rows(v, b, jb, st));
    }
    unsigned int flag = 0;
    BRM_CUDA(cudaMemcpyAsync(&flag, err, sizeof flag, cudaMemcpyDeviceToHost, st));
    BRM_CUDA(cudaStreamSynchronize(st));
    if (flag) return fail(BRM_ERR_INVALID, "a row's length disagrees with its slot in C_row_ptr");
    return BRM_OK;
}

}  // namespace
}  // namespace brm

extern "C" int brm_spgemm_numeric_noalloc(const brm_csr *A, const brm_csr *B, const int64_t *C_row_ptr,
                                          int32_t *C_col_idx, void *C_val, const brm_options *opts, void *stream) {
    brm::g_err.clear();
    return brm::numeric_noalloc(A, B, C_row_ptr, C_col_idx, C_val, opts, static_cast<cudaStream_t>(stream));
}
