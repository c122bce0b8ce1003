// Gradients of a scalar loss through C = A * B (the differentiable form).
//
// With G = dLoss/dC given on C's pattern,
//   dA_ik = sum over j in B_k* of G_ij * B_kj      (k in A_i*: (G * B^T) on A's pattern)
//   dB_kj = sum over i with k in A_i* of A_ik * G_ij   ((A^T * G) on B's pattern).
// Row i of C holds every column of every B_k*, k in A_i* (C keeps structural
// entries, Eq. 2 summed over the union of the B rows), so each G_ij is found
// by a search in the sorted columns of C_i*.
//
// dA: one thread per stored entry (i, k) of A, so that long and short rows of
// A spread evenly over the GPU: the thread finds its row i by a binary search
// in A's row pointer, then walks B_k* in column order; dA_ik is a sequential
// sum over B_k*.  The columns of B_k* ascend, so each search in C_i* starts
// where the previous one ended.
// dB: every entry of B sums its terms over the rows i in increasing order,
// sequentially, so the result is deterministic and the same as a plain loop
// over the rows.  The dA pass stores every product's G_ij on the way (at the
// product's place in A's entry order), so a term is two loads.  That needs, for every column k of A, its entries in row
// order (A^T's rows): they are bucketed by column (a count, a prefix sum and
// an atomic scatter of the entry indices), and every bucket is then sorted --
// an entry index grows with the row, so sorting the indices orders the rows.
// A bucket of at most 1024 entries is sorted by one warp in registers, a
// longer one by a thread block in device memory.  An entry of B sums its
// bucket alone when the bucket is short, with a warp forming 32 terms at a
// time when it is long.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "brm_internal.h"
#include "brm_reg_rows.cuh"

namespace brm {
namespace {

// First position in [lo, hi) whose column is >= c.
__device__ __forceinline__ int64_t lower_bound_col(const int32_t *__restrict__ col, int64_t lo, int64_t hi,
                                                   int32_t c) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(col + mid) < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Row of entry p: the last i with arp[i] <= p (arp non-decreasing, arp[0] = 0).
__device__ __forceinline__ int64_t row_of_entry(const int32_t *__restrict__ arp, int64_t m, int64_t p) {
    int64_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(arp + mid) <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Products of every entry of A: plen[p] = |B_k*| for its column k.
__global__ void __launch_bounds__(256) k_bwd_plen(BackwardArgs a, int64_t *plen) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.nnz_a;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int k = a.acol[p];
        plen[p] = a.brp[k + 1] - a.brp[k];
    }
}

// Bucket sizes: cnt[k] = entries of A in column k; row_of[p] = the row of entry p.
__global__ void __launch_bounds__(256) k_bwd_count(BackwardArgs a, unsigned long long *cnt, int32_t *row_of) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.nnz_a;
         p += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(cnt + a.acol[p], 1ull);
        row_of[p] = (int32_t)row_of_entry(a.arp, a.m, p);
    }
}

// Entry indices into their column's bucket (any order inside a bucket).
__global__ void __launch_bounds__(256) k_bwd_scatter(BackwardArgs a, unsigned long long *cursor, int32_t *ent) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.nnz_a;
         p += (int64_t)gridDim.x * blockDim.x)
        ent[atomicAdd(cursor + a.acol[p], 1ull)] = (int32_t)p;
}

// Sorts every bucket of at most 1024 entries, one warp per bucket: the
// indices as keys of a bitonic network sized to the bucket (one key per lane
// up to 32 entries, else the register network of 32 lanes x 8, 16 or 32
// keys).
template <int E>
__device__ __forceinline__ void bwd_sort_warp(int32_t *e, int64_t n, int lane) {
    uint32_t key[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int64_t q = (int64_t)i * 32 + lane;
        key[i] = q < n ? (uint32_t)e[q] : kKeyPad;
    }
    reg_bitonic_sort<32, E>(key, lane);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int64_t q = (int64_t)lane * E + i;
        if (q < n) e[q] = (int32_t)key[i];
    }
}

__global__ void __launch_bounds__(256) k_bwd_sort_small(const int64_t *colptr, int64_t ncols, int32_t *ent) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < ncols; k += warps) {
        const int64_t b = colptr[k], n = colptr[k + 1] - b;
        if (n < 2 || n > 1024) continue;
        if (n <= 32) {
            // one key per lane: lane x ends with the x-th smallest
            uint32_t key = lane < n ? (uint32_t)ent[b + lane] : kKeyPad;
#pragma unroll
            for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
                for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                    const uint32_t o = __shfl_xor_sync(kFull, key, jj);
                    const bool up = (lane & kk) == 0, low = (lane & jj) == 0;
                    key = (up == low) ? min(key, o) : max(key, o);
                }
            }
            if (lane < n) ent[b + lane] = (int32_t)key;
        } else if (n <= 256) {
            bwd_sort_warp<8>(ent + b, n, lane);
        } else if (n <= 512) {
            bwd_sort_warp<16>(ent + b, n, lane);
        } else {
            bwd_sort_warp<32>(ent + b, n, lane);
        }
    }
}

// Sorts every bucket of more than 1024 entries, one thread block per bucket,
// in device memory: the all-ascending bitonic network over the next power of
// two, positions past the end standing for +infinity (a comparison with one
// of them leaves the real key where it is).
__global__ void __launch_bounds__(1024) k_bwd_sort_big(const int64_t *colptr, int64_t ncols, int32_t *ent) {
    for (int64_t k = blockIdx.x; k < ncols; k += gridDim.x) {
        const int64_t b = colptr[k], n = colptr[k + 1] - b;
        if (n <= 1024) continue;
        int32_t *e = ent + b;
        int64_t np2 = 1;
        while (np2 < n) np2 <<= 1;
        for (int64_t kk = 2; kk <= np2; kk <<= 1) {
            for (int64_t jj = kk >> 1; jj >= 1; jj >>= 1) {
                // the first step of each size is the flip x <-> x ^ (kk - 1)
                const int64_t msk = jj == (kk >> 1) ? kk - 1 : jj;
                for (int64_t x = threadIdx.x; x < np2; x += blockDim.x) {
                    const int64_t y = x ^ msk;
                    if (y > x && y < n) {
                        const int32_t u = e[x], v = e[y];
                        if (u > v) {
                            e[x] = v;
                            e[y] = u;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
}

// Buckets longer than this are summed by the warps of a block per row of B.
constexpr int64_t kBwdWarpCol = 64;

// The term A_ik * G_ij of bucket entry p (an entry (i, k) of A) for the jj-th
// entry of B_k*: G_ij was stored per product by the dA pass.
template <class V>
__device__ __forceinline__ V bwd_term(const BackwardArgs &a, int32_t p, int jj) {
    return __ldg(static_cast<const V *>(a.aval) + p) * static_cast<const V *>(a.ws_gp)[a.ws_poff[p] + jj];
}

// dB_kj: one thread per entry q = (k, j) of B whose bucket (column k of A)
// has at most kBwdWarpCol entries, the terms A_ik * G_ij summed over the
// bucket in order (rows increasing), from zero.
template <class V>
__global__ void __launch_bounds__(256) k_bwd_db(BackwardArgs a, const int64_t *colptr, const int32_t *ent) {
    V *db = static_cast<V *>(a.dB);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.nnz_b;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = row_of_entry(a.brp, a.kb, q);
        const int64_t e0 = colptr[k], e1 = colptr[k + 1];
        if (e1 - e0 > kBwdWarpCol) continue;
        const int jj = (int)(q - a.brp[k]);
        V acc = V(0);
        for (int64_t e = e0; e < e1; ++e) acc += bwd_term<V>(a, ent[e], jj);
        db[q] = acc;
    }
}

// dB for the rows k of B whose bucket has more than kBwdWarpCol entries: one
// thread block per row, its warps taking the row's entries in turn; for an
// entry the lanes form 32 terms at a time and every lane adds them in bucket
// order, so the sum is the same sequential sum as above.
template <class V>
__global__ void __launch_bounds__(256) k_bwd_db_warp(BackwardArgs a, const int64_t *colptr, const int32_t *ent) {
    constexpr unsigned kFull = 0xffffffffu;
    V *db = static_cast<V *>(a.dB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t k = blockIdx.x; k < a.kb; k += gridDim.x) {
        const int64_t e0 = colptr[k], e1 = colptr[k + 1];
        if (e1 - e0 <= kBwdWarpCol) continue;
        const int q0 = a.brp[k], q1 = a.brp[k + 1];
        for (int q = q0 + wid; q < q1; q += nw) {
            const int jj = q - q0;
            V acc = V(0);
            for (int64_t eb = e0; eb < e1; eb += 32) {
                const int64_t e = eb + lane;
                const V t = e < e1 ? bwd_term<V>(a, ent[e], jj) : V(0);
                const int n = (int)min((int64_t)32, e1 - eb);
                for (int l = 0; l < n; ++l) acc += __shfl_sync(kFull, t, l);
            }
            if (lane == 0) db[q] = acc;
        }
    }
}

template <class V>
__global__ void __launch_bounds__(256) k_backward(BackwardArgs a) {
    const V *bval = static_cast<const V *>(a.bval);
    const V *g = static_cast<const V *>(a.dC);
    V *da = static_cast<V *>(a.dA);
    V *gp = static_cast<V *>(a.ws_gp);
    const int64_t nnz = a.nnz_a;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row_of_entry(a.arp, a.m, p);
        const int64_t c0 = a.crp[i], c1 = a.crp[i + 1];
        const int k = a.acol[p];
        V acc = V(0);
        int64_t lo = c0;
        for (int q = a.brp[k]; q < a.brp[k + 1]; ++q) {
            const int32_t j = __ldg(a.bcol + q);
            lo = lower_bound_col(a.ccol, lo, c1, j);
            if (lo >= c1 || __ldg(a.ccol + lo) != j) {
                atomicOr(a.err, 1u);   // C's pattern is not the one of A * B
                break;
            }
            const V gij = __ldg(g + lo);
            acc += gij * __ldg(bval + q);
            if (gp) gp[a.ws_poff[p] + (q - a.brp[k])] = gij;
            ++lo;
        }
        if (da) da[p] = acc;
    }
}

}  // namespace

cudaError_t launch_backward(const BackwardArgs &a, bool f64, cudaStream_t st) {
    if (a.m <= 0 || a.nnz_a <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int T = 256;
    auto grid_for = [&](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + T - 1) / T, (int64_t)sms * 32)); };
    cudaError_t e;
    const bool want_db = a.dB && a.nnz_b > 0;
    if (want_db) {
        // where every entry of A keeps the G_ij of its products
        k_bwd_plen<<<grid_for(a.nnz_a), T, 0, st>>>(a, a.ws_plen);
        if ((e = launch_scan(a.ws_plen, a.ws_poff, a.nnz_a, a.ws_scan2, st)) != cudaSuccess) return e;
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    if (a.dA || want_db) {
        if (f64) k_backward<double><<<grid_for(a.nnz_a), T, 0, st>>>(a);
        else k_backward<float><<<grid_for(a.nnz_a), T, 0, st>>>(a);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (want_db) {
        // A^T's rows: bucket sizes, their prefix sum, scatter, sort
        if ((e = cudaMemsetAsync(a.ws_cnt, 0, (size_t)a.ka * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        k_bwd_count<<<grid_for(a.nnz_a), T, 0, st>>>(a, reinterpret_cast<unsigned long long *>(a.ws_cnt), a.ws_row);
        if ((e = launch_scan(a.ws_cnt, a.ws_colptr, a.ka, a.ws_scan, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(a.ws_cnt, a.ws_colptr, (size_t)a.ka * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                 st)) != cudaSuccess)
            return e;
        k_bwd_scatter<<<grid_for(a.nnz_a), T, 0, st>>>(a, reinterpret_cast<unsigned long long *>(a.ws_cnt), a.ws_ent);
        const int gw = (int)std::max<int64_t>(1, std::min<int64_t>((a.ka + 7) / 8, (int64_t)sms * 16));
        k_bwd_sort_small<<<gw, T, 0, st>>>(a.ws_colptr, a.ka, a.ws_ent);
        k_bwd_sort_big<<<std::max(sms, 1), 1024, 0, st>>>(a.ws_colptr, a.ka, a.ws_ent);
        if (f64) k_bwd_db<double><<<grid_for(a.nnz_b), T, 0, st>>>(a, a.ws_colptr, a.ws_ent);
        else k_bwd_db<float><<<grid_for(a.nnz_b), T, 0, st>>>(a, a.ws_colptr, a.ws_ent);
        const int gwb = (int)std::max<int64_t>(1, std::min<int64_t>(a.kb, (int64_t)sms * 8));
        if (f64) k_bwd_db_warp<double><<<gwb, T, 0, st>>>(a, a.ws_colptr, a.ws_ent);
        else k_bwd_db_warp<float><<<gwb, T, 0, st>>>(a, a.ws_colptr, a.ws_ent);
        g_launches.fetch_add(7, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace brm
