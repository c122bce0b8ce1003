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
// over the rows.  That needs, for every column k of A, its entries in row
// order (A^T's rows): they are bucketed by column (a count, a prefix sum and
// an atomic scatter of the entry indices), and every bucket is then sorted --
// an entry index grows with the row, so sorting the indices orders the rows.
// A bucket of at most 1024 entries is sorted by one warp in registers, a
// longer one by a thread block in device memory.
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
// indices as keys of the register bitonic network (32 lanes x 32 keys).
__global__ void __launch_bounds__(256) k_bwd_sort_small(const int64_t *colptr, int64_t ncols, int32_t *ent) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < ncols; k += warps) {
        const int64_t b = colptr[k], n = colptr[k + 1] - b;
        if (n < 2 || n > 1024) continue;
        uint32_t key[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int64_t q = (int64_t)i * 32 + lane;
            key[i] = q < n ? (uint32_t)ent[b + q] : kKeyPad;
        }
        reg_bitonic_sort<32, 32>(key, lane);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int64_t q = (int64_t)lane * 32 + i;
            if (q < n) ent[b + q] = (int32_t)key[i];
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

// dB_kj: one thread per entry q = (k, j) of B, the terms A_ik * G_ij summed
// over the bucket of column k in order (rows increasing), from zero.
template <class V>
__global__ void __launch_bounds__(256) k_bwd_db(BackwardArgs a, const int64_t *colptr, const int32_t *ent,
                                                const int32_t *row_of, int64_t nnz_b) {
    const V *aval = static_cast<const V *>(a.aval);
    const V *g = static_cast<const V *>(a.dC);
    V *db = static_cast<V *>(a.dB);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz_b;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = row_of_entry(a.brp, a.kb, q);
        const int32_t j = __ldg(a.bcol + q);
        V acc = V(0);
        for (int64_t e = colptr[k]; e < colptr[k + 1]; ++e) {
            const int32_t p = ent[e];
            const int32_t i = row_of[p];
            const int64_t c0 = a.crp[i], c1 = a.crp[i + 1];
            const int64_t w = lower_bound_col(a.ccol, c0, c1, j);
            if (w >= c1 || __ldg(a.ccol + w) != j) {
                atomicOr(a.err, 1u);   // C's pattern is not the one of A * B
                break;
            }
            acc += __ldg(aval + p) * __ldg(g + w);
        }
        db[q] = acc;
    }
}

template <class V>
__global__ void __launch_bounds__(256) k_backward(BackwardArgs a) {
    const V *bval = static_cast<const V *>(a.bval);
    const V *g = static_cast<const V *>(a.dC);
    V *da = static_cast<V *>(a.dA);
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
    if (a.dA) {
        if (f64) k_backward<double><<<grid_for(a.nnz_a), T, 0, st>>>(a);
        else k_backward<float><<<grid_for(a.nnz_a), T, 0, st>>>(a);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.dB && a.nnz_b > 0) {
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
        if (f64) k_bwd_db<double><<<grid_for(a.nnz_b), T, 0, st>>>(a, a.ws_colptr, a.ws_ent, a.ws_row, a.nnz_b);
        else k_bwd_db<float><<<grid_for(a.nnz_b), T, 0, st>>>(a, a.ws_colptr, a.ws_ent, a.ws_row, a.nnz_b);
        g_launches.fetch_add(6, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace brm
