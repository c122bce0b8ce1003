// Gradients of a scalar loss through C = A * B (the differentiable form).
//
// With G = dLoss/dC given on C's pattern,
//   dA_ik = sum over j in B_k* of G_ij * B_kj      (k in A_i*: (G * B^T) on A's pattern)
//   dB_kj = sum over i with k in A_i* of A_ik * G_ij   ((A^T * G) on B's pattern).
// Row i of C holds every column of every B_k*, k in A_i* (C keeps structural
// entries, Eq. 2 summed over the union of the B rows), so each G_ij is found
// by a search in the sorted columns of C_i*.
//
// One thread per stored entry (i, k) of A, so that long and short rows of A
// spread evenly over the GPU: the thread finds its row i by a binary search
// in A's row pointer, then walks B_k* in column order; dA_ik is a
// sequential, deterministic sum over B_k*.  The columns of B_k* ascend, so
// each search in C_i* starts where the previous one ended.  dB gathers
// contributions from many entries and is accumulated with atomics.
#include <cstdint>
#include <cuda_runtime.h>

#include "brm_internal.h"

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

template <class V>
__global__ void __launch_bounds__(256) k_backward(BackwardArgs a) {
    const V *aval = static_cast<const V *>(a.aval);
    const V *bval = static_cast<const V *>(a.bval);
    const V *g = static_cast<const V *>(a.dC);
    V *da = static_cast<V *>(a.dA);
    V *db = static_cast<V *>(a.dB);
    const int64_t nnz = a.nnz_a;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row_of_entry(a.arp, a.m, p);
        const int64_t c0 = a.crp[i], c1 = a.crp[i + 1];
        const int k = a.acol[p];
        const V aik = aval[p];
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
            if (db) atomicAdd(db + q, aik * gij);
            ++lo;
        }
        if (da) da[p] = acc;
    }
}

}  // namespace

cudaError_t launch_backward(const BackwardArgs &a, bool f64, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (a.nnz_a <= 0) return cudaSuccess;
    const int T = 256;
    const int64_t want = (a.nnz_a + T - 1) / T;
    const int grid = (int)(want < (int64_t)sms * 32 ? want : (int64_t)sms * 32);
    if (f64) k_backward<double><<<grid, T, 0, st>>>(a);
    else k_backward<float><<<grid, T, 0, st>>>(a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace brm
