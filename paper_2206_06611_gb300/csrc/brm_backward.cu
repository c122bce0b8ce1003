// Gradients of a scalar loss through C = A * B (the differentiable form).
//
// With G = dLoss/dC given on C's pattern,
//   dA_ik = sum over j in B_k* of G_ij * B_kj      (k in A_i*: (G * B^T) on A's pattern)
//   dB_kj = sum over i with k in A_i* of A_ik * G_ij   ((A^T * G) on B's pattern).
// Row i of C holds every column of every B_k*, k in A_i* (C keeps structural
// entries, Eq. 2 summed over the union of the B rows), so each G_ij is found
// by a search in the sorted columns of C_i*.
//
// One warp per row i of A; each lane takes whole lists k of the row in turn,
// so dA_ik is a sequential, deterministic sum over B_k* in column order.  The
// columns of B_k* ascend, so each search starts where the previous one ended.
// dB gathers contributions from many rows and is accumulated with atomics.
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

template <class V>
__global__ void __launch_bounds__(256) k_backward(BackwardArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const V *aval = static_cast<const V *>(a.aval);
    const V *bval = static_cast<const V *>(a.bval);
    const V *g = static_cast<const V *>(a.dC);
    V *da = static_cast<V *>(a.dA);
    V *db = static_cast<V *>(a.dB);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < a.m; i += nw) {
        const int64_t c0 = a.crp[i], c1 = a.crp[i + 1];
        const int p1 = a.arp[i + 1];
        for (int p = a.arp[i] + lane; p < p1; p += 32) {
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
}

}  // namespace

cudaError_t launch_backward(const BackwardArgs &a, bool f64, cudaStream_t st) {
    if (a.m <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int T = 256;
    const int64_t want = (a.m + (T / 32) - 1) / (T / 32);
    const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    if (f64) k_backward<double><<<grid, T, 0, st>>>(a);
    else k_backward<float><<<grid, T, 0, st>>>(a);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace brm
