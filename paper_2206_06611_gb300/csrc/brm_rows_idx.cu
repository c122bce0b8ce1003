// Row kernels instantiated for column indices only (the symbolic pass).
#include "brm_rows.cuh"

namespace brm {
cudaError_t launch_rows_idx(int bin, const RowJob &j, cudaStream_t st) { return launch_rows_t<PIdx>(bin, j, st); }
size_t long_bytes_idx(int64_t n, int64_t L, bool bucket) { return long_bytes_t<PIdx>(n, L, bucket); }
}  // namespace brm
