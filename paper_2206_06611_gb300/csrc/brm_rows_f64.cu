// Row kernels instantiated for double values.
#include "brm_rows.cuh"

namespace brm {
cudaError_t launch_rows_f64(int bin, const RowJob &j, cudaStream_t st) { return launch_rows_t<PF64>(bin, j, st); }
size_t long_bytes_f64(int64_t n, int64_t L, bool bucket) { return long_bytes_t<PF64>(n, L, bucket); }
int tile_grid_f64() { return tile_grid_t<PF64>(); }
}  // namespace brm
