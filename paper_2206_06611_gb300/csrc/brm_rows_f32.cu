// Row kernels instantiated for float values, plain and TwoSum-compensated.
#include "brm_rows.cuh"

namespace brm {
cudaError_t launch_rows_f32(int bin, const RowJob &j, cudaStream_t st) { return launch_rows_t<PF32>(bin, j, st); }
cudaError_t launch_rows_f32c(int bin, const RowJob &j, cudaStream_t st) { return launch_rows_t<PF32C>(bin, j, st); }
size_t long_bytes_f32(int64_t n, int64_t L, bool bucket) { return long_bytes_t<PF32>(n, L, bucket); }
size_t long_bytes_f32c(int64_t n, int64_t L, bool bucket) { return long_bytes_t<PF32C>(n, L, bucket); }
int tile_grid_f32() { return tile_grid_t<PF32>(); }
int tile_grid_f32c() { return tile_grid_t<PF32C>(); }
}  // namespace brm
