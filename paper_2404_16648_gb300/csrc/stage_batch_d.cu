// Persistent batched stage kernel (dg_batch_persist.cuh) with the register budget of 4 resident
// CTAs of 128 threads per SM (at most 128 registers a thread).
#include "dg_batch_persist.cuh"
#include "dg_launch.hpp"

namespace dgk {
cudaError_t init_stage_batch_d(const double* dtab_all) {
  const cudaError_t e = upload_dtab(dtab_all);
  return e != cudaSuccess ? e : upload_dtab_fb(dtab_all);
}
cudaError_t launch_batch_d(const BatchArgs& B, int grid, size_t smem, cudaStream_t s) {
  return launch_batch<4>(B, grid, smem, s);
}
cudaError_t occupancy_batch_d(size_t smem, int* ctas_per_sm) { return occupancy_batch<4>(smem, ctas_per_sm); }
}  // namespace dgk
