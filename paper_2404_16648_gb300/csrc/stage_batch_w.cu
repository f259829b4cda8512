// Persistent batched stage kernel (dg_batch_persist.cuh) with the register budget of 2 resident
// CTAs of 128 threads per SM (up to 255 registers a thread: no body spills).
#include "dg_batch_persist.cuh"
#include "dg_launch.hpp"

namespace dgk {
cudaError_t init_stage_batch_w(const double* dtab_all) {
  const cudaError_t e = upload_dtab(dtab_all);
  return e != cudaSuccess ? e : upload_dtab_fb(dtab_all);
}
cudaError_t launch_batch_w(const BatchArgs& B, int grid, size_t smem, cudaStream_t s) {
  return launch_batch<2>(B, grid, smem, s);
}
cudaError_t occupancy_batch_w(size_t smem, int* ctas_per_sm) { return occupancy_batch<2>(smem, ctas_per_sm); }
size_t batch_body_smem_bytes(int prec32, int N, int layout) { return batch_body_smem_any(prec32, N, layout); }
}  // namespace dgk
