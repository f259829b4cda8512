// Stage and mortar kernels, float state, 3D.
#include "stage_inst.cuh"

namespace dgk {
bool launch_stage_f32_3d(int N, const StageArgs& A, cudaStream_t s) {
  return stage_dispatch<float, 3>(N, A, s);
}
bool launch_mortar_f32_3d(int N, const MortarArgs& A, cudaStream_t s) {
  return mortar_dispatch<float, 3>(N, A, s);
}
cudaError_t init_stage_f32_3d(const double* dtab_all) {
  const cudaError_t e = upload_dtab(dtab_all);
  return e != cudaSuccess ? e : upload_dtab_fb(dtab_all);
}
cudaError_t launch_stage_batched_f32_3d(int N, int layout, const StageArgs* tab, const int2* map,
                                        int nblocks, cudaStream_t s) {
  return batched_dispatch<float, 3>(N, layout, tab, map, nblocks, s);
}
cudaError_t launch_face_f32_3d(int N, const FaceArgs& F, bool pdl, cudaStream_t s) {
  return face_dispatch<float, 3>(N, F, pdl, s);
}
}  // namespace dgk
