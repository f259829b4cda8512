// Internal launch interface between the C ABI (dg_api.cu) and the kernel translation units.
#pragma once
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include <cuda_runtime.h>

#include "dg_adjoint.cuh"
#include "dg_device.cuh"
#include "dg_face.cuh"
#include "dg_tracer.cuh"
#include "dg_viscous.cuh"

namespace dgk {

constexpr int NUM_INTEGRALS = 5;

// Function attributes (dynamic shared-memory limit, carveout) belong to a device's context: a
// kernel is configured once per (kernel, device), under a mutex, so concurrent host threads and
// a second GPU in the same process each see a configured kernel.  Shared by every stage unit
// (an inline function's statics are one object across translation units).
inline cudaError_t configure_kernel(const void* fn, size_t smem, bool max_carveout) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && max_carveout)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  done.insert({fn, dev});
  return cudaSuccess;
}

// Tracer meshes (tracer_f64.cu): stage, hanging faces (mortar or point interpolation), initial
// bell, indicator max |C| and the compensated totals {int C, volume} into out[0..1].
bool launch_tracer_stage(int N, const TracerArgs& A, cudaStream_t s);
bool launch_tracer_mortar(int N, const TracerMortarArgs& A, cudaStream_t s);
cudaError_t launch_tracer_bell(int32_t E, int n1, const int32_t* elem, const double* xi,
                               const double* root_h, const double* center, const double* radius,
                               double amp, double* C, cudaStream_t s);
cudaError_t launch_tracer_indicator(int32_t E, int n1, const double* C, double* out, cudaStream_t s);
size_t tracer_total_scratch_doubles();
cudaError_t launch_tracer_total(int32_t E, int n1, const int32_t* elem, const double* w,
                                const double* root_h, const double* C, double* partial, int* bad,
                                double* out, cudaStream_t s);

// Fused RK stage (or pure RHS) and mortar launches; return false when (D, N) is not compiled.
bool launch_stage_f64_2d(int N, const StageArgs& A, cudaStream_t s);
bool launch_stage_f64_3d(int N, const StageArgs& A, cudaStream_t s);
bool launch_stage_f32_2d(int N, const StageArgs& A, cudaStream_t s);
bool launch_stage_f32_3d(int N, const StageArgs& A, cudaStream_t s);
bool launch_mortar_f64_2d(int N, const MortarArgs& A, cudaStream_t s);
bool launch_mortar_f64_3d(int N, const MortarArgs& A, cudaStream_t s);
bool launch_mortar_f32_2d(int N, const MortarArgs& A, cudaStream_t s);
bool launch_mortar_f32_3d(int N, const MortarArgs& A, cudaStream_t s);
// Face kernel of stage layout 5 (conforming and wall fluxes into the face buffer); pdl: as the
// programmatic dependent of the mortar kernel launched just before.
cudaError_t launch_face_f64_2d(int N, const FaceArgs& F, bool pdl, cudaStream_t s);
cudaError_t launch_face_f64_3d(int N, const FaceArgs& F, bool pdl, cudaStream_t s);
cudaError_t launch_face_f32_2d(int N, const FaceArgs& F, bool pdl, cudaStream_t s);
cudaError_t launch_face_f32_3d(int N, const FaceArgs& F, bool pdl, cudaStream_t s);
// Upload the derivative matrices of every degree (concatenated, N = 1..8) to each unit's
// constant memory; called once before the first stage launch.
cudaError_t init_stage_f64_2d(const double* dtab_all);
cudaError_t init_stage_f64_3d(const double* dtab_all);
cudaError_t init_stage_f32_2d(const double* dtab_all);
cudaError_t init_stage_f32_3d(const double* dtab_all);
// Persistent batched stage kernel over the 2D members of a batch (dg_batch_persist.cuh), in two
// register budgets: "w" for 2 resident CTAs of 128 threads per SM, "d" for 4.
struct BatchArgs;
cudaError_t init_stage_batch_w(const double* dtab_all);
cudaError_t init_stage_batch_d(const double* dtab_all);
cudaError_t launch_batch_w(const BatchArgs& B, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_d(const BatchArgs& B, int grid, size_t smem, cudaStream_t s);
cudaError_t occupancy_batch_w(size_t smem, int* ctas_per_sm);
cudaError_t occupancy_batch_d(size_t smem, int* ctas_per_sm);
// Largest dynamic shared memory of the persistent kernel's bodies for one (precision, N, layout)
// (layout 0 node, 1 column-async, 2 mortar).
size_t batch_body_smem_bytes(int prec32, int N, int layout);

// Stage kernels over many meshes at once (tab: per-mesh arguments on the device, map: per block
// the mesh index and its first element); layout 1 node-per-thread, 2 column with async staging.
cudaError_t launch_stage_batched_f64_2d(int N, int layout, const StageArgs* tab, const int2* map, int nblocks, cudaStream_t s);
cudaError_t launch_stage_batched_f64_3d(int N, int layout, const StageArgs* tab, const int2* map, int nblocks, cudaStream_t s);
cudaError_t launch_stage_batched_f32_2d(int N, int layout, const StageArgs* tab, const int2* map, int nblocks, cudaStream_t s);
cudaError_t launch_stage_batched_f32_3d(int N, int layout, const StageArgs* tab, const int2* map, int nblocks, cudaStream_t s);

cudaError_t launch_background(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                              double root_hz, const PhysC& ph, double* bg, float* bgf,
                              double* bgc, cudaStream_t s);
cudaError_t launch_pprime(int prec, int32_t E, int n1, int D, const void* theta_plane,
                          const double* bg, const double* bgc, const PhysC& ph, void* pp, cudaStream_t s);
cudaError_t launch_vortex(int prec, int32_t E, int n1, const int32_t* elem, const double* xi,
                          const double* root_h, const double* length, const int* periodic,
                          const double* center, double beta, const double* uinf, double t,
                          double gamma, const double* bg, void* q, int64_t plane, cudaStream_t s);
cudaError_t launch_bubble(int prec, int32_t E, int n1, int D, const int32_t* elem,
                          const double* xi, const double* root_h, const double* bg,
                          const double* center, const double* radius, double amp, int n_rff,
                          double rff_scale, const double* rff_k, const double* rff_phase,
                          double theta0, void* q, int64_t plane, double* theta_out,
                          cudaStream_t s);
cudaError_t launch_indicator(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                             int64_t plane, double theta0, double* out, cudaStream_t s);
// State layout conversion between element-major [E][NV][NP] and the mesh's planes
// [NV][plane] (to_planes = 1: into planes); tsize 4 or 8 bytes per value.
cudaError_t launch_state_layout(int tsize, int to_planes, int64_t E, int NP, int NV, const void* src,
                                void* dst, int64_t plane, cudaStream_t s);
// tag[e] = (the theta' indicator of element e > thr), as 0 / 1 bytes.
cudaError_t launch_tags(int prec, int32_t E, int n1, int D, const double* bg, const void* q, int64_t plane,
                        double theta0, double thr, uint8_t* tag, cudaStream_t s);
cudaError_t launch_primitives(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                              int64_t plane, double theta0, double* out, cudaStream_t s);
size_t integrals_scratch_doubles();
// Three compensated sums (see dg_misc.cu) into out[0..2], their rounding errors into out[3..5]:
// background = true: int rho_bar, int (p_bar cv/R + rho_bar g z), volume;
// background = false: int rho', int (P' cv/R + |U|^2/(2 rho) + rho' g z), int |U|^2/(2 rho).
cudaError_t launch_integrals(int prec, bool background, int32_t E, int n1, int D, const int32_t* elem,
                             const double* xi, const double* w, const double* root_h,
                             const double* bg, const void* q, int64_t plane, const PhysC& ph,
                             double* partial, int* bad, double* out, cudaStream_t s);
// Halo traces of a sharded mesh (dg_halo_pack / dg_halo_unpack): slot rows {element, axis,
// side}; pp may be null (its plane is then packed as zeros and not unpacked).
cudaError_t launch_halo(int prec, int unpack, int64_t slots, int n1, int D, int NV, const int32_t* rows,
                        void* q, void* pp, int64_t plane, void* buf, cudaStream_t s);
// res[0..5] = {mass, energy, kinetic energy, volume, perturbation mass, non-finite flag} from the
// state sums S[6] and background sums B[6] (the combination of dg_integrals, on the device).
cudaError_t launch_integrals_combine(const double* S, const double* B, const int* bad, double* res, cudaStream_t s);
cudaError_t launch_transfer(int prec, int32_t Enew, int n1, int D, int nv, const int32_t* tmap,
                            const double* ops, const void* qold, int64_t plane_old, void* qnew,
                            int64_t plane_new, cudaStream_t s);

// BR1 viscous term (FP64): pass 1 writes sigma, pass 2 writes V (mortar values included).
bool launch_viscous_pass(int D, int N, const ViscArgs& A, int pass, cudaStream_t s);
cudaError_t launch_visc_add(int32_t E, int n1, int D, const double* V, double coef, double* out,
                            int64_t plane, const double* bg, const PhysC& ph, double* pp,
                            cudaStream_t s);

// Adjoint (FP64): right-hand-side vector-Jacobian products and their helpers.
// false: (D, N) not compiled; err: the kernel configuration's error, if any
bool launch_vjp(int D, int N, const AdjArgs& A, cudaStream_t s, cudaError_t& err);
bool launch_mortar_vjp(int D, int N, const MortarAdjArgs& A, cudaStream_t s);
cudaError_t launch_theta_state(int prec, int32_t E, int n1, int D, const double* bg,
                               const double* theta, double theta0, void* q, int64_t plane,
                               cudaStream_t s);
cudaError_t launch_theta_vjp(int32_t E, int n1, int D, const double* bg, const double* theta,
                             double theta0, const double* lam_q, double* lam_theta, cudaStream_t s);
cudaError_t launch_ke_grad(int32_t E, int n1, int D, const int32_t* elem, const double* w,
                          const double* root_h, const double* bg, const double* q, int64_t plane,
                          double* out, cudaStream_t s);

}  // namespace dgk
