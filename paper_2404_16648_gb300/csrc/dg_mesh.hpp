// Internal definition of the dg_mesh handle, shared by the C ABI units (dg_api.cu, dg_batch.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "basis.hpp"
#include "dg_launch.hpp"
#include "tree.hpp"

struct dg_mesh {
  dg_mesh_desc desc{};
  int D = 2, N = 1, n1 = 2, NP = 4, NV = 4, NSUB = 2, NF = 2;
  int prec = 0;
  size_t tsize = 8;
  cudaStream_t stream = nullptr;
  dgl::Forest forest;
  dgl::Basis1D basis;
  dgk::PhysC ph{};
  double root_h[3] = {1, 1, 1};
  int64_t E = 0, G = 0, cap = 0;
  std::vector<int32_t> conf, mort, bnd;
  // device buffers; every size-dependent one grows only (capacity in bytes, with headroom), so a
  // regrid that keeps the mesh near its size allocates nothing
  void* q[3] = {nullptr, nullptr, nullptr};
  size_t q_cap[3] = {0, 0, 0};
  void* q_spare = nullptr;     // receives the transferred state at the next regrid
  size_t q_spare_cap = 0;
  int64_t generation = 0;      // incremented by every dg_adapt
  size_t c_elem = 0, c_conn = 0, c_groups = 0, c_bg = 0, c_mbuf = 0, c_bgf = 0, c_bgc = 0, c_pps = 0;
  size_t c_sigma = 0, c_V = 0, c_vbuf = 0, c_tm = 0, c_ind = 0;
  int32_t* d_tm = nullptr;     // transfer map of the last regrid
  // pinned host staging of a regrid's uploads (transfer map; tables) and of its indicator
  // read-back: asynchronous copies at the link's rate instead of pageable synchronous ones
  unsigned char* h_pin[3] = {nullptr, nullptr, nullptr};
  size_t c_pin[3] = {0, 0, 0};
  double* d_ind = nullptr;     // refinement indicator
  int32_t* d_elem = nullptr;
  int32_t* d_conn = nullptr;
  int32_t* d_groups = nullptr;
  double* d_bg = nullptr;
  float* d_bgf = nullptr;      // FP32 copy of the background (FP32 path)
  double* d_bgc = nullptr;     // gamma p_bar / Theta_bar per z-level (FP32 path's P')
  void* d_mbuf = nullptr;
  void* d_fbuf = nullptr;      // layout 5: conforming and wall face fluxes (dg_face.cuh)
  int32_t* d_fconf = nullptr;  // the conforming and boundary face lists on the device
  int32_t* d_fbnd = nullptr;
  size_t c_fbuf = 0, c_fconf = 0, c_fbnd = 0;
  void* d_ppscratch = nullptr; // P' plane of a caller's state in dg_rhs
  bool pp_valid = false;       // P' plane of q[0] matches q[0]
  int variant = 2;             // stage kernel layout (DG_OPT_STAGE_KERNEL); set at creation
  int fail_next_adapt = 0;     // DG_OPT_FAIL_NEXT_ADAPT: host-side failure injection for tests
  bool broken = false;         // a regrid failed after its commit: every later call is refused
  // SFC partition (dg_set_partition): stage launches cover elements e_begin .. e_end - 1 of the
  // replicated tree; the face traces of the other elements arrive through the halo functions.
  // Slot lists are rows {element, axis, side}; send slots grouped by destination part, receive
  // slots by source part (offsets per part, nparts + 1 entries each).
  int nparts = 1, part = 0;
  int64_t e_begin = 0, e_end = 0;
  std::vector<int64_t> send_off, recv_off;
  int32_t* d_send = nullptr;
  int32_t* d_recv = nullptr;
  int32_t* d_glist = nullptr;  // mortar groups touching the part's elements
  size_t c_send = 0, c_recv = 0, c_glist = 0;
  int64_t G_part = 0;
  bool tracer = false;         // DG_EQ_TRACER: one passive tracer plane, prescribed wind
  double time = 0.0;           // model time of the state (dg_set_time, advanced by dg_step)
  double stage_g = 1.0;        // tracer wind factor cos(pi t / T) of the stage being launched
  // adjoint / pure-step workspace, allocated on first use for the current mesh size
  void* adj_q[3] = {nullptr, nullptr, nullptr};   // states with P' planes
  double* adj_l[2] = {nullptr, nullptr};          // cotangents
  double* d_abuf = nullptr;                       // mortar adjoint contributions
  int64_t adj_E = -1, adj_G = -1;
  // viscous term (nu > 0, FP64): gradients, tendency, mortar values
  double* d_sigma = nullptr;
  double* d_V = nullptr;
  double* d_vbuf = nullptr;
  void* d_ops = nullptr;       // precision T
  double* d_opsd = nullptr;    // FP64: D, P0, P1, C0, C1, w, x
  double* d_partial = nullptr;
  double* d_out = nullptr;
  double bgint[6] = {0, 0, 0, 0, 0, 0};   // background sums of the integrals (see dg_integrals)
  double* d_bgint = nullptr;   // the same on the device, and the combined results (12 doubles)
  bool bgint_valid = false;
  int* d_bad = nullptr;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  cudaEvent_t ev_order = nullptr;   // orders a caller's stream after the mesh stream
  std::string err;
};


namespace dgi {

int64_t plane(const dg_mesh* m);
void* pp_plane(const dg_mesh* m, void* q);
// Arguments of one fused stage launch on mesh m (mode 1: Shu-Osher combination).
void fill_stage_args(const dg_mesh* m, const void* qs, const void* pp_in, const void* qn, void* out,
                     void* pp_out, int mode, double dt, double ca, double cb, dgk::StageArgs* A);
// Arguments of the mortar work of mesh m for stage input qs.
void fill_mortar_args(const dg_mesh* m, const void* qs, const void* pp_in, dgk::MortarArgs* M);
// Arguments of the face kernel of mesh m (stage layout 5) for stage input qs.
void fill_face_args(const dg_mesh* m, const void* qs, const void* pp_in, dgk::FaceArgs* F);
// Sizes the face buffer of layout 5 for the mesh's conforming and boundary faces.
dg_status ensure_face_buffer(dg_mesh* m);
// Launches the mortar kernel of mesh m for stage input qs (no-op without hanging faces).
dg_status launch_mortars(dg_mesh* m, const void* qs, const void* pp_in, cudaStream_t s);
// Makes the P' plane of m->q[0] current.
dg_status ensure_pp(dg_mesh* m, cudaStream_t s);
dg_status set_error(dg_mesh* m, dg_status st, const char* msg);

}  // namespace dgi
