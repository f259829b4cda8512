// Face kernel of stage layout 5: the Rusanov flux F* (Sec. 2.2) of every conforming face and
// every wall face, once per face, into a face buffer that the stage kernel then reads like the
// mortar fluxes of hanging faces (Sec. 3.3).  The layouts that evaluate F* inside the stage
// kernel do it once from each side of a conforming face (both sides' fluxes and wave speeds,
// the sound speed's square root included); on the FP64 path, bound by its FP64 pipe, doing it
// once per face saves that work at the cost of a buffer the stage kernel reads back.
//
// The arithmetic is the stage kernels' (node_der, flux_axis, wave_speed, face_side, rusanov,
// the low side's background for both sides, which is the high side's bit for bit), so F* has
// the bits the in-kernel evaluation gives.  Face slots: conforming faces 0 .. C-1 in the
// order of the conforming-face list (low element, high element, axis), then boundary faces
// C .. C+B-1 in the order of the boundary list (element, axis, side); thread t of a face takes
// tangential node t in the kernels' face_node order.
#pragma once
#include "dg_device.cuh"

namespace dgk {

struct FaceArgs {
  const void* qs;         // stage input state (T)
  const void* pp_in;      // its P' plane
  void* fbuf;             // [C + B][NV][NF] (T)
  int64_t plane;
  int32_t C, B;           // conforming and boundary face counts
  const int32_t* conf;    // [C][3]: low element, high element, axis
  const int32_t* bnd;     // [B][3]: element, axis, side
  const void* bgt;        // background rows [E][N+1][4] in T
  float gammaf;
  PhysC ph;
};

template <int D, int N>
__host__ __device__ constexpr int face_per_block() {
  return ipow(N + 1, D - 1) >= 256 ? 1 : 256 / ipow(N + 1, D - 1);
}

// F* of face slot `slot` at its tangential node t, to the face buffer.
template <class T, int D, int N>
__device__ __forceinline__ void face_flux_node(const FaceArgs& A, int64_t slot, int t) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  const T* qs = (const T*)A.qs;
  const T* ppl = (const T*)A.pp_in;
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  T Fs[NV];
  if (slot < A.C) {
    const int32_t* r = A.conf + slot * 3;
    const int64_t el = r[0], eh = r[1];
    const int a = r[2];
    const int nm = face_node<D, N>(a, 1, t), np = face_node<D, N>(a, 0, t);
    const int k = (D == 3) ? nm / (n1 * n1) : nm / n1;
    const T* b = (const T*)A.bgt + ((size_t)el * n1 + k) * 4;
    const NodeBg<T> bg{b[0], b[1], b[2]};
    T qm[NV], qp[NV], Fm[NV], Fp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qm[v] = qs[(size_t)v * A.plane + (size_t)el * NP + nm];
      qp[v] = qs[(size_t)v * A.plane + (size_t)eh * NP + np];
    }
    const T sm = face_side<T, D>(qm, bg, ppl[(size_t)el * NP + nm], a, gamma, Fm);
    const T sp = face_side<T, D>(qp, bg, ppl[(size_t)eh * NP + np], a, gamma, Fp);
    rusanov<T, D>(qm, Fm, sm, qp, Fp, sp, Fs);
  } else {
    const int32_t* r = A.bnd + (slot - A.C) * 3;
    const int64_t e = r[0];
    const int a = r[1], s = r[2];
    const int n = face_node<D, N>(a, s, t);
    const int k = (D == 3) ? n / (n1 * n1) : n / n1;
    const T* b = (const T*)A.bgt + ((size_t)e * n1 + k) * 4;
    const NodeBg<T> bg{b[0], b[1], b[2]};
    T q[NV], qo[NV], Fo[NV], Fn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = qs[(size_t)v * A.plane + (size_t)e * NP + n];
    const T pp = ppl[(size_t)e * NP + n];
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    flux_axis<T, D>(q, nd, pp, a, Fo);
    const T so = wave_speed<T>(q, nd, bg, pp, a, gamma);
    // no-flux wall as a mirror state: same Theta, rho and P', normal momentum negated
#pragma unroll
    for (int v = 0; v < NV; ++v) qo[v] = q[v];
    qo[1 + a] = -q[1 + a];
    flux_axis<T, D>(qo, nd, pp, a, Fn);
    if (s) rusanov<T, D>(q, Fo, so, qo, Fn, so, Fs);
    else   rusanov<T, D>(qo, Fn, so, q, Fo, so, Fs);
  }
  T* dst = (T*)A.fbuf + (size_t)slot * NV * NF;
#pragma unroll
  for (int v = 0; v < NV; ++v) dst[v * NF + t] = Fs[v];
}

template <class T, int D, int N>
__global__ void __launch_bounds__(256) face_kernel(const __grid_constant__ FaceArgs A) {
  constexpr int NF = ipow(N + 1, D - 1);
  constexpr int FPB = face_per_block<D, N>();
  const int lf = threadIdx.x / NF, t = threadIdx.x - lf * NF;
  const int64_t slot = (int64_t)blockIdx.x * FPB + lf;
  if (lf < FPB && slot < (int64_t)A.C + A.B) face_flux_node<T, D, N>(A, slot, t);
  // the stage kernel launched after this grid may start once every CTA of this grid has got
  // here (its prologue then overlaps this grid's last wave); it waits for this grid's
  // completion before it reads the face buffer.  Signalled at the start instead, the stage
  // kernel's CTAs would fill the SMs while most of this grid still had to run.
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  // launched as the programmatic dependent of this stage's mortar kernel, this grid completes
  // only after it, so the stage kernel's wait for this grid covers the mortar fluxes too
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

}  // namespace dgk
