// Solution transfer on the cubed sphere (Sec. 3.4, spherical geometry;
// Appendix B): dg_sphere_geometry and dg_sphere_transfer of include/dg.h.
//
// The sphere is six equiangular gnomonic tiles laid side by side in one 2D forest of 6n x n
// roots (tile t = root column / n).  Every element is an isoparametric quadrilateral: its
// surface is the degree-N interpolant of the sphere points at its LGL nodes.
//  * geometry (one CTA per element): the node points, the tangent vectors x_xi, x_eta from the
//    collocation derivative of the node points, the surface Jacobian J = |x_xi x x_eta| (the
//    2D measure behind App. B's pseudo-inverse), the nodal weights W = w_i w_j J, and the
//    element area as the spherical excess r^2 (A + B + C - pi) of the two spherical triangles
//    of its corners (great-circle edges: the areas of children add up to their parent's);
//  * transfer (one CTA per event of the regrid map): a kept element is copied; the four
//    children of a refined parent take the reference interpolation P_c and then one factor per
//    field, uniform over the four, that makes the field's integral (sum W q) equal the
//    parent's; a coarsened parent takes sum_c (4 V_c / sum V) R_c q_c, the reference
//    restriction R_c weighted by the children's spherical-excess areas V_c, and the same
//    integral-matching factor.  A factor is applied only when the new integral is not the
//    residue of cancellation (|I_new| > 1e-8 sum W |q|).
// One set of reference projections serves every element, as the section proposes; the scale
// factors repair the conservation that per-element projections would give.
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "basis.hpp"

namespace {

constexpr int kSphMaxN1 = 9;
constexpr int kSphMaxNV = 8;

struct SphereOps {
  int n1, ntile;
  double radius;
  double x[kSphMaxN1], w[kSphMaxN1];
  double D[kSphMaxN1 * kSphMaxN1];
  double P[2][kSphMaxN1 * kSphMaxN1], C[2][kSphMaxN1 * kSphMaxN1];
};

// Unit point of tile t at equiangular coordinates (a, b).
__device__ void sph_unit_point(int t, double a, double b, double* p) {
  const double X = tan(a), Y = tan(b);
  double v[3];
  switch (t) {
    case 0: v[0] = 1.0; v[1] = X; v[2] = Y; break;
    case 1: v[0] = -X; v[1] = 1.0; v[2] = Y; break;
    case 2: v[0] = -1.0; v[1] = -X; v[2] = Y; break;
    case 3: v[0] = X; v[1] = -1.0; v[2] = Y; break;
    case 4: v[0] = -Y; v[1] = X; v[2] = 1.0; break;
    default: v[0] = Y; v[1] = X; v[2] = -1.0; break;
  }
  const double s = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  p[0] = v[0] / s; p[1] = v[1] / s; p[2] = v[2] / s;
}

__device__ void sph_cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ double sph_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Internal angle at unit vertex p of the spherical triangle p q1 q2: the angle between the
// great circles p-q1 and p-q2, from their tangent vectors at p.
__device__ double sph_angle(const double* p, const double* q1, const double* q2) {
  const double d1 = sph_dot(p, q1), d2 = sph_dot(p, q2);
  double t1[3], t2[3], c[3];
  for (int k = 0; k < 3; ++k) { t1[k] = q1[k] - d1 * p[k]; t2[k] = q2[k] - d2 * p[k]; }
  sph_cross(t1, t2, c);
  return atan2(sqrt(sph_dot(c, c)), sph_dot(t1, t2));
}

__device__ double sph_excess(const double* a, const double* b, const double* c) {
  return sph_angle(a, b, c) + sph_angle(b, c, a) + sph_angle(c, a, b) - M_PI;
}

// Equiangular coordinate along a layout axis of the node at reference coordinate z of an element
// with anchor c at level lev: root units u = (c + (z + 1)/2) / 2^lev, minus the tile offset.
__device__ double sph_coord(int c, int lev, double z, double offset, int n) {
  const double u = ((double)c + (z + 1.0) / 2.0) / ldexp(1.0, lev) - offset;
  return -M_PI / 4.0 + (M_PI / 2.0) * u / (double)n;
}

// One CTA per element: node points, J, W = w_i w_j J, and the spherical-excess area.
__global__ void sphere_geometry_kernel(const __grid_constant__ SphereOps O, int64_t E, const int32_t* leaves,
                                       double* W, double* area) {
  const int n1 = O.n1, NP = n1 * n1;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  __shared__ double sx[kSphMaxN1 * kSphMaxN1][3];
  const int32_t* lf = leaves + e * 5;
  const int lev = lf[1], cx = lf[2], cy = lf[3];
  const int n = O.ntile;
  const int t = (cx >> lev) / n;
  const double off = (double)(t * n);
  for (int k = threadIdx.x; k < NP; k += blockDim.x) {
    const int i = k % n1, j = k / n1;
    double p[3];
    sph_unit_point(t, sph_coord(cx, lev, O.x[i], off, n), sph_coord(cy, lev, O.x[j], 0.0, n), p);
    for (int d = 0; d < 3; ++d) sx[k][d] = O.radius * p[d];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NP; k += blockDim.x) {
    const int i = k % n1, j = k / n1;
    double xa[3] = {0.0, 0.0, 0.0}, xb[3] = {0.0, 0.0, 0.0}, c[3];
    for (int m = 0; m < n1; ++m)
      for (int d = 0; d < 3; ++d) {
        xa[d] += O.D[i * n1 + m] * sx[m + n1 * j][d];
        xb[d] += O.D[j * n1 + m] * sx[i + n1 * m][d];
      }
    sph_cross(xa, xb, c);
    W[e * NP + k] = (O.w[j] * O.w[i]) * sqrt(sph_dot(c, c));
  }
  if (threadIdx.x == 0) {
    double p[4][3];
    const double z[4][2] = {{-1.0, -1.0}, {1.0, -1.0}, {1.0, 1.0}, {-1.0, 1.0}};
    for (int q = 0; q < 4; ++q)
      sph_unit_point(t, sph_coord(cx, lev, z[q][0], off, n), sph_coord(cy, lev, z[q][1], 0.0, n), p[q]);
    area[e] = O.radius * O.radius * (sph_excess(p[0], p[1], p[2]) + sph_excess(p[0], p[2], p[3]));
  }
}

// 1D operator M (n1 x n1) along axis `axis` (0: xi, i fastest; 1: eta) of nv planes of NP
// values: out[v][node] = sum_m M[row][m] in[v][node with m on that axis].
__device__ void sph_apply_1d(const double* M, int axis, int n1, int nv, const double* in, double* out) {
  const int NP = n1 * n1;
  for (int x = threadIdx.x; x < nv * NP; x += blockDim.x) {
    const int v = x / NP, k = x - v * NP;
    const int i = k % n1, j = k / n1;
    double s = 0.0;
    if (axis == 0) for (int m = 0; m < n1; ++m) s += M[i * n1 + m] * in[v * NP + m + n1 * j];
    else           for (int m = 0; m < n1; ++m) s += M[j * n1 + m] * in[v * NP + i + n1 * m];
    out[x] = s;
  }
}

// Events: {0, k, old} keep; {1, k0, parent} the children k0 .. k0 + 3 of an old parent (child
// indices 0..3); {2, k, c0, c1, c2, c3} a new parent of four old children.
__global__ void sphere_transfer_kernel(const __grid_constant__ SphereOps O, int nv, const int32_t* ev,
                                       int64_t nev, const double* W_old, const double* area_old,
                                       const double* q_old, int64_t plane_old, const double* W_new,
                                       double* q_new, int64_t plane_new) {
  const int n1 = O.n1, NP = n1 * n1;
  const int64_t id = blockIdx.x;
  if (id >= nev) return;
  extern __shared__ double smem[];
  double* A = smem;                    // [4][nv][NP]
  double* B = A + 4 * nv * NP;         // [4][nv][NP]
  __shared__ double s_scale[kSphMaxNV], s_wgt[4];
  const int32_t* r = ev + id * 6;
  const int kind = r[0];
  const int64_t k = r[1];
  if (kind == 0) {
    const int64_t e = r[2];
    for (int x = threadIdx.x; x < nv * NP; x += blockDim.x) {
      const int v = x / NP, n = x - v * NP;
      q_new[v * plane_new + k * NP + n] = q_old[v * plane_old + e * NP + n];
    }
    return;
  }
  const int nin = kind == 1 ? 1 : 4;
  const int nout = kind == 1 ? 4 : 1;
  for (int x = threadIdx.x; x < nin * nv * NP; x += blockDim.x) {
    const int c = x / (nv * NP), rem = x - c * nv * NP;
    const int v = rem / NP, n = rem - v * NP;
    const int64_t e = r[2 + c];
    A[x] = q_old[v * plane_old + e * NP + n];
  }
  __syncthreads();
  // integral of each field over the old element(s), before A is overwritten
  double I_old = 0.0;
  if (threadIdx.x < nv) {
    const int v = threadIdx.x;
    for (int c = 0; c < nin; ++c) {
      const int64_t e = r[2 + c];
      for (int n = 0; n < NP; ++n) I_old += W_old[e * NP + n] * A[(c * nv + v) * NP + n];
    }
  }
  if (kind == 2 && threadIdx.x == 0) {
    double V = 0.0;
    for (int c = 0; c < 4; ++c) V += area_old[r[2 + c]];
    for (int c = 0; c < 4; ++c) s_wgt[c] = 4.0 * area_old[r[2 + c]] / V;
  }
  if (kind == 1) {
    // children c = 0..3: P_{c_0} along xi, then P_{c_1} along eta, of the parent
    for (int c = 0; c < 4; ++c) sph_apply_1d(O.P[c & 1], 0, n1, nv, A, B + c * nv * NP);
    __syncthreads();
    for (int c = 0; c < 4; ++c) sph_apply_1d(O.P[(c >> 1) & 1], 1, n1, nv, B + c * nv * NP, A + c * nv * NP);
  } else {
    for (int c = 0; c < 4; ++c) sph_apply_1d(O.C[c & 1], 0, n1, nv, A + c * nv * NP, B + c * nv * NP);
    __syncthreads();
    for (int c = 0; c < 4; ++c) sph_apply_1d(O.C[(c >> 1) & 1], 1, n1, nv, B + c * nv * NP, A + c * nv * NP);
    __syncthreads();
    for (int x = threadIdx.x; x < nv * NP; x += blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < 4; ++c) acc = acc + s_wgt[c] * A[c * nv * NP + x];
      B[x] = acc;
    }
  }
  __syncthreads();
  const double* R = kind == 1 ? A : B;    // the new element(s): [nout][nv][NP]
  if (threadIdx.x < nv) {
    const int v = threadIdx.x;
    double I_new = 0.0, mag = 0.0;
    for (int c = 0; c < nout; ++c)
      for (int n = 0; n < NP; ++n) {
        const double wq = W_new[(k + c) * NP + n];
        I_new += wq * R[(c * nv + v) * NP + n];
        mag += wq * fabs(R[(c * nv + v) * NP + n]);
      }
    s_scale[v] = fabs(I_new) > 1e-8 * mag ? I_old / I_new : 1.0;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < nout * nv * NP; x += blockDim.x) {
    const int c = x / (nv * NP), rem = x - c * nv * NP;
    const int v = rem / NP, n = rem - v * NP;
    q_new[v * plane_new + (k + c) * NP + n] = R[x] * s_scale[v];
  }
}

SphereOps make_ops(int N, int n, double radius) {
  SphereOps O{};
  const dgl::Basis1D b = dgl::make_basis(N);
  O.n1 = N + 1;
  O.ntile = n;
  O.radius = radius;
  for (int i = 0; i < O.n1; ++i) { O.x[i] = b.x[i]; O.w[i] = b.w[i]; }
  for (int i = 0; i < O.n1 * O.n1; ++i) {
    O.D[i] = b.D[i];
    for (int c = 0; c < 2; ++c) { O.P[c][i] = b.P[c][i]; O.C[c][i] = b.C[c][i]; }
  }
  return O;
}

dg_status cuda_status(cudaError_t e) {
  return e == cudaSuccess ? DG_OK : (e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA);
}

}  // namespace

extern "C" {

dg_status dg_sphere_geometry(int32_t N, int32_t n, double radius, const int32_t* leaves, int64_t E,
                             double* W, double* area, void* stream) {
  if (N < 1 || N > DG_MAX_N || n < 1 || !(radius > 0.0) || E < 0 || (E > 0 && (!leaves || !W || !area)))
    return DG_ERR_ARG;
  if (E == 0) return DG_OK;
  const SphereOps O = make_ops(N, n, radius);
  sphere_geometry_kernel<<<(unsigned)E, 128, 0, (cudaStream_t)stream>>>(O, E, leaves, W, area);
  return cuda_status(cudaGetLastError());
}

dg_status dg_sphere_transfer(int32_t N, int32_t n, int32_t nv, const int32_t* tmap, int64_t E_new,
                             const double* W_old, const double* area_old, const double* q_old,
                             int64_t E_old, const double* W_new, double* q_new, void* stream) {
  if (N < 1 || N > DG_MAX_N || n < 1 || nv < 1 || nv > kSphMaxNV || E_new < 0 || E_old < 0 ||
      (E_new > 0 && (!tmap || !W_old || !area_old || !q_old || !W_new || !q_new)))
    return DG_ERR_ARG;
  if (E_new == 0) return DG_OK;
  // events of the regrid map, every index checked before upload
  std::vector<int32_t> ev;
  ev.reserve((size_t)E_new * 6);
  for (int64_t k = 0; k < E_new; ++k) {
    const int32_t* r = tmap + k * 9;
    if (r[0] == 0) {
      if (r[1] < 0 || r[1] >= E_old) return DG_ERR_ARG;
      ev.insert(ev.end(), {0, (int32_t)k, r[1], -1, -1, -1});
    } else if (r[0] == 1) {
      if (r[2] != 0) continue;   // the family is the event of its first child
      if (k + 3 >= E_new || r[1] < 0 || r[1] >= E_old) return DG_ERR_ARG;
      for (int c = 1; c < 4; ++c) {
        const int32_t* s = tmap + (k + c) * 9;
        if (s[0] != 1 || s[1] != r[1] || s[2] != c) return DG_ERR_ARG;
      }
      ev.insert(ev.end(), {1, (int32_t)k, r[1], -1, -1, -1});
    } else if (r[0] == 2) {
      for (int c = 0; c < 4; ++c)
        if (r[1 + c] < 0 || r[1 + c] >= E_old) return DG_ERR_ARG;
      ev.insert(ev.end(), {2, (int32_t)k, r[1], r[2], r[3], r[4]});
    } else {
      return DG_ERR_ARG;
    }
  }
  const SphereOps O = make_ops(N, n, 1.0);
  const int64_t nev = (int64_t)(ev.size() / 6);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* d_ev = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_ev, ev.size() * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(d_ev, ev.data(), ev.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  const int NP = (N + 1) * (N + 1);
  const size_t smem = sizeof(double) * 8 * (size_t)nv * NP;
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(sphere_transfer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    sphere_transfer_kernel<<<(unsigned)nev, 256, smem, s>>>(O, nv, d_ev, nev, W_old, area_old, q_old,
                                                          E_old * NP, W_new, q_new, E_new * NP);
    e = cudaGetLastError();
  }
  // the host copy of the events must outlive the asynchronous upload
  const cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFreeAsync(d_ev, s);
  return cuda_status(e != cudaSuccess ? e : e2);
}

}  // extern "C"
