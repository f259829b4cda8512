// Column-mapped fused stage kernel (layout 0).
//
// Same operator as stage_kernel in dg_device.cuh (strong-form volume term, Rusanov face terms,
// precomputed mortar fluxes, Shu-Osher combination, FP64 P' epilogue), with a thread layout
// that cuts shared-memory traffic and divergence:
//  * one thread per vertical line (column) of an element: (i, j) in 3D, i in 2D; the thread
//    keeps the N+1 nodes of its column in registers, so the vertical derivative needs no shared
//    memory and reads D from constant memory (uniform across the warp);
//  * the horizontal derivatives go through shared memory, one tile per axis holding the flux
//    of all nodes; along x the D-row is contiguous and read with vector loads;
//  * face terms are evaluated face-node-major: on a horizontal-normal face, thread t takes
//    face node t (all lanes busy, no divergence) and leaves its lift in shared memory for the
//    column that owns the node; the bottom and top faces belong to every column.
// The arithmetic of each flux and Rusanov evaluation is the same explicitly rounded code as in
// dg_device.cuh, so both elements of a conforming face still compute bit-identical F*.
#pragma once
#include <cstring>
#include "dg_device.cuh"

namespace dgk {

// Offsets of the degree-N blocks in the constant D tables (N = 1..8).
__host__ __device__ constexpr int dtab_offset(int N) {
  return N <= 1 ? 0 : dtab_offset(N - 1) + N * N;
}
constexpr int kDTabSize = dtab_offset(9);   // sum_{N=1..8} (N+1)^2

// Collocation derivative matrices of every degree, per translation unit (static); filled by
// upload_dtab() of the same unit before its first launch.
static __constant__ float c_dtab_f[kDTabSize];
static __constant__ double c_dtab_d[kDTabSize];
// The antisymmetric part (D[m][i] - D[N-m][N-i]) / 2 of each matrix.  The LGL derivative is
// antisymmetric under the reflection x -> -x of the nodes, so this is D up to the rounding of the
// computed nodes; being exactly antisymmetric, it lets a kernel apply the rows of the upper half
// of a line through those of the lower half (the line layout).
static __constant__ float c_dtab_af[kDTabSize];
static __constant__ double c_dtab_ad[kDTabSize];
// The FP32 antisymmetric entries as packed FP32 pairs: c_dtab_af2[m][i] holds entry (m, i) in
// both halves; c_dtab_afr[m][i] for even m holds entries (m, i) and (m + 1, i).
static __constant__ unsigned long long c_dtab_af2[kDTabSize];
static __constant__ unsigned long long c_dtab_afr[kDTabSize];
// Even/odd split of the antisymmetric matrix A (odd N, K2 = (N+1)/2): with E_m = F_m + F_{N-m} and
// O_m = F_m - F_{N-m} (m < K2), (A F)_i = SE_i + SO_i and (A F)_{N-i} = SO_i - SE_i for i < K2,
// SE_i = sum_m Ae[i][m] E_m, SO_i = sum_m Ao[i][m] O_m, Ae = (A[i][m] + A[i][N-m]) / 2,
// Ao = (A[i][m] - A[i][N-m]) / 2.  Ae at the degree's offset, Ao K2^2 entries after it.
static __constant__ float c_dtab_eo_f[kDTabSize];
static __constant__ double c_dtab_eo_d[kDTabSize];

static inline cudaError_t upload_dtab(const double* all) {
  float f[kDTabSize];
  for (int i = 0; i < kDTabSize; ++i) f[i] = (float)all[i];
  cudaError_t e = cudaMemcpyToSymbol(c_dtab_f, f, sizeof(f));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_dtab_d, all, sizeof(double) * kDTabSize);
  if (e != cudaSuccess) return e;
  double a[kDTabSize];
  for (int N = 1; N <= 8; ++N) {
    const int o = dtab_offset(N), n1 = N + 1;
    for (int m = 0; m < n1; ++m)
      for (int i = 0; i < n1; ++i)
        a[o + m * n1 + i] = 0.5 * (all[o + m * n1 + i] - all[o + (N - m) * n1 + (N - i)]);
  }
  for (int i = 0; i < kDTabSize; ++i) f[i] = (float)a[i];
  e = cudaMemcpyToSymbol(c_dtab_af, f, sizeof(f));
  if (e != cudaSuccess) return e;
  {
    double eo[kDTabSize];
    float eof[kDTabSize];
    for (int i = 0; i < kDTabSize; ++i) eo[i] = 0.0;
    for (int N = 1; N <= 8; N += 2) {
      const int o = dtab_offset(N), n1 = N + 1, K2 = n1 / 2;
      for (int i = 0; i < K2; ++i)
        for (int m = 0; m < K2; ++m) {
          eo[o + i * K2 + m] = 0.5 * (a[o + i * n1 + m] + a[o + i * n1 + (N - m)]);
          eo[o + K2 * K2 + i * K2 + m] = 0.5 * (a[o + i * n1 + m] - a[o + i * n1 + (N - m)]);
        }
    }
    for (int i = 0; i < kDTabSize; ++i) eof[i] = (float)eo[i];
    e = cudaMemcpyToSymbol(c_dtab_eo_d, eo, sizeof(eo));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(c_dtab_eo_f, eof, sizeof(eof));
    if (e != cudaSuccess) return e;
  }
  unsigned long long f2[kDTabSize];
  for (int i = 0; i < kDTabSize; ++i) {
    uint32_t b;
    std::memcpy(&b, &f[i], sizeof b);
    f2[i] = ((unsigned long long)b << 32) | b;
  }
  e = cudaMemcpyToSymbol(c_dtab_af2, f2, sizeof(f2));
  if (e != cudaSuccess) return e;
  for (int N = 1; N <= 8; ++N) {
    const int o = dtab_offset(N), n1 = N + 1;
    for (int m = 0; m < n1; ++m)
      for (int i = 0; i < n1; ++i) {
        const unsigned long long lo = f2[o + m * n1 + i] & 0xffffffffull;
        const unsigned long long hi = (m + 1 < n1) ? (f2[o + (m + 1) * n1 + i] & 0xffffffffull) : 0ull;
        // rows are rewritten in increasing order, so rows m and m + 1 still hold the originals
        f2[o + m * n1 + i] = (hi << 32) | lo;
      }
  }
  e = cudaMemcpyToSymbol(c_dtab_afr, f2, sizeof(f2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dtab_ad, a, sizeof(double) * kDTabSize);
}

template <class T> __device__ __forceinline__ T dtab(int i);
template <> __device__ __forceinline__ float dtab<float>(int i) { return c_dtab_f[i]; }
template <> __device__ __forceinline__ double dtab<double>(int i) { return c_dtab_d[i]; }
template <class T> __device__ __forceinline__ T dtab_eo(int i);
template <> __device__ __forceinline__ float dtab_eo<float>(int i) { return c_dtab_eo_f[i]; }
template <> __device__ __forceinline__ double dtab_eo<double>(int i) { return c_dtab_eo_d[i]; }
template <class T> __device__ __forceinline__ T dtab_anti(int i);
template <> __device__ __forceinline__ float dtab_anti<float>(int i) { return c_dtab_af[i]; }
template <> __device__ __forceinline__ double dtab_anti<double>(int i) { return c_dtab_ad[i]; }

// Dynamic shared memory of the column kernel per CTA (bytes).
template <class T, int D, int N, int EPB>
__host__ __device__ constexpr size_t col_smem_bytes() {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NV = D + 2, NT = D - 1;
  constexpr int QT = (n1 + 1) * ((D == 3) ? n1 : 1) * n1;
  return sizeof(T) * ((size_t)EPB * NT * NV * NP + (size_t)EPB * (NV + 1) * QT +
                      (size_t)EPB * n1 * 3 + (size_t)n1 * n1);
}

template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D - 1))
stage_kernel_col(const __grid_constant__ StageArgs A) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  constexpr int NT = D - 1;                 // horizontal axes
  constexpr int P1 = n1 + 1;                // padded row of the state tile
  constexpr int JS = (D == 3) ? n1 : 1;
  constexpr int QT = P1 * JS * n1;          // padded state tile per variable
  constexpr bool VEC = (sizeof(T) == 4) && (n1 % 4 == 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // horizontal fluxes: tile 0 in node order (x lines contiguous), tile 1 (3D) transposed so that
  // y lines are contiguous; reused for the face lifts.  Then the state and P' tile, background, D.
  T (*sFh)[NT][NV][NP] = reinterpret_cast<T (*)[NT][NV][NP]>(smem_raw);
  T (*sQ)[NV + 1][QT] = reinterpret_cast<T (*)[NV + 1][QT]>(smem_raw + sizeof(T) * EPB * NT * NV * NP);
  T (*sBg)[n1][3] = reinterpret_cast<T (*)[n1][3]>(smem_raw + sizeof(T) * (EPB * NT * NV * NP + EPB * (NV + 1) * QT));
  T* sDh = reinterpret_cast<T*>(smem_raw + sizeof(T) * (EPB * NT * NV * NP + EPB * (NV + 1) * QT + EPB * n1 * 3));
  const int tid = threadIdx.x;
  const int le = tid / NF, t = tid - le * NF;
  const int64_t e = (int64_t)A.e_begin + (int64_t)blockIdx.x * EPB + le;
  const bool valid = e < A.E;
  const int ci = t % n1, cj = (D == 3) ? t / n1 : 0;
  const T* ops = (const T*)A.ops;
  for (int x = tid; x < n1 * n1; x += blockDim.x) sDh[x] = ops[x];
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  const T g = sizeof(T) == 4 ? (T)A.gf : (T)A.ph.g;
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + (valid ? e : 0) * NP;
  const T* ppe = (const T*)A.pp_in + (valid ? e : 0) * NP;
  T acc[NV][n1];
  T inv2h[D];
  int level = 0;
  if (valid) {
    level = A.elem[e * 4];
    if (t < n1) {
      const T* b = (const T*)A.bgt + ((size_t)e * n1 + t) * 4;
      sBg[le][t][0] = b[0]; sBg[le][t][1] = b[1]; sBg[le][t][2] = b[2];
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) inv2h[a] = valid ? inv2h_of<T>(A, level, a) : (T)0;
  __syncthreads();
  // ---- load the column; horizontal fluxes to shared memory, the vertical one kept here
  T Fz[NV][n1];
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    const int n = t + NF * k;
    T q[NV];
    T pp = (T)0;
    NodeBg<T> bg{(T)1, (T)1, (T)1};
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = qe[v * P + n];
      pp = ppe[n];
      bg = NodeBg<T>{sBg[le][k][0], sBg[le][k][1], sBg[le][k][2]};
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = (T)0;
    }
    const int qi = ci + P1 * (cj + JS * k);
#pragma unroll
    for (int v = 0; v < NV; ++v) sQ[le][v][qi] = q[v];
    sQ[le][NV][qi] = pp;
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v][k] = (T)0;
    acc[D][k] = -(q[0] * g);               // buoyancy -rho' g on the vertical momentum
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    T F[NV];
    flux_axis<T, D>(q, nd, pp, 0, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) sFh[le][0][v][n] = F[v];
    if (D == 3) {
      flux_axis<T, D>(q, nd, pp, 1, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) sFh[le][NT - 1][v][NF * k + n1 * ci + cj] = F[v];
    }
    flux_axis<T, D>(q, nd, pp, D - 1, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fz[v][k] = F[v];
  }
  // ---- vertical derivative from registers, D from constant memory
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      T s = (T)0;
#pragma unroll
      for (int m = 0; m < n1; ++m) s = fma(dtab<T>(dtab_offset(N) + k * n1 + m), Fz[v][m], s);
      acc[v][k] = fma(-inv2h[D - 1], s, acc[v][k]);
    }
  __syncthreads();
  // ---- horizontal derivatives through shared memory (contiguous lines, vector loads)
  auto line_dot = [&](const T* row, const T* Dr) {
    T s = (T)0;
    if constexpr (VEC) {
#pragma unroll
      for (int m = 0; m < n1; m += 4) {
        const float4 f = *reinterpret_cast<const float4*>(row + m);
        s = fma(Dr[m], (T)f.x, s);
        s = fma(Dr[m + 1], (T)f.y, s);
        s = fma(Dr[m + 2], (T)f.z, s);
        s = fma(Dr[m + 3], (T)f.w, s);
      }
    } else {
#pragma unroll
      for (int m = 0; m < n1; ++m) s = fma(Dr[m], row[m], s);
    }
    return s;
  };
  if (valid) {
    T Dr[n1];
#pragma unroll
    for (int m = 0; m < n1; ++m) Dr[m] = sDh[ci * n1 + m];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < n1; ++k)
        acc[v][k] = fma(-inv2h[0], line_dot(&sFh[le][0][v][NF * k + n1 * cj], Dr), acc[v][k]);
    if (D == 3) {
#pragma unroll
      for (int m = 0; m < n1; ++m) Dr[m] = sDh[cj * n1 + m];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < n1; ++k)
          acc[v][k] = fma(-inv2h[1], line_dot(&sFh[le][NT - 1][v][NF * k + n1 * ci], Dr), acc[v][k]);
    }
  }
  __syncthreads();
  // ---- face terms
  const T* mbuf = (const T*)A.mbuf;
  T (*sLift)[NV][NF] = reinterpret_cast<T (*)[NV][NF]>(&sFh[le][0][0][0]);   // [2*NT][NV][NF]
  // lift contribution coef (F* - F_own) of face (a, s) at face node fn, own node own_node
  auto face_lift = [&](int a, int s, int fn, int own_qi, int k, int own_node, T* L) {
    const int32_t* c = A.conn + ((size_t)e * 2 * D + 2 * a + s) * 5;
    const int kind = c[0];
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = sQ[le][v][own_qi];
    const T pp = sQ[le][NV][own_qi];
    const NodeBg<T> bg{sBg[le][k][0], sBg[le][k][1], sBg[le][k][2]};
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    T Fo[NV], Fs[NV];
    flux_axis<T, D>(q, nd, pp, a, Fo);
    if (kind == FACE_WALL || kind == FACE_CONF) {
      const T so = wave_speed<T>(q, nd, bg, pp, a, gamma);
      T qo[NV], Fn[NV], sn;
      if (kind == FACE_WALL) {
#pragma unroll
        for (int v = 0; v < NV; ++v) qo[v] = q[v];
        qo[1 + a] = -q[1 + a];
        flux_axis<T, D>(qo, nd, pp, a, Fn);
        sn = so;
      } else {
        const int stride_a = (a == 0) ? 1 : (a == 1 ? n1 : n1 * n1);
        const int no = own_node + (s ? -N : N) * stride_a;
        const T* qb = (const T*)A.qs + (int64_t)c[1] * NP;
#pragma unroll
        for (int v = 0; v < NV; ++v) qo[v] = qb[v * P + no];
        const T ppo = ((const T*)A.pp_in)[(int64_t)c[1] * NP + no];
        sn = face_side<T, D>(qo, bg, ppo, a, gamma, Fn);
      }
      if (s) rusanov<T, D>(q, Fo, so, qo, Fn, sn, Fs);
      else   rusanov<T, D>(qo, Fn, sn, q, Fo, so, Fs);
    } else {
      const int64_t gg = (kind == FACE_FINE) ? c[2] : c[1];
      const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
      const T* src = mbuf + (((size_t)gg * (1 + NSUB) + slot) * NV) * NF + fn;
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v] = src[(size_t)v * NF];
    }
    const T coef = s ? -lift_of<T>(A, level, a) : lift_of<T>(A, level, a);
#pragma unroll
    for (int v = 0; v < NV; ++v) L[v] = coef * (Fs[v] - Fo[v]);
  };
  if (valid) {
    // horizontal-normal faces: thread t takes face node t (the other horizontal axis fastest)
#pragma unroll
    for (int a = 0; a < NT; ++a) {
      const int u = (D == 3) ? t % n1 : 0;
      const int k = (D == 3) ? t / n1 : t;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int ii, jj;
        if (a == 0) { ii = s ? N : 0; jj = u; } else { ii = u; jj = s ? N : 0; }
        T L[NV];
        face_lift(a, s, t, ii + P1 * (jj + JS * k), k, ii + n1 * jj + NF * k, L);
#pragma unroll
        for (int v = 0; v < NV; ++v) sLift[2 * a + s][v][t] = L[v];
      }
    }
    // bottom and top faces: every column owns one node on each
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k = s ? N : 0;
      T L[NV];
      face_lift(D - 1, s, t, ci + P1 * (cj + JS * k), k, t + NF * k, L);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v][k] += L[v];
    }
  }
  __syncthreads();
  if (!valid) return;
  // lifts of the horizontal-normal faces into the owning columns
#pragma unroll
  for (int a = 0; a < NT; ++a) {
    const int own = (a == 0) ? ci : cj;
    const int u = (a == 0) ? cj : ci;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (own != (s ? N : 0)) continue;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < n1; ++k) acc[v][k] += sLift[2 * a + s][v][(D == 3 ? u : 0) + (D == 3 ? n1 : 1) * k];
    }
  }
  // ---- output
  T* oute = (T*)A.out + e * NP;
  if (A.mode == 0) {
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) oute[v * P + t + NF * k] = acc[v][k];
    return;
  }
  const StageCoef<T> scf = stage_coef<T>(A);
  const T dt = scf.dt, ca = scf.ca, cb = scf.cb;
  const bool first = A.first != 0;
  const T* qne = (const T*)A.qn + e * NP;
  T* ppo = (T*)A.pp_out + e * NP;
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    const int n = t + NF * k;
    const int qi = ci + P1 * (cj + JS * k);
    T qnew[NV];
    if (first) {   // uniform over the grid: stage 1 reads no q^n
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = sQ[le][v][qi] + dt * acc[v][k];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = ca * qne[v * P + n] + cb * (sQ[le][v][qi] + dt * acc[v][k]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
    const size_t zk = (size_t)e * n1 + k;
    ppo[n] = pprime_of<T>(qnew[D + 1], ((const T*)A.bgt)[zk * 4 + 3], A.bg + zk * 4, A.bgc + zk, A.ph);
  }
}

}  // namespace dgk
