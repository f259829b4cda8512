// BR1 viscous term (FP64): nabla . (nu rho nabla phi) on momentum and Theta', phi = (u, theta').
//
// The paper names an artificial viscosity (Sec. 4.3) without giving its operator; this is the
// two-pass method of Bassi & Rebay with central face values:
//  pass 1  sigma_a(phi) = (2/h_a) D_a phi + lift of n_a (phi* - phi) on the faces of axis a,
//  pass 2  V = sum_a (2/h_a) D_a G_a + lift of n_a (G*_a - G_a),  G_a = nu rho sigma_a,
// with phi* and G* the averages of both sides, no flux through walls (phi* = phi, G* = 0), and
// on hanging faces the mortar treatment of the inviscid flux: the coarse value projected with P,
// averaged with the fine one on each mortar, returned to the coarse face as sum_m C X*_m.
// theta' = (Theta' - theta0 rho') / rho, exact for Theta_bar = rho_bar theta0, so a fluid at
// rest gives exactly zero.  There is no viscous mass flux.
#pragma once
#include "dg_device.cuh"

namespace dgk {

struct ViscArgs {
  const double* q;       // state [NV][plane]
  double* sigma;         // [(d+1) d][plane]: component c, axis a at plane c*d + a
  double* V;             // [d+1][plane]
  double* vbuf;          // [G][1 + 2^(d-1)][d+1][NF]
  int64_t plane;
  int32_t E, G;
  const int32_t* elem;
  const int32_t* conn;
  const int32_t* groups;
  const double* bg;
  const double* ops;
  double inv2h[kMaxLevels][3];
  double lift[kMaxLevels][3];   // (2/h_a) / w0 per level and axis
  double nu, theta0;
};

// phi = (u, theta') of one node, with the reciprocal of rho formed once (the forward kernels'
// Newton reciprocal, within one ulp) and multiplied, instead of d + 1 divisions.
template <int D>
__device__ __forceinline__ void visc_phi(const double* q, double rb, double theta0, double* phi) {
  const double rinv = recip(rb + q[0]);
#pragma unroll
  for (int b = 0; b < D; ++b) phi[b] = q[1 + b] * rinv;
  phi[D] = (q[D + 1] - theta0 * q[0]) * rinv;
}

// Mortar values of one pass: pass 1 phi, pass 2 G_a = nu rho sigma_{., a}.  Thread (m, t).
template <int D, int N>
__global__ void __launch_bounds__((1 << (D - 1)) * ipow(N + 1, D - 1))
visc_mortar_kernel(const __grid_constant__ ViscArgs A, int pass) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2, NC = D + 1;
  constexpr int NSUB = 1 << (D - 1);
  __shared__ double sP[2][n1 * n1], sC[2][n1 * n1];
  __shared__ double sX[NC][NF];
  __shared__ double sT[NSUB][NC][NF];
  const int tid = threadIdx.x;
  for (int i = tid; i < n1 * n1; i += blockDim.x) {
    sP[0][i] = A.ops[1 * n1 * n1 + i];
    sP[1][i] = A.ops[2 * n1 * n1 + i];
    sC[0][i] = A.ops[3 * n1 * n1 + i];
    sC[1][i] = A.ops[4 * n1 * n1 + i];
  }
  const int g = blockIdx.x;
  const int32_t* row = A.groups + (size_t)g * 7;
  const int64_t ec = row[0];
  const int a = row[1], side = row[2];
  const int m = tid / NF, t = tid - m * NF;
  // value of the pass at node `node` of element `el`
  auto value = [&](int64_t el, int node, double* X) {
    const int k = (D == 3) ? node / (n1 * n1) : node / n1;
    const double rb = A.bg[((size_t)el * n1 + k) * 4];
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = A.q[(size_t)v * A.plane + (size_t)el * NP + node];
    if (pass == 1) {
      visc_phi<D>(q, rb, A.theta0, X);
    } else {
      const double nr = A.nu * (rb + q[0]);
#pragma unroll
      for (int c = 0; c < NC; ++c) X[c] = nr * A.sigma[(size_t)(c * D + a) * A.plane + (size_t)el * NP + node];
    }
  };
  if (tid < NF) {
    double X[NC];
    value(ec, face_node<D, N>(a, side, tid), X);
#pragma unroll
    for (int c = 0; c < NC; ++c) sX[c][tid] = X[c];
  }
  __syncthreads();
  const int b0 = m & 1, b1 = (m >> 1) & 1;
  const int t0 = t % n1, t1 = t / n1;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += sP[b0][t0 * n1 + j] * sX[c][j + n1 * t1];
    sT[m][c][t] = s;
  }
  __syncthreads();
  double xs[NC], Xf[NC];
  value(row[3 + m], face_node<D, N>(a, 1 - side, t), Xf);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double xp = sT[m][c][t];
    if (D == 3) {
      xp = 0.0;
#pragma unroll
      for (int j = 0; j < n1; ++j) xp += sP[b1][t1 * n1 + j] * sT[m][c][t0 + n1 * j];
    }
    xs[c] = 0.5 * (xp + Xf[c]);
  }
  __syncthreads();
  double* vb = A.vbuf + ((size_t)g * (1 + NSUB) * NC) * NF;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    vb[((size_t)(1 + m) * NC + c) * NF + t] = xs[c];
    sT[m][c][t] = xs[c];
  }
  __syncthreads();
  // back to the coarse face: sum_m (C_b1 x C_b0) X*_m, first along t0 ...
  double first[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += sC[b0][t0 * n1 + j] * sT[m][c][j + n1 * t1];
    first[c] = s;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) sT[m][c][t] = first[c];
  __syncthreads();
  if (m == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double acc = 0.0;
      for (int mm = 0; mm < NSUB; ++mm) {
        if (D == 3) {
          const int c1 = (mm >> 1) & 1;
          double s = 0.0;
#pragma unroll
          for (int j = 0; j < n1; ++j) s += sC[c1][t1 * n1 + j] * sT[mm][c][t0 + n1 * j];
          acc += s;
        } else {
          acc += sT[mm][c][t];
        }
      }
      vb[(size_t)c * NF + t] = acc;
    }
  }
}

// Pass 1 (sigma) or pass 2 (V), one thread per node.
template <int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D))
visc_pass_kernel(const __grid_constant__ ViscArgs A, int pass) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2, NC = D + 1;
  constexpr int NSUB = 1 << (D - 1);
  __shared__ double sD[n1 * n1];
  __shared__ double sX[EPB][NC][NP];
  const int tid = threadIdx.x;
  for (int i = tid; i < n1 * n1; i += blockDim.x) sD[i] = A.ops[i];
  const int le = tid / NP, n = tid - le * NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool valid = e < A.E;
  int idx[3];
  idx[0] = n % n1;
  idx[1] = (n / n1) % n1;
  idx[2] = (D == 3) ? n / (n1 * n1) : 0;
  const size_t base = (size_t)(valid ? e : 0) * NP + n;
  double q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = valid ? A.q[(size_t)v * A.plane + base] : 0.0;
  const double rb = valid ? A.bg[((size_t)e * n1 + idx[D - 1]) * 4] : 1.0;
  const int level = valid ? A.elem[e * 4] : 0;
  double phi[NC];
  visc_phi<D>(q, rb, A.theta0, phi);
  const double nr = A.nu * (rb + q[0]);
  double out[NC * D];
#pragma unroll
  for (int i = 0; i < NC * D; ++i) out[i] = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double Xa[NC];    // the field differentiated along a: phi (pass 1) or G_a (pass 2)
#pragma unroll
    for (int c = 0; c < NC; ++c)
      Xa[c] = pass == 1 ? phi[c] : (valid ? nr * A.sigma[(size_t)(c * D + a) * A.plane + base] : 0.0);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) sX[le][c][n] = Xa[c];
    __syncthreads();
    if (!valid) continue;
    const int stride = ipow(n1, a);
    const int ia = idx[a];
    const int b0 = n - ia * stride;
    const double s2h = A.inv2h[level][a];
    double dX[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double s = 0.0;
#pragma unroll
      for (int mm = 0; mm < n1; ++mm) s += sD[ia * n1 + mm] * sX[le][c][b0 + mm * stride];
      dX[c] = s2h * s;
    }
    // face lifts n_a (2/h_a)/w0 (X* - X) on this axis
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (ia != (s ? N : 0)) continue;
      const int32_t* cn = A.conn + ((size_t)e * 2 * D + 2 * a + s) * 5;
      const int kind = cn[0];
      const double coef = s ? A.lift[level][a] : -A.lift[level][a];
      double xs[NC];
      bool have = true;
      if (kind == FACE_CONF) {
        const int64_t nb = cn[1];
        const size_t no = (size_t)nb * NP + n + ((s ? 0 : N) - ia) * stride;
        double qo[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) qo[v] = A.q[(size_t)v * A.plane + no];
        if (pass == 1) {
          double po[NC];
          visc_phi<D>(qo, rb, A.theta0, po);
#pragma unroll
          for (int c = 0; c < NC; ++c) xs[c] = 0.5 * (Xa[c] + po[c]);
        } else {
          const double nro = A.nu * (rb + qo[0]);
#pragma unroll
          for (int c = 0; c < NC; ++c) xs[c] = 0.5 * (Xa[c] + nro * A.sigma[(size_t)(c * D + a) * A.plane + no]);
        }
      } else if (kind == FACE_WALL) {
        if (pass == 1) have = false;         // phi* = phi: no lift
        else {
#pragma unroll
          for (int c = 0; c < NC; ++c) xs[c] = 0.0;   // no viscous flux through the wall
        }
      } else {
        int t = 0, mul = 1;
#pragma unroll
        for (int b = 0; b < D; ++b)
          if (b != a) { t += idx[b] * mul; mul *= n1; }
        const int64_t g = (kind == FACE_FINE) ? cn[2] : cn[1];
        const int slot = (kind == FACE_FINE) ? 1 + cn[3] : 0;
        const double* src = A.vbuf + (((size_t)g * (1 + NSUB) + slot) * NC) * NF + t;
#pragma unroll
        for (int c = 0; c < NC; ++c) xs[c] = src[(size_t)c * NF];
      }
      if (have) {
#pragma unroll
        for (int c = 0; c < NC; ++c) dX[c] += coef * (xs[c] - Xa[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c * D + a] = dX[c];
  }
  if (!valid) return;
  if (pass == 1) {
#pragma unroll
    for (int i = 0; i < NC * D; ++i) A.sigma[(size_t)i * A.plane + base] = out[i];
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) s += out[c * D + a];
      A.V[(size_t)c * A.plane + base] = s;
    }
  }
}

}  // namespace dgk
