// Passive tracer C advected by a prescribed wind (2D, FP64): the linear-advection test of
// Sec. 4.2 (swirling deformational flow after LeVeque) and the conservation comparison there,
// mortars vs point-to-point interpolation on hanging faces.
//
// dC/dt + div(C u) = 0 with u = sin^2(pi x) sin(2 pi y) g,  v = -sin^2(pi y) sin(2 pi x) g,
// g = cos(pi t / T) evaluated by the host at each stage time.  Strong-form dGSEM as for the Euler
// equations (Sec. 2.2): volume term -sum_a (2/h_a) D_a (C u_a), face lifts
// n (2/h)/w0 (F* - C u_n) with the upwind flux F* = u_n (C- + C+)/2 - |u_n| (C+ - C-)/2, no flux
// through walls.  Hanging faces (one CTA per coarse face and its two fine neighbours):
//   fine side    F*_m at the fine face nodes against the projected coarse trace P_m C_c;
//   coarse side  mortar: sum_m C_m F*_m (conservative, Sec. 3.3);
//                interp: F* at its own nodes against the fine traces evaluated there,
//                sum_m G_m C_f,m (the non-conservative point-to-point alternative).
#pragma once
#include "dg_device.cuh"

namespace dgk {

struct TracerArgs {
  const double* cs;      // stage input C [plane]
  const double* cn;      // C^n for the Shu-Osher combination
  double* out;           // dC/dt (mode 0) or the next stage (mode 1)
  const double* mbuf;    // [G][3][N+1]: slot 0 coarse side, 1 + m fine face m
  int64_t plane;
  int32_t E;
  const int32_t* elem;   // [E][4] level, c0, c1, c2
  const int32_t* conn;   // [E][4][5]
  const double* ops;     // D, P0, P1, C0, C1, w, x, G0, G1 (FP64)
  double root_h[2];
  double inv2h[kMaxLevels][2];
  double lift[kMaxLevels][2];
  double g;              // cos(pi t / T) at the stage time
  double dt, ca, cb;
  int32_t mode;
};

struct TracerMortarArgs {
  const double* cs;
  double* mbuf;
  int64_t plane;
  int32_t G;
  const int32_t* groups; // [G][7]: coarse element, axis, side, fine elements
  const int32_t* elem;
  const double* ops;
  double root_h[2];
  double g;
  int32_t interp;        // 0 mortar, 1 point-to-point interpolation
};

// Wind of Sec. 4.2 at (x, y) (g = cos(pi t / T)), as the oracle writes it.
__device__ __forceinline__ void swirl_wind(double x, double y, double g, double* u, double* v) {
  const double sx = sin(M_PI * x), sy = sin(M_PI * y);
  *u = sx * sx * sin(2.0 * M_PI * y) * g;
  *v = -(sy * sy) * sin(2.0 * M_PI * x) * g;
}

__device__ __forceinline__ double upwind_flux(double cm, double cp, double un) {
  return 0.5 * un * (cm + cp) - 0.5 * fabs(un) * (cp - cm);
}

// Coordinates of node (i, j) of element e: (c + (xi + 1)/2) h per axis.
__device__ __forceinline__ void tracer_xy(const int32_t* elem, int64_t e, const double* xi, const double* root_h,
                                          int i, int j, double* x, double* y) {
  const int level = elem[e * 4];
  const double hx = ldexp(root_h[0], -level), hy = ldexp(root_h[1], -level);
  *x = (elem[e * 4 + 1] + (xi[i] + 1.0) * 0.5) * hx;
  *y = (elem[e * 4 + 2] + (xi[j] + 1.0) * 0.5) * hy;
}

template <int N, int EPB>
__global__ void __launch_bounds__(EPB * (N + 1) * (N + 1))
tracer_stage_kernel(const __grid_constant__ TracerArgs A) {
  constexpr int n1 = N + 1, NP = n1 * n1, NF = n1, NSUB = 2;
  __shared__ double sD[n1 * n1];
  __shared__ double sF[EPB][2][NP];
  const int tid = threadIdx.x;
  for (int k = tid; k < n1 * n1; k += blockDim.x) sD[k] = A.ops[k];
  const double* xi = A.ops + 5 * n1 * n1 + n1;
  const int le = tid / NP, n = tid - le * NP;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool valid = e < A.E;
  const int idx[2] = {n % n1, n / n1};
  double C = 0.0, U[2] = {0.0, 0.0};
  int level = 0;
  if (valid) {
    double x, y;
    tracer_xy(A.elem, e, xi, A.root_h, idx[0], idx[1], &x, &y);
    swirl_wind(x, y, A.g, &U[0], &U[1]);
    C = A.cs[e * NP + n];
    level = A.elem[e * 4];
  }
  sF[le][0][n] = C * U[0];
  sF[le][1][n] = C * U[1];
  __syncthreads();
  if (!valid) return;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int stride = a == 0 ? 1 : n1;
    const int b0 = n - idx[a] * stride;
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < n1; ++m) s += sD[idx[a] * n1 + m] * sF[le][a][b0 + m * stride];
    acc -= A.inv2h[level][a] * s;
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (idx[a] != (s ? N : 0)) continue;
      const int32_t* c = A.conn + ((size_t)e * 4 + 2 * a + s) * 5;
      const int kind = c[0];
      const double un = U[a];
      double Fs;
      if (kind == FACE_WALL) {
        Fs = 0.0;                              // mirror state: the normal wind reverses
      } else if (kind == FACE_CONF) {
        const int stride = a == 0 ? 1 : n1;
        const double cnb = A.cs[(int64_t)c[1] * NP + n + ((s ? 0 : N) - idx[a]) * stride];
        Fs = s ? upwind_flux(C, cnb, un) : upwind_flux(cnb, C, un);
      } else {
        const int t = idx[1 - a];
        const int64_t g = (kind == FACE_FINE) ? c[2] : c[1];
        const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
        Fs = A.mbuf[((size_t)g * (1 + NSUB) + slot) * NF + t];
      }
      const double lc = A.lift[level][a];
      acc += (s ? -lc : lc) * (Fs - C * un);
    }
  }
  double* o = A.out + e * NP + n;
  if (A.mode == 0) { *o = acc; return; }
  const double cs = C;
  *o = A.ca == 0.0 ? cs + A.dt * acc : A.ca * A.cn[e * NP + n] + A.cb * (cs + A.dt * acc);
}

// One CTA per hanging face: thread (m, t) = fine face m, face node t.
template <int N>
__global__ void __launch_bounds__(2 * (N + 1))
tracer_mortar_kernel(const __grid_constant__ TracerMortarArgs A) {
  constexpr int n1 = N + 1, NP = n1 * n1, NF = n1;
  __shared__ double sP[2][n1 * n1], sCm[2][n1 * n1], sG[2][n1 * n1];
  __shared__ double sc[NF], sf[2][NF], sFs[2][NF];
  const int tid = threadIdx.x;
  for (int k = tid; k < n1 * n1; k += blockDim.x) {
    sP[0][k] = A.ops[1 * n1 * n1 + k];
    sP[1][k] = A.ops[2 * n1 * n1 + k];
    sCm[0][k] = A.ops[3 * n1 * n1 + k];
    sCm[1][k] = A.ops[4 * n1 * n1 + k];
    sG[0][k] = A.ops[5 * n1 * n1 + 2 * n1 + k];
    sG[1][k] = A.ops[6 * n1 * n1 + 2 * n1 + k];
  }
  const double* xi = A.ops + 5 * n1 * n1 + n1;
  const int32_t* row = A.groups + (size_t)blockIdx.x * 7;
  const int64_t ec = row[0];
  const int a = row[1], side = row[2];
  const int m = tid / NF, t = tid - m * NF;
  const int64_t ef = row[3 + m];
  // face node t of face (a, s): the normal index at 0 or N, the tangential one t
  auto node_ij = [&](int s, int tt, int* i, int* j) {
    if (a == 0) { *i = s ? N : 0; *j = tt; } else { *i = tt; *j = s ? N : 0; }
  };
  int ic, jc, iff, jf;
  node_ij(side, t, &ic, &jc);
  node_ij(1 - side, t, &iff, &jf);
  if (m == 0) sc[t] = A.cs[ec * NP + ic + n1 * jc];
  sf[m][t] = A.cs[ef * NP + iff + n1 * jf];
  __syncthreads();
  double proj = 0.0;
#pragma unroll
  for (int j = 0; j < n1; ++j) proj += sP[m][t * n1 + j] * sc[j];
  double x, y, u, v;
  tracer_xy(A.elem, ef, xi, A.root_h, iff, jf, &x, &y);
  swirl_wind(x, y, A.g, &u, &v);
  const double unf = a == 0 ? u : v;
  // the coarse element is the low side when its face is at side 1
  const double Fs = side ? upwind_flux(proj, sf[m][t], unf) : upwind_flux(sf[m][t], proj, unf);
  double* mb = A.mbuf + (size_t)blockIdx.x * 3 * NF;
  mb[(1 + m) * NF + t] = Fs;
  sFs[m][t] = Fs;
  __syncthreads();
  if (m != 0) return;
  double Fc;
  if (!A.interp) {
    Fc = 0.0;
#pragma unroll
    for (int mm = 0; mm < 2; ++mm)
#pragma unroll
      for (int j = 0; j < n1; ++j) Fc += sCm[mm][t * n1 + j] * sFs[mm][j];
  } else {
    double gath = 0.0;
#pragma unroll
    for (int mm = 0; mm < 2; ++mm)
#pragma unroll
      for (int j = 0; j < n1; ++j) gath += sG[mm][t * n1 + j] * sf[mm][j];
    tracer_xy(A.elem, ec, xi, A.root_h, ic, jc, &x, &y);
    swirl_wind(x, y, A.g, &u, &v);
    const double unc = a == 0 ? u : v;
    Fc = side ? upwind_flux(sc[t], gath, unc) : upwind_flux(gath, sc[t], unc);
  }
  mb[t] = Fc;
}

}  // namespace dgk
