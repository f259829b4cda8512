// Helper kernels of the GB300 dGSEM library that run once per regrid or per diagnostic:
// hydrostatic background (FP64), initial bubble, refinement indicator, compensated integrals
// and the conservative parent<->child transfer of Sec. 3.3.
#include "dg_launch.hpp"

#include <cmath>

namespace dgk {
namespace {

__device__ __forceinline__ double node_coord(int c, double xi, double h) {
  // (c + (xi + 1)/2) h: faces shared by two elements get bit-identical coordinates
  return (c + (xi + 1.0) * 0.5) * h;
}

// Hydrostatic neutral background at the z-nodes of every element (Sec. 4.3):
// pi = 1 - g z / (cp theta0), rho_bar = p0 pi^(cv/R) / (R theta0), Theta_bar = rho_bar theta0,
// p_bar := P(Theta_bar) = p0 (R Theta_bar / p0)^gamma so that a fluid at rest has P' = 0.
__global__ void background_kernel(int32_t E, int n1, int D, const int32_t* elem,
                                  const double* xi, double root_hz, PhysC ph, double* bg,
                                  float* bgf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)E * n1) return;
  const int64_t e = i / n1;
  const int k = (int)(i - e * n1);
  const int level = elem[e * 4];
  const double hz = ldexp(root_hz, -level);
  const double z = node_coord(elem[e * 4 + D], xi[k], hz);
  const double pi = 1.0 - ph.g * z / (ph.cp * ph.theta0);
  const double rb = ph.p0 * pow(pi, ph.cv / ph.R) / (ph.R * ph.theta0);
  const double Tb = rb * ph.theta0;
  const double pb = ph.p0 * pow(ph.R * Tb / ph.p0, ph.gamma);
  double* o = bg + i * 4;
  o[0] = rb; o[1] = Tb; o[2] = pb; o[3] = 1.0 / Tb;
  if (bgf) {
    float* f = bgf + i * 4;
    f[0] = (float)rb; f[1] = (float)Tb; f[2] = (float)pb; f[3] = (float)(1.0 / Tb);
  }
}

template <class T>
__global__ void bubble_kernel(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                              double rh0, double rh1, double rh2, const double* bg,
                              double c0, double c1, double c2, double r0, double r1, double r2,
                              double amp, int n_rff, double rff_scale, const double* rff_k,
                              const double* rff_phase, double theta0, T* q, int64_t plane,
                              double* theta_out) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)E * NP) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
  const int level = elem[e * 4];
  const double rh[3] = {rh0, rh1, rh2}, cen[3] = {c0, c1, c2}, rad[3] = {r0, r1, r2};
  double x[3] = {0.0, 0.0, 0.0};
  double r2s = 0.0;
  for (int a = 0; a < D; ++a) {
    x[a] = node_coord(elem[e * 4 + 1 + a], xi[idx[a]], ldexp(rh[a], -level));
    const double s = (x[a] - cen[a]) / rad[a];
    r2s = r2s + s * s;
  }
  const double r = sqrt(r2s);
  double th = r <= 1.0 ? amp * (1.0 + cos(M_PI * r)) : 0.0;
  if (n_rff > 0) {
    double acc = 0.0;
    for (int m = 0; m < n_rff; ++m) {
      double arg = rff_phase[m];
      for (int a = 0; a < D; ++a) arg = arg + rff_k[m * 3 + a] * x[a];
      acc = acc + cos(arg);
    }
    th = th + rff_scale * acc;
  }
  if (theta_out) { theta_out[i] = th; return; }
  const double rb = bg[(e * n1 + idx[D - 1]) * 4];
  q[i] = (T)(-rb * th / (theta0 + th));
  for (int v = 1; v < D + 2; ++v) q[(int64_t)v * plane + i] = (T)0;
}

// max over the element's nodes of |theta'|, theta' = (Theta_bar + Theta') / (rho_bar + rho')
// - theta0, in FP64 (refinement criterion of Sec. 4.3, tagging by potential temperature).
template <class T>
__global__ void indicator_kernel(int32_t E, int n1, int D, const double* bg, const T* q,
                                 int64_t plane, double theta0, double* out) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t e = blockIdx.x;
  __shared__ double red[256];
  double m = 0.0;
  for (int n = threadIdx.x; n < NP; n += blockDim.x) {
    const int k = D == 3 ? n / (n1 * n1) : n / n1;
    const double* b = bg + (e * n1 + k) * 4;
    const int64_t i = e * NP + n;
    const double th = (b[1] + (double)q[(int64_t)(D + 1) * plane + i]) / (b[0] + (double)q[i]) - theta0;
    m = fmax(m, fabs(th));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = red[0];
}

// Primitive diagnostics per node in FP64: out[a] = U_a / rho (a < D), out[D] = theta'
// = (Theta_bar + Theta') / (rho_bar + rho') - theta0; planes of length E * NP.
template <class T>
__global__ void primitives_kernel(int32_t E, int n1, int D, const double* bg, const T* q,
                                  int64_t plane, double theta0, double* out) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int k = D == 3 ? n / (n1 * n1) : n / n1;
  const double* b = bg + (e * n1 + k) * 4;
  const double rho = b[0] + (double)q[i];
  for (int a = 0; a < D; ++a) out[a * total + i] = (double)q[(int64_t)(1 + a) * plane + i] / rho;
  out[D * total + i] = (b[1] + (double)q[(int64_t)(D + 1) * plane + i]) / rho - theta0;
}

// Neumaier-compensated accumulator.
struct Comp {
  double s, c;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ void merge(const Comp& o) { add(o.s); c += o.c; }
};

constexpr int kIntBlocks = 512;
constexpr int kIntThreads = 256;

// Partial integrals: each block reduces a fixed grid-stride slice in a fixed tree order.
template <class T>
__global__ void __launch_bounds__(kIntThreads)
integrals_partial(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                  const double* w, double rh0, double rh1, double rh2, const double* bg,
                  const T* q, int64_t plane, PhysC ph, double* partial, int* bad) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  Comp acc[NUM_INTEGRALS];
  for (int k = 0; k < NUM_INTEGRALS; ++k) acc[k] = Comp{0.0, 0.0};
  const double rh[3] = {rh0, rh1, rh2};
  int nonfinite = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / NP;
    const int n = (int)(i - e * NP);
    int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
    const int level = elem[e * 4];
    double wn = 1.0, J = 1.0, z = 0.0;
    for (int a = 0; a < D; ++a) {
      const double h = ldexp(rh[a], -level);
      wn = wn * w[idx[a]];
      J = J * (h * 0.5);
      if (a == D - 1) z = node_coord(elem[e * 4 + 1 + a], xi[idx[a]], h);
    }
    const double W = wn * J;
    const double* b = bg + (e * n1 + idx[D - 1]) * 4;
    const double rp = (double)q[i];
    const double rho = b[0] + rp;
    double u2 = 0.0;
    for (int a = 0; a < D; ++a) {
      const double U = (double)q[(int64_t)(1 + a) * plane + i];
      u2 = u2 + U * U;
    }
    const double ke = 0.5 * u2 / rho;
    const double tp = (double)q[(int64_t)(D + 1) * plane + i];
    const double pp = pressure_pert<kSeries>(tp, b[3], b[2], ph);
    const double p = b[2] + pp;
    const double en = p * ph.cv / ph.R + ke + rho * ph.g * z;
    if (!isfinite(rho) || !isfinite(en)) nonfinite = 1;
    acc[0].add(W * rho);
    acc[1].add(W * en);
    acc[2].add(W * ke);
    acc[3].add(W);
    acc[4].add(W * rp);
  }
  if (nonfinite) atomicOr(bad, 1);
  __shared__ double ss[NUM_INTEGRALS][kIntThreads], sc[NUM_INTEGRALS][kIntThreads];
  for (int k = 0; k < NUM_INTEGRALS; ++k) { ss[k][threadIdx.x] = acc[k].s; sc[k][threadIdx.x] = acc[k].c; }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < NUM_INTEGRALS; ++k) {
        Comp a{ss[k][threadIdx.x], sc[k][threadIdx.x]};
        a.merge(Comp{ss[k][threadIdx.x + s], sc[k][threadIdx.x + s]});
        ss[k][threadIdx.x] = a.s; sc[k][threadIdx.x] = a.c;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < NUM_INTEGRALS; ++k) {
      partial[(blockIdx.x * NUM_INTEGRALS + k) * 2] = ss[k][0];
      partial[(blockIdx.x * NUM_INTEGRALS + k) * 2 + 1] = sc[k][0];
    }
}

// Final pass: one thread per integral walks the block partials in order.
__global__ void integrals_final(int nblocks, const double* partial, double* out) {
  const int k = threadIdx.x;
  if (k >= NUM_INTEGRALS) return;
  Comp a{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b)
    a.merge(Comp{partial[(b * NUM_INTEGRALS + k) * 2], partial[(b * NUM_INTEGRALS + k) * 2 + 1]});
  out[k] = a.s + a.c;
}

// Conservative transfer after a regrid (Sec. 3.3), one CTA per new element, FP64 arithmetic:
//   keep:   copy;
//   child:  (P_{c_2} x P_{c_1} x P_{c_0}) parent, P_c the half-interval interpolation;
//   parent: sum_c (C_{c_2} x C_{c_1} x C_{c_0}) child_c, C_c = (1/2) M^{-1} S_c^T.
template <class T>
__global__ void transfer_kernel(int32_t Enew, int n1, int D, const int32_t* tmap,
                                const double* ops, const T* qold, int64_t plane_old, T* qnew,
                                int64_t plane_new) {
  extern __shared__ double sm[];
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int nn = n1 * n1;
  double* sP = sm;              // P0, P1, C0, C1
  double* s0 = sm + 4 * nn;
  double* s1 = s0 + NP;
  double* sacc = s1 + NP;
  for (int i = threadIdx.x; i < 4 * nn; i += blockDim.x) sP[i] = ops[nn + i];
  const int64_t e = blockIdx.x;
  const int32_t* row = tmap + e * 9;
  const int kind = row[0];
  const int n = threadIdx.x;
  int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
  const int nv = D + 2;
  __syncthreads();
  for (int v = 0; v < nv; ++v) {
    if (kind == 0) {
      if (n < NP) qnew[(int64_t)v * plane_new + e * NP + n] = qold[(int64_t)v * plane_old + (int64_t)row[1] * NP + n];
      continue;
    }
    const int nsrc = kind == 1 ? 1 : (1 << D);
    if (n < NP) sacc[n] = 0.0;
    for (int c = 0; c < nsrc; ++c) {
      const int64_t src = kind == 1 ? row[1] : row[1 + c];
      const int ci = kind == 1 ? row[2] : c;
      const double* mats = kind == 1 ? sP : sP + 2 * nn;
      __syncthreads();
      if (n < NP) s0[n] = (double)qold[(int64_t)v * plane_old + src * NP + n];
      __syncthreads();
      double* in = s0;
      double* out = s1;
      for (int a = 0; a < D; ++a) {
        const double* M = mats + ((ci >> a) & 1) * nn;
        const int stride = a == 0 ? 1 : (a == 1 ? n1 : nn);
        if (n < NP) {
          const int ia = idx[a];
          const int b0 = n - ia * stride;
          double s = 0.0;
          for (int m = 0; m < n1; ++m) s += M[ia * n1 + m] * in[b0 + m * stride];
          out[n] = s;
        }
        __syncthreads();
        double* t = in; in = out; out = t;
      }
      if (n < NP) sacc[n] += in[n];
    }
    __syncthreads();
    if (n < NP) qnew[(int64_t)v * plane_new + e * NP + n] = (T)sacc[n];
  }
}

}  // namespace

cudaError_t launch_background(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                              double root_hz, const PhysC& ph, double* bg, float* bgf,
                              cudaStream_t s) {
  const int64_t n = (int64_t)E * n1;
  if (n == 0) return cudaSuccess;
  background_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, n1, D, elem, xi, root_hz, ph, bg, bgf);
  return cudaGetLastError();
}

cudaError_t launch_pprime(int prec, int32_t E, int n1, int D, const void* theta_plane,
                          const double* bg, const PhysC& ph, void* pp, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t n = (int64_t)E * NP;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 0)
    pprime_kernel<double><<<blocks, 256, 0, s>>>(n, NP, n1, D, (const double*)theta_plane, bg, ph, (double*)pp);
  else
    pprime_kernel<float><<<blocks, 256, 0, s>>>(n, NP, n1, D, (const float*)theta_plane, bg, ph, (float*)pp);
  return cudaGetLastError();
}

cudaError_t launch_bubble(int prec, int32_t E, int n1, int D, const int32_t* elem,
                          const double* xi, const double* root_h, const double* bg,
                          const double* center, const double* radius, double amp, int n_rff,
                          double rff_scale, const double* rff_k, const double* rff_phase,
                          double theta0, void* q, int64_t plane, double* theta_out,
                          cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t n = (int64_t)E * NP;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 0)
    bubble_kernel<double><<<blocks, 256, 0, s>>>(E, n1, D, elem, xi, root_h[0], root_h[1], root_h[2], bg,
        center[0], center[1], center[2], radius[0], radius[1], radius[2], amp, n_rff, rff_scale,
        rff_k, rff_phase, theta0, (double*)q, plane, theta_out);
  else
    bubble_kernel<float><<<blocks, 256, 0, s>>>(E, n1, D, elem, xi, root_h[0], root_h[1], root_h[2], bg,
        center[0], center[1], center[2], radius[0], radius[1], radius[2], amp, n_rff, rff_scale,
        rff_k, rff_phase, theta0, (float*)q, plane, theta_out);
  return cudaGetLastError();
}

cudaError_t launch_indicator(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                             int64_t plane, double theta0, double* out, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  if (prec == 0) indicator_kernel<double><<<E, 256, 0, s>>>(E, n1, D, bg, (const double*)q, plane, theta0, out);
  else indicator_kernel<float><<<E, 256, 0, s>>>(E, n1, D, bg, (const float*)q, plane, theta0, out);
  return cudaGetLastError();
}

cudaError_t launch_primitives(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                              int64_t plane, double theta0, double* out, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (prec == 0) primitives_kernel<double><<<grid, 256, 0, s>>>(E, n1, D, bg, (const double*)q, plane, theta0, out);
  else primitives_kernel<float><<<grid, 256, 0, s>>>(E, n1, D, bg, (const float*)q, plane, theta0, out);
  return cudaGetLastError();
}

size_t integrals_scratch_doubles() { return (size_t)kIntBlocks * NUM_INTEGRALS * 2; }

cudaError_t launch_integrals(int prec, int32_t E, int n1, int D, const int32_t* elem,
                             const double* xi, const double* w, const double* root_h,
                             const double* bg, const void* q, int64_t plane, const PhysC& ph,
                             double* partial, int* bad, double* out, cudaStream_t s) {
  if (prec == 0)
    integrals_partial<double><<<kIntBlocks, kIntThreads, 0, s>>>(E, n1, D, elem, xi, w, root_h[0],
        root_h[1], root_h[2], bg, (const double*)q, plane, ph, partial, bad);
  else
    integrals_partial<float><<<kIntBlocks, kIntThreads, 0, s>>>(E, n1, D, elem, xi, w, root_h[0],
        root_h[1], root_h[2], bg, (const float*)q, plane, ph, partial, bad);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  integrals_final<<<1, 32, 0, s>>>(kIntBlocks, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_transfer(int prec, int32_t Enew, int n1, int D, const int32_t* tmap,
                            const double* ops, const void* qold, int64_t plane_old, void* qnew,
                            int64_t plane_new, cudaStream_t s) {
  if (Enew == 0) return cudaSuccess;
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int threads = ((NP + 31) / 32) * 32;
  const size_t smem = (size_t)(4 * n1 * n1 + 3 * NP) * sizeof(double);
  if (prec == 0)
    transfer_kernel<double><<<Enew, threads, smem, s>>>(Enew, n1, D, tmap, ops, (const double*)qold,
                                                        plane_old, (double*)qnew, plane_new);
  else
    transfer_kernel<float><<<Enew, threads, smem, s>>>(Enew, n1, D, tmap, ops, (const float*)qold,
                                                       plane_old, (float*)qnew, plane_new);
  return cudaGetLastError();
}

}  // namespace dgk
