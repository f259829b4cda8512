// FP64 adjoint kernels (instantiations) and the small maps around them: the initial state of a
// nodal theta' field and its transpose, and the gradient of the kinetic-energy integral.
#include "dg_adjoint.cuh"
#include "dg_launch.hpp"

namespace dgk {
namespace {

template <int D, int N>
void run_vjp(const AdjArgs& A, cudaStream_t s, cudaError_t& err) {
  constexpr int NP = ipow(N + 1, D);
  constexpr int EPB = NP >= 128 ? 1 : 256 / NP;
  constexpr size_t smem = VjpSmem<D, N, EPB>::bytes;
  const unsigned blocks = (unsigned)((A.E + EPB - 1) / EPB);
  if (!blocks) return;
  err = configure_kernel((const void*)vjp_kernel<D, N, EPB>, smem, false);
  if (err == cudaSuccess) vjp_kernel<D, N, EPB><<<blocks, EPB * NP, smem, s>>>(A);
}

template <int D, int N>
void run_mortar_vjp(const MortarAdjArgs& A, cudaStream_t s) {
  if (A.G) mortar_vjp_kernel<D, N><<<A.G, (1 << (D - 1)) * ipow(N + 1, D - 1), 0, s>>>(A);
}

template <int D>
bool vjp_dispatch(int N, const AdjArgs& A, cudaStream_t s, cudaError_t& err) {
  switch (N) {
    case 1: run_vjp<D, 1>(A, s, err); return true;
    case 2: run_vjp<D, 2>(A, s, err); return true;
    case 3: run_vjp<D, 3>(A, s, err); return true;
    case 4: run_vjp<D, 4>(A, s, err); return true;
    case 5: run_vjp<D, 5>(A, s, err); return true;
    case 6: run_vjp<D, 6>(A, s, err); return true;
    case 7: run_vjp<D, 7>(A, s, err); return true;
    case 8: run_vjp<D, 8>(A, s, err); return true;
    default: return false;
  }
}

template <int D>
bool mortar_vjp_dispatch(int N, const MortarAdjArgs& A, cudaStream_t s) {
  switch (N) {
    case 1: run_mortar_vjp<D, 1>(A, s); return true;
    case 2: run_mortar_vjp<D, 2>(A, s); return true;
    case 3: run_mortar_vjp<D, 3>(A, s); return true;
    case 4: run_mortar_vjp<D, 4>(A, s); return true;
    case 5: run_mortar_vjp<D, 5>(A, s); return true;
    case 6: run_mortar_vjp<D, 6>(A, s); return true;
    case 7: run_mortar_vjp<D, 7>(A, s); return true;
    case 8: run_mortar_vjp<D, 8>(A, s); return true;
    default: return false;
  }
}

// rho' = -rho_bar theta' / (theta0 + theta'), U = 0, Theta' = 0 (hydrostatic-pressure initial
// state of a theta' field, as for the bubble).
template <class T>
__global__ void theta_state_kernel(int64_t total, int NP, int n1, int D, const double* bg,
                                   const double* theta, double theta0, T* q, int64_t plane) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int k = D == 3 ? n / (n1 * n1) : n / n1;
  const double rb = bg[(e * n1 + k) * 4];
  const double th = theta[i];
  q[i] = (T)(-rb * th / (theta0 + th));
  for (int v = 1; v < D + 2; ++v) q[(int64_t)v * plane + i] = (T)0;
}

// d rho'/d theta' = -rho_bar theta0 / (theta0 + theta')^2; the other variables do not depend on
// theta'.
__global__ void theta_vjp_kernel(int64_t total, int NP, int n1, int D, const double* bg,
                                 const double* theta, double theta0, const double* lam_q,
                                 double* lam_theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int k = D == 3 ? n / (n1 * n1) : n / n1;
  const double rb = bg[(e * n1 + k) * 4];
  const double den = theta0 + theta[i];
  lam_theta[i] = lam_q[i] * (-rb * theta0 / (den * den));
}

// Gradient of KE = sum w J |U|^2 / (2 rho): dKE/drho' = -w J |U|^2 / (2 rho^2),
// dKE/dU = w J U / rho, dKE/dTheta' = 0.
__global__ void ke_grad_kernel(int64_t total, int NP, int n1, int D, const int32_t* elem,
                               const double* w, double rh0, double rh1, double rh2,
                               const double* bg, const double* q, int64_t plane, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
  const int level = elem[e * 4];
  const double rh[3] = {rh0, rh1, rh2};
  double W = 1.0;
  for (int a = 0; a < D; ++a) W = W * w[idx[a]];
  double J = 1.0;
  for (int a = 0; a < D; ++a) J = J * (ldexp(rh[a], -level) * 0.5);
  W = W * J;
  const double rho = bg[(e * n1 + idx[D - 1]) * 4] + q[i];
  double u2 = 0.0;
  for (int a = 0; a < D; ++a) {
    const double U = q[(int64_t)(1 + a) * plane + i];
    u2 += U * U;
    out[(int64_t)(1 + a) * plane + i] = W * U / rho;
  }
  out[i] = -W * u2 / (2.0 * rho * rho);
  out[(int64_t)(D + 1) * plane + i] = 0.0;
}

}  // namespace

bool launch_vjp(int D, int N, const AdjArgs& A, cudaStream_t s, cudaError_t& err) {
  err = cudaSuccess;
  return D == 2 ? vjp_dispatch<2>(N, A, s, err) : vjp_dispatch<3>(N, A, s, err);
}

bool launch_mortar_vjp(int D, int N, const MortarAdjArgs& A, cudaStream_t s) {
  return D == 2 ? mortar_vjp_dispatch<2>(N, A, s) : mortar_vjp_dispatch<3>(N, A, s);
}

cudaError_t launch_theta_state(int prec, int32_t E, int n1, int D, const double* bg,
                               const double* theta, double theta0, void* q, int64_t plane,
                               cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (prec == 0)
    theta_state_kernel<double><<<blocks, 256, 0, s>>>(total, NP, n1, D, bg, theta, theta0, (double*)q, plane);
  else
    theta_state_kernel<float><<<blocks, 256, 0, s>>>(total, NP, n1, D, bg, theta, theta0, (float*)q, plane);
  return cudaGetLastError();
}

cudaError_t launch_theta_vjp(int32_t E, int n1, int D, const double* bg, const double* theta,
                             double theta0, const double* lam_q, double* lam_theta, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  theta_vjp_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, NP, n1, D, bg, theta,
                                                                   theta0, lam_q, lam_theta);
  return cudaGetLastError();
}

cudaError_t launch_ke_grad(int32_t E, int n1, int D, const int32_t* elem, const double* w,
                          const double* root_h, const double* bg, const double* q, int64_t plane,
                          double* out, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  ke_grad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, NP, n1, D, elem, w, root_h[0],
                                                                 root_h[1], root_h[2], bg, q, plane, out);
  return cudaGetLastError();
}

}  // namespace dgk
