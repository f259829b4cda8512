// BR1 viscous kernels (FP64) for D = 2, 3 and N = 1..8.
#include "dg_launch.hpp"
#include "dg_viscous.cuh"

namespace dgk {
namespace {

// out[1 + c] += coef V[c] (momentum and Theta'), then P' of the updated Theta' when pp != null.
__global__ void visc_add_kernel(int64_t total, int NP, int n1, int D, const double* V, double coef,
                                double* out, int64_t plane, const double* bg, PhysC ph, double* pp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  for (int c = 0; c <= D; ++c) out[(int64_t)(1 + c) * plane + i] += coef * V[(int64_t)c * plane + i];
  if (pp) {
    const int64_t e = i / NP;
    const int n = (int)(i - e * NP);
    const int k = D == 3 ? n / (n1 * n1) : n / n1;
    const double* b = bg + (e * n1 + k) * 4;
    pp[i] = pressure_pert<kSeries>(out[(int64_t)(D + 1) * plane + i], b[3], b[2], ph);
  }
}


template <int D, int N>
void run_visc(const ViscArgs& A, int pass, cudaStream_t s) {
  constexpr int EPB = epb_node(D, N);
  if (A.G > 0)
    visc_mortar_kernel<D, N><<<A.G, (1 << (D - 1)) * ipow(N + 1, D - 1), 0, s>>>(A, pass);
  const unsigned blocks = (unsigned)((A.E + EPB - 1) / EPB);
  if (blocks) visc_pass_kernel<D, N, EPB><<<blocks, EPB * ipow(N + 1, D), 0, s>>>(A, pass);
}

template <int D>
bool visc_dispatch(int N, const ViscArgs& A, int pass, cudaStream_t s) {
  switch (N) {
    case 1: run_visc<D, 1>(A, pass, s); return true;
    case 2: run_visc<D, 2>(A, pass, s); return true;
    case 3: run_visc<D, 3>(A, pass, s); return true;
    case 4: run_visc<D, 4>(A, pass, s); return true;
    case 5: run_visc<D, 5>(A, pass, s); return true;
    case 6: run_visc<D, 6>(A, pass, s); return true;
    case 7: run_visc<D, 7>(A, pass, s); return true;
    case 8: run_visc<D, 8>(A, pass, s); return true;
    default: return false;
  }
}

}  // namespace

bool launch_viscous_pass(int D, int N, const ViscArgs& A, int pass, cudaStream_t s) {
  return D == 2 ? visc_dispatch<2>(N, A, pass, s) : visc_dispatch<3>(N, A, pass, s);
}

cudaError_t launch_visc_add(int32_t E, int n1, int D, const double* V, double coef, double* out,
                            int64_t plane, const double* bg, const PhysC& ph, double* pp,
                            cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  visc_add_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, NP, n1, D, V, coef, out,
                                                                  plane, bg, ph, pp);
  return cudaGetLastError();
}

}  // namespace dgk
