// Tracer kernels (dg_tracer.cuh) instantiated for N = 1..8, plus the tracer's initial cosine
// bell, refinement indicator and compensated total.
#include "dg_launch.hpp"
#include "dg_tracer.cuh"

namespace dgk {
namespace {

template <int N>
void run_tracer(const TracerArgs& A, cudaStream_t s) {
  constexpr int NP = (N + 1) * (N + 1);
  constexpr int EPB = epb_node(2, N);
  const unsigned blocks = (unsigned)((A.E + EPB - 1) / EPB);
  if (blocks) tracer_stage_kernel<N, EPB><<<blocks, EPB * NP, 0, s>>>(A);
}

template <int N>
void run_tracer_mortar(const TracerMortarArgs& A, cudaStream_t s) {
  if (A.G) tracer_mortar_kernel<N><<<A.G, 2 * (N + 1), 0, s>>>(A);
}

// C = amp (1 + cos(pi r)) for r <= 1, r = |(x - center) / radius| (Eq. "cosine-bell").
__global__ void tracer_bell_kernel(int32_t E, int n1, const int32_t* elem, const double* xi,
                                   double rx, double ry, double cx, double cy, double sx,
                                   double sy, double amp, double* C) {
  const int NP = n1 * n1;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)E * NP) return;
  const int64_t e = k / NP;
  const int n = (int)(k - e * NP);
  const double root_h[2] = {rx, ry};
  double x, y;
  tracer_xy(elem, e, xi, root_h, n % n1, n / n1, &x, &y);
  const double dx = (x - cx) / sx, dy = (y - cy) / sy;
  const double r = sqrt(dx * dx + dy * dy);
  C[k] = r <= 1.0 ? amp * (1.0 + cos(M_PI * r)) : 0.0;
}

__global__ void tracer_indicator_kernel(int32_t E, int NP, const double* C, double* out) {
  const int64_t e = blockIdx.x;
  __shared__ double red[128];
  double mx = 0.0;
  for (int n = threadIdx.x; n < NP; n += blockDim.x) mx = fmax(mx, fabs(C[e * NP + n]));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = red[0];
}

struct Neu {   // Neumaier-compensated sum
  double s, c;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
};

constexpr int kTotBlocks = 304, kTotThreads = 256;

// Per block: Neumaier sums of w_i w_j |J| C and of w_i w_j |J|, then a fixed tree.
__global__ void __launch_bounds__(kTotThreads)
tracer_total_partial(int32_t E, int n1, const int32_t* elem, const double* w, double rx, double ry,
                     const double* C, double* partial, int* bad) {
  const int NP = n1 * n1;
  Neu a{0.0, 0.0}, v{0.0, 0.0};
  int nonfinite = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (int64_t)E * NP;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = k / NP;
    const int n = (int)(k - e * NP);
    const int level = elem[e * 4];
    const double J = (ldexp(rx, -level) * 0.5) * (ldexp(ry, -level) * 0.5);
    const double W = w[n % n1] * w[n / n1] * J;
    if (!isfinite(C[k])) nonfinite = 1;
    a.add(W * C[k]);
    v.add(W);
  }
  if (nonfinite) atomicOr(bad, 1);
  __shared__ double s0[kTotThreads], c0[kTotThreads], s1[kTotThreads], c1[kTotThreads];
  const int t = threadIdx.x;
  s0[t] = a.s; c0[t] = a.c; s1[t] = v.s; c1[t] = v.c;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (t < st) {
      Neu x{s0[t], c0[t]}; x.add(s0[t + st]); x.c += c0[t + st]; s0[t] = x.s; c0[t] = x.c;
      Neu y{s1[t], c1[t]}; y.add(s1[t + st]); y.c += c1[t + st]; s1[t] = y.s; c1[t] = y.c;
    }
    __syncthreads();
  }
  if (t == 0) {
    partial[blockIdx.x * 4 + 0] = s0[0]; partial[blockIdx.x * 4 + 1] = c0[0];
    partial[blockIdx.x * 4 + 2] = s1[0]; partial[blockIdx.x * 4 + 3] = c1[0];
  }
}

__global__ void tracer_total_final(int nblocks, const double* partial, double* out) {
  const int k = threadIdx.x;
  if (k >= 2) return;
  Neu a{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) { a.add(partial[b * 4 + 2 * k]); a.c += partial[b * 4 + 2 * k + 1]; }
  out[k] = a.s + a.c;
}

}  // namespace

bool launch_tracer_stage(int N, const TracerArgs& A, cudaStream_t s) {
  switch (N) {
    case 1: run_tracer<1>(A, s); return true;
    case 2: run_tracer<2>(A, s); return true;
    case 3: run_tracer<3>(A, s); return true;
    case 4: run_tracer<4>(A, s); return true;
    case 5: run_tracer<5>(A, s); return true;
    case 6: run_tracer<6>(A, s); return true;
    case 7: run_tracer<7>(A, s); return true;
    case 8: run_tracer<8>(A, s); return true;
    default: return false;
  }
}

bool launch_tracer_mortar(int N, const TracerMortarArgs& A, cudaStream_t s) {
  switch (N) {
    case 1: run_tracer_mortar<1>(A, s); return true;
    case 2: run_tracer_mortar<2>(A, s); return true;
    case 3: run_tracer_mortar<3>(A, s); return true;
    case 4: run_tracer_mortar<4>(A, s); return true;
    case 5: run_tracer_mortar<5>(A, s); return true;
    case 6: run_tracer_mortar<6>(A, s); return true;
    case 7: run_tracer_mortar<7>(A, s); return true;
    case 8: run_tracer_mortar<8>(A, s); return true;
    default: return false;
  }
}

cudaError_t launch_tracer_bell(int32_t E, int n1, const int32_t* elem, const double* xi,
                               const double* root_h, const double* center, const double* radius,
                               double amp, double* C, cudaStream_t s) {
  const int64_t total = (int64_t)E * n1 * n1;
  if (total == 0) return cudaSuccess;
  tracer_bell_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      E, n1, elem, xi, root_h[0], root_h[1], center[0], center[1], radius[0], radius[1], amp, C);
  return cudaGetLastError();
}

cudaError_t launch_tracer_indicator(int32_t E, int n1, const double* C, double* out, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  tracer_indicator_kernel<<<E, 128, 0, s>>>(E, n1 * n1, C, out);
  return cudaGetLastError();
}

size_t tracer_total_scratch_doubles() { return (size_t)kTotBlocks * 4; }

cudaError_t launch_tracer_total(int32_t E, int n1, const int32_t* elem, const double* w,
                                const double* root_h, const double* C, double* partial, int* bad,
                                double* out, cudaStream_t s) {
  tracer_total_partial<<<kTotBlocks, kTotThreads, 0, s>>>(E, n1, elem, w, root_h[0], root_h[1], C,
                                                          partial, bad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tracer_total_final<<<1, 32, 0, s>>>(kTotBlocks, partial, out);
  return cudaGetLastError();
}

}  // namespace dgk
