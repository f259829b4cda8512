// Allocation-free domain integrals (entry point dg_integrals_noalloc of include/dg.h).
//
// Some callers cannot allocate device memory: code that runs while a CUDA stream is being
// captured into a graph (cudaMalloc is not capturable), host code whose device memory is owned
// by an external pool or arena, or real-time loops that must not enter the CUDA allocator.
// For them this unit computes the same integrals as dg_integrals from caller-owned inputs and
// outputs only: the leaf table, the state and the 5-double result are the caller's device
// buffers, the hydrostatic background is evaluated inline, the 1D quadrature rule travels in
// the kernel arguments, and the reduction scratch (one compensated partial sum per block and
// a non-finite flag) is the file-scope array g_noalloc_scratch below.  Nothing here calls
// cudaMalloc, cudaFree or any allocating library routine.
//
// The array is sized for kNoAllocMaxBlocks blocks of kNoAllocThreads threads with at most
// kNoAllocNodesPerThread nodes per thread: states above kNoAllocMaxNodes nodes are rejected.
// Every loaded GPU holds the array (about 160 KB) until the process exits.  All calls share
// it, so calls that overlap on the GPU (different streams, or host threads without ordering)
// race; calls on one stream are ordered and safe.  The array keeps the last call's contents;
// each call overwrites every partial it reads and clears the flag before use.
#include <cmath>
#include <map>
#include <mutex>

#include "../../include/dg.h"
#include "basis.hpp"
#include "dg_launch.hpp"

namespace dgk {
namespace {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocNodesPerThread = 128;
constexpr int64_t kNoAllocMaxNodes = (int64_t)kNoAllocMaxBlocks * kNoAllocThreads * kNoAllocNodesPerThread;
constexpr int kFlagSlot = kNoAllocMaxBlocks * NUM_INTEGRALS * 2;

// Reduction scratch: [block][integral][sum, compensation], then the non-finite flag.
static __device__ __align__(256) double g_noalloc_scratch[kFlagSlot + 32];

struct Rule {
  double x[DG_MAX_N + 1];   // LGL nodes
  double w[DG_MAX_N + 1];   // LGL weights
};

struct NComp {
  double s, c;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ void merge(const NComp& o) { add(o.s); c += o.c; }
};

__global__ void noalloc_clear(double* scratch) { scratch[kFlagSlot] = 0.0; }

// Same per-node quantities as integrals_partial (dg_misc.cu), with the background evaluated
// here instead of read from a table: pi = 1 - g z/(cp theta0), rho_bar = p0 pi^(cv/R)/(R theta0),
// Theta_bar = rho_bar theta0, p_bar = P(Theta_bar) (Sec. 2.1 EOS, Sec. 4.3 background).
template <class T>
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_partial(int64_t E, int n1, int D, const int32_t* elem, Rule rule, double rh0, double rh1,
                double rh2, const T* q, int64_t plane, PhysC ph, double* scratch) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = E * NP;
  NComp acc[NUM_INTEGRALS];
  for (int k = 0; k < NUM_INTEGRALS; ++k) acc[k] = NComp{0.0, 0.0};
  const double rh[3] = {rh0, rh1, rh2};
  bool nonfinite = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / NP;
    const int n = (int)(i - e * NP);
    const int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
    const int level = elem[e * 4];
    double wn = 1.0, J = 1.0, z = 0.0;
    for (int a = 0; a < D; ++a) {
      const double h = ldexp(rh[a], -level);
      wn = wn * rule.w[idx[a]];
      J = J * (h * 0.5);
      if (a == D - 1) z = (elem[e * 4 + 1 + a] + (rule.x[idx[a]] + 1.0) * 0.5) * h;
    }
    const double W = wn * J;
    const double pi = 1.0 - ph.g * z / (ph.cp * ph.theta0);
    const double rb = ph.p0 * pow(pi, ph.cv / ph.R) / (ph.R * ph.theta0);
    const double Tb = rb * ph.theta0;
    const double pb = ph.p0 * pow(ph.R * Tb / ph.p0, ph.gamma);
    const double rp = (double)q[i];
    const double rho = rb + rp;
    double u2 = 0.0;
    for (int a = 0; a < D; ++a) {
      const double U = (double)q[(int64_t)(1 + a) * plane + i];
      u2 = u2 + U * U;
    }
    const double ke = 0.5 * u2 / rho;
    const double tp = (double)q[(int64_t)(D + 1) * plane + i];
    const double p = pb + pressure_pert<kSeries>(tp, 1.0 / Tb, pb, ph);
    const double en = p * ph.cv / ph.R + ke + rho * ph.g * z;
    if (!isfinite(rho) || !isfinite(en)) nonfinite = true;
    acc[0].add(W * rho);
    acc[1].add(W * en);
    acc[2].add(W * ke);
    acc[3].add(W);
    acc[4].add(W * rp);
  }
  if (nonfinite) scratch[kFlagSlot] = 1.0;
  __shared__ double ss[NUM_INTEGRALS][kNoAllocThreads], sc[NUM_INTEGRALS][kNoAllocThreads];
  for (int k = 0; k < NUM_INTEGRALS; ++k) { ss[k][threadIdx.x] = acc[k].s; sc[k][threadIdx.x] = acc[k].c; }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < NUM_INTEGRALS; ++k) {
        NComp a{ss[k][threadIdx.x], sc[k][threadIdx.x]};
        a.merge(NComp{ss[k][threadIdx.x + s], sc[k][threadIdx.x + s]});
        ss[k][threadIdx.x] = a.s; sc[k][threadIdx.x] = a.c;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < NUM_INTEGRALS; ++k) {
      scratch[(blockIdx.x * NUM_INTEGRALS + k) * 2] = ss[k][0];
      scratch[(blockIdx.x * NUM_INTEGRALS + k) * 2 + 1] = sc[k][0];
    }
}

// Sums the block partials in block order; out[k] for k < 5, out[5] = 1 when a non-finite value
// was met.
__global__ void noalloc_final(int nblocks, const double* scratch, double* out) {
  const int k = threadIdx.x;
  if (k < NUM_INTEGRALS) {
    NComp a{0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
      a.merge(NComp{scratch[(b * NUM_INTEGRALS + k) * 2], scratch[(b * NUM_INTEGRALS + k) * 2 + 1]});
    out[k] = a.s + a.c;
  } else if (k == NUM_INTEGRALS) {
    out[k] = scratch[kFlagSlot];
  }
}

// Device address of the scratch array, looked up once per device with that device current.
cudaError_t scratch_address(double** out) {
  static std::mutex mu;
  static std::map<int, double*> addr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) { *out = it->second; return cudaSuccess; }
  double* p = nullptr;
  e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  addr[dev] = p;
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace dgk

extern "C" dg_status dg_integrals_noalloc(const dg_mesh_desc* desc, const int32_t* elem,
                                          int64_t num_elements, const void* q, double* out,
                                          void* stream) {
  if (!desc || !elem || !q || !out || num_elements < 0) return DG_ERR_ARG;
  if ((desc->dim != 2 && desc->dim != 3) || desc->N < 1 || desc->N > DG_MAX_N) return DG_ERR_ARG;
  if (desc->precision != DG_FP64 && desc->precision != DG_FP32_PERT) return DG_ERR_ARG;
  if (desc->equations != DG_EQ_EULER) return DG_ERR_UNSUPPORTED;
  const int D = desc->dim, n1 = desc->N + 1;
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  // beyond the static scratch (compared before multiplying, so no product can wrap)
  if (num_elements > dgk::kNoAllocMaxNodes / NP) return DG_ERR_ARG;
  const int64_t nodes = num_elements * NP;
  if (!(desc->cp > desc->R) || !(desc->R > 0.0) || !(desc->p0 > 0.0) || !(desc->theta0 > 0.0))
    return DG_ERR_ARG;
  for (int a = 0; a < D; ++a)
    if (desc->base[a] < 1 || !(desc->length[a] > 0.0)) return DG_ERR_ARG;
  // the neutral background exists below z = cp theta0 / g (the same rule as dg_mesh_create)
  if (desc->g > 0.0 && !(desc->length[D - 1] < desc->cp * desc->theta0 / desc->g)) return DG_ERR_ARG;
  double* scratch = nullptr;
  if (dgk::scratch_address(&scratch) != cudaSuccess) return DG_ERR_CUDA;
  dgk::PhysC ph{};
  ph.theta0 = desc->theta0; ph.p0 = desc->p0; ph.g = desc->g; ph.R = desc->R; ph.cp = desc->cp;
  ph.cv = desc->cp - desc->R; ph.gamma = desc->cp / ph.cv;
  double c = 1.0;
  for (int k = 1; k <= dgk::kSeries; ++k) { c = c * (ph.gamma - (k - 1)) / k; ph.binom[k - 1] = c; }
  dgk::Rule rule{};
  const dgl::Basis1D b = dgl::make_basis(desc->N);
  for (int i = 0; i < n1; ++i) { rule.x[i] = b.x[i]; rule.w[i] = b.w[i]; }
  double rh[3] = {1.0, 1.0, 1.0};
  for (int a = 0; a < D; ++a) rh[a] = desc->length[a] / desc->base[a];
  int64_t per_block = (int64_t)dgk::kNoAllocThreads * dgk::kNoAllocNodesPerThread;
  int nblocks = (int)((nodes + per_block - 1) / per_block);
  if (nblocks < 1) nblocks = 1;
  cudaStream_t s = (cudaStream_t)stream;
  dgk::noalloc_clear<<<1, 1, 0, s>>>(scratch);
  if (desc->precision == DG_FP64)
    dgk::noalloc_partial<double><<<nblocks, dgk::kNoAllocThreads, 0, s>>>(
        num_elements, n1, D, elem, rule, rh[0], rh[1], rh[2], (const double*)q, nodes, ph, scratch);
  else
    dgk::noalloc_partial<float><<<nblocks, dgk::kNoAllocThreads, 0, s>>>(
        num_elements, n1, D, elem, rule, rh[0], rh[1], rh[2], (const float*)q, nodes, ph, scratch);
  dgk::noalloc_final<<<1, 32, 0, s>>>(nblocks, scratch, out);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
