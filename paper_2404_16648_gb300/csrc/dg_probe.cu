// Arithmetic-rate probe: the rate of independent fused multiply-adds the SMs sustain, timed on
// the device with CUDA events.  It is the measured denominator for the rooflines of kernels
// bound by the FP64 (or FP32) pipe.
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_device.cuh"

namespace {

constexpr int kChains = 8;        // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  // the chains converge to b / (1 - a) = 1: the store never happens but keeps them live
  if (s < (T)-1) out[blockIdx.x] = s;
}

template <class T>
cudaError_t time_probe(int blocks, int iters, cudaStream_t s, float* ms) {
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters / 8, (T)0.999, (T)0.001);   // warm-up
    cudaEventRecord(e0, s);
    fma_probe_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return e;
}

__global__ void recip_sqrt_probe_kernel(int64_t n, const double* x, double* r, double* s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = dgk::recip(x[i]);
  s[i] = dgk::sqrt_fast(x[i]);
}

}  // namespace

extern "C" dg_status dg_probe_recip_sqrt(int64_t n, const double* x, double* rcp, double* sqrt_out,
                                         void* stream) {
  if (n < 0 || (n > 0 && (!x || !rcp || !sqrt_out))) return DG_ERR_ARG;
  if (n == 0) return DG_OK;
  recip_sqrt_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, x, rcp, sqrt_out);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

extern "C" dg_status dg_probe_fma_rate(int32_t precision, double* flop_per_s, void* stream) {
  if (!flop_per_s || (precision != DG_FP64 && precision != DG_FP32_PERT)) return DG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DG_ERR_CUDA;
  const int blocks = sms * kBlocksPerSM;
  // a few milliseconds of work at the expected rates (about 1.2 TFLOP/s FP64, 80 FP32)
  const int iters = precision == DG_FP64 ? 2048 : 65536;
  float ms = 0.f;
  const cudaError_t e = precision == DG_FP64
                            ? time_probe<double>(blocks, iters, (cudaStream_t)stream, &ms)
                            : time_probe<float>(blocks, iters, (cudaStream_t)stream, &ms);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  const double fmas = (double)blocks * kThreads * kChains * (double)iters;
  *flop_per_s = 2.0 * fmas / (ms * 1e-3);
  return DG_OK;
}
