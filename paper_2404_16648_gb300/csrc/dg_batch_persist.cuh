// Persistent batched stage kernel for 2D meshes (dg_batch_* entry points of include/dg.h).
//
// One launch per SSP-RK3 stage covers every 2D member of a batch, whatever its degree N and
// precision.  The host lists the stage's work as items in a device array: first the mortar
// items (2^(d-1) mortars of a group of hanging faces each, Sec. 3.3), then the stage items (a
// tile of elements of one member: volume term, face lifts, Shu-Osher combination, P').  A fixed
// grid of 128-thread CTAs, sized to what stays resident, takes items in order from an atomic
// counter until the array is exhausted.  Item codes select the body: the node-per-thread
// layout (layout 1 of the single-mesh kernels), the column layout with asynchronous staging
// (layout 2) or, for FP64 members, that layout reading the Rusanov fluxes of conforming and
// wall faces from a face buffer (layout 5), instantiated for N = 1..8; a tile is the elements
// one pass of that body covers, and an item holds `count` elements (a multiple of the tile).
// A layout-5 member also has face items, queued with the mortar items: `count` face slots, one
// thread per face node, the arithmetic of face_kernel.
//
// A stage item reads the mortar fluxes (and, in layout 5, the face fluxes) of its member, which
// the member's mortar and face items write in the same launch.  Each member has a counter of
// mortar groups and face slots done: a mortar or face item adds its count after its writes are
// fenced, and a CTA that takes a stage item waits (thread 0, with an iteration limit) until its
// member's count is complete.  This cannot deadlock: items are
// taken in array order, so every mortar item of the member was taken earlier by a CTA that is
// running and that waits for nothing.  If the limit runs out the kernel records it in
// `status` and goes on (the host reports DG_ERR_TIMEOUT); the results are then not valid.
//
// The per-element arithmetic is that of the single-mesh kernels (same bodies, same rounding,
// the unit compiled without implicit contraction), so a member advanced in the batch gets the
// bits it gets from dg_step with the same layout.
#pragma once
#include <type_traits>

#include "dg_face.cuh"
#include "dg_launch.hpp"
#include "dg_stage_async.cuh"
#include "dg_stage_fb.cuh"

namespace dgk {

constexpr int kBatchThreads = 128;
// spins of __nanosleep(64) before a wait for mortar fluxes gives up (of the order of a second)
constexpr int kBatchSpinLimit = 1 << 23;

// Item code: bits 0-1 kind (0 mortar, 1 stage, 2 face), bits 2-3 layout (0 node, 1 column-async,
// 2 column-async with the face buffer, FP64 only), bit 4 precision (0 FP64, 1 FP32), bits 5.. N.
__host__ __device__ constexpr int batch_code(int kind, int layout, int prec32, int N) {
  return kind | (layout << 2) | (prec32 << 4) | (N << 5);
}

// Elements per pass of the node layout in a 128-thread CTA (NP = (N+1)^2 threads each).
__host__ __device__ constexpr int batch_epb_node(int N) {
  return (N + 1) * (N + 1) >= kBatchThreads ? 1 : kBatchThreads / ((N + 1) * (N + 1));
}
// Elements per pass of the column layout (N + 1 threads each).
__host__ __device__ constexpr int batch_epb_col(int N) { return kBatchThreads / (N + 1); }
// Mortar groups per pass (2 (N + 1) threads each).
__host__ __device__ constexpr int batch_gpb(int N) { return kBatchThreads / (2 * (N + 1)); }
// Face slots per pass of a face item (N + 1 threads each).
__host__ __device__ constexpr int batch_fpb(int N) { return kBatchThreads / (N + 1); }

struct BatchArgs {
  const int4* items;         // {code, member, first element / group, count}
  int32_t nitems;
  const StageArgs* stage;    // per member: the stage's arguments
  const MortarArgs* mortar;  // per member: the stage's mortar arguments
  const FaceArgs* face;      // per member: the stage's face-kernel arguments (layout 5)
  const int32_t* need;       // per member: mortar groups, plus face slots in layout 5
  int32_t* fetch;            // item counter of this stage (zero before the launch)
  int32_t* done;             // per member: mortar groups finished in this stage (zero before)
  int32_t* status;           // set to 1 when a wait for mortar fluxes ran out
};

// Dynamic shared memory of one mortar pass: P and C (2 x (N+1)^2 each), then per group the
// coarse trace, the projected traces and the mortar states ([NV][N+1] blocks: 1 + 2 + 2).
template <class T, int N>
__host__ __device__ constexpr size_t batch_mortar_smem_bytes() {
  return sizeof(T) * ((size_t)4 * (N + 1) * (N + 1) + (size_t)batch_gpb(N) * 5 * 4 * (N + 1));
}

// Mortar groups g0 .. gend-1 (at most batch_gpb(N) of them) of a 2D mesh: the arithmetic of
// mortar_kernel (projection of the coarse trace onto the two mortars, Rusanov flux at the mortar
// nodes with the fine side's background, fluxes to the fine sides, back-projection
// sum_m C_m F*_m to the coarse side), with the groups of a pass side by side in the CTA and
// every barrier taken by all threads.
template <class T, int N>
__device__ __forceinline__ void mortar_pass_2d(const MortarArgs& A, int64_t g0, int64_t gend) {
  constexpr int D = 2, n1 = N + 1, NP = n1 * n1, NF = n1, NV = D + 2, NSUB = 2;
  constexpr int TPG = NSUB * NF, GPB = batch_gpb(N), GW = NV * NF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);   // [2][n1 * n1]
  T* sC = sP + 2 * n1 * n1;                  // [2][n1 * n1]
  const int tid = threadIdx.x;
  const int lg = tid / TPG, r = tid - lg * TPG;
  const int m = r / NF, t = r - m * NF;
  const int64_t g = g0 + lg;
  const bool active = lg < GPB && g < gend;
  T* sQc = sC + 2 * n1 * n1 + (lg < GPB ? lg : 0) * 5 * GW;   // [NV][NF]
  T* sT = sQc + GW;                                           // [NSUB][NV][NF]
  T* sM = sT + 2 * GW;                                        // [NSUB][NV][NF]
  const T* ops = (const T*)A.ops;
  for (int i = tid; i < n1 * n1; i += blockDim.x) {
    sP[i] = ops[1 * n1 * n1 + i];
    sP[n1 * n1 + i] = ops[2 * n1 * n1 + i];
    sC[i] = ops[3 * n1 * n1 + i];
    sC[n1 * n1 + i] = ops[4 * n1 * n1 + i];
  }
  const T* qs = (const T*)A.qs;
  T qf[NV];
  NodeBg<T> bgf{(T)1, (T)1, (T)1};
  T invTbf = (T)1, ppf = (T)0;
  size_t zf = 0;
  int a = 0, side = 0;
  if (active) {
    const int32_t* row = A.groups + (size_t)g * 7;
    const int64_t ec = row[0];
    a = row[1];
    side = row[2];
    const int64_t ef = row[3 + m];
    const int nf = face_node<D, N>(a, 1 - side, t);
#pragma unroll
    for (int v = 0; v < NV; ++v) qf[v] = qs[(size_t)v * A.plane + (size_t)ef * NP + nf];
    const int kf = nf / n1;
    zf = (size_t)ef * n1 + kf;
    const T* bt = (const T*)A.bgt + zf * 4;
    bgf = NodeBg<T>{bt[0], bt[1], bt[2]};
    invTbf = bt[3];
    ppf = ((const T*)A.pp_in)[(size_t)ef * NP + nf];
    for (int i = r; i < NV * NF; i += TPG) {
      const int v = i / NF, tt = i - v * NF;
      sQc[v * NF + tt] = qs[(size_t)v * A.plane + (size_t)ec * NP + face_node<D, N>(a, side, tt)];
    }
  }
  __syncthreads();
  const int b0 = m & 1;
  if (active) {
    // coarse trace -> mortar m along the face's tangential axis
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T s = (T)0;
#pragma unroll
      for (int j = 0; j < n1; ++j) s = fma(sP[b0 * n1 * n1 + t * n1 + j], sQc[v * NF + j], s);
      sT[(m * NV + v) * NF + t] = s;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sM[(m * NV + v) * NF + t] = sT[(m * NV + v) * NF + t];
  }
  __syncthreads();
  if (active) {
    T qc[NV], Fs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) qc[v] = sM[(m * NV + v) * NF + t];
    const T ppc = pprime_of<T>(qc[D + 1], invTbf, A.bg + zf * 4, A.bgc + zf, A.ph);
    const T gamma = gamma_of<T>(A.ph, A.gammaf);
    T Ff[NV], Fc[NV];
    const T sf = face_side<T, D>(qf, bgf, ppf, a, gamma, Ff);
    const T sc = face_side<T, D>(qc, bgf, ppc, a, gamma, Fc);
    if (side) rusanov<T, D>(qc, Fc, sc, qf, Ff, sf, Fs);
    else      rusanov<T, D>(qf, Ff, sf, qc, Fc, sc, Fs);
    T* mb = (T*)A.mbuf + ((size_t)g * (1 + NSUB) * NV) * NF;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      mb[((size_t)(1 + m) * NV + v) * NF + t] = Fs[v];
      sM[(m * NV + v) * NF + t] = Fs[v];
    }
  }
  __syncthreads();
  if (active) {
    // back to the coarse face: C_m F*_m
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T s = (T)0;
#pragma unroll
      for (int j = 0; j < n1; ++j) s = fma(sC[b0 * n1 * n1 + t * n1 + j], sM[(m * NV + v) * NF + j], s);
      sT[(m * NV + v) * NF + t] = s;
    }
  }
  __syncthreads();
  if (active && m == 0) {
    T* mb = (T*)A.mbuf + ((size_t)g * (1 + NSUB) * NV) * NF;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = (T)0;
      for (int mm = 0; mm < NSUB; ++mm) acc += sT[(mm * NV + v) * NF + t];
      mb[(size_t)v * NF + t] = acc;
    }
  }
}

// A mortar item: `count` groups from `first`, in passes of batch_gpb(N); then the member's
// counter is advanced once every thread's flux stores are fenced.
template <class T, int N>
__device__ __noinline__ void batch_mortar_item(const BatchArgs& B, int member, int64_t first, int count) {
  const MortarArgs& A = B.mortar[member];
  const int64_t end = first + count;
  for (int64_t g0 = first; g0 < end; g0 += batch_gpb(N)) {
    mortar_pass_2d<T, N>(A, g0, end);
    __syncthreads();   // the next pass rewrites the shared traces
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(B.done + member, count);
}

// A face item: F* of face slots first .. first + count - 1 of a 2D FP64 member, one thread per
// face node, then the member's counter is advanced once every thread's stores are fenced.
template <int N>
__device__ __noinline__ void batch_face_item(const BatchArgs& B, int member, int64_t first, int count) {
  constexpr int NF = N + 1, FPB = batch_fpb(N);
  const FaceArgs& A = B.face[member];
  const int lf = threadIdx.x / NF, t = threadIdx.x - lf * NF;
  const int64_t end = first + count;
  for (int64_t s0 = first; s0 < end; s0 += FPB) {
    const int64_t slot = s0 + lf;
    if (lf < FPB && slot < end) face_flux_node<double, 2, N>(A, slot, t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(B.done + member, count);
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits, with an iteration limit, until every mortar group of the member is done.
__device__ __forceinline__ void batch_wait_mortars(const BatchArgs& B, int member) {
  if (threadIdx.x == 0) {
    const int need = B.need[member];
    if (need > 0) {
      int spins = 0;
      while (ld_acquire_gpu(B.done + member) < need) {
        // give up after the limit, or at once when another wait already gave up
        if (++spins > kBatchSpinLimit || ld_acquire_gpu(B.status) != 0) {
          atomicExch(B.status, 1);
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
}

// A stage item: elements first .. first + count - 1 of one member in passes of one tile
// (`first` is a multiple of the tile; the member's last item may end at its element count).
template <class T, int N, int LAYOUT>
__device__ __noinline__ void batch_stage_item(const StageArgs& A, int64_t first, int count) {
  constexpr int EPB = LAYOUT == 0 ? batch_epb_node(N) : batch_epb_col(N);
  static_assert(LAYOUT != 2 || std::is_same<T, double>::value, "the face-buffer layout is FP64 only");
  const int64_t end = first + count;
  for (int64_t e0 = first; e0 < end; e0 += EPB) {
    if constexpr (LAYOUT == 0) stage_body_node<T, 2, N, EPB>(A, e0);
    else if constexpr (LAYOUT == 1) stage_body_async<T, 2, N, EPB>(A, e0);
    else                       stage_body_fb<T, 2, N, EPB>(A, e0);
    __syncthreads();   // the next pass rewrites the shared tiles
  }
}

template <class T, int N>
__device__ __forceinline__ void batch_dispatch_n(const BatchArgs& B, int kind, int layout, int member,
                                                 int64_t first, int count) {
  if (kind == 0) {
    batch_mortar_item<T, N>(B, member, first, count);
  } else if (kind == 2) {
    if constexpr (std::is_same<T, double>::value) batch_face_item<N>(B, member, first, count);
  } else {
    batch_wait_mortars(B, member);
    if (layout == 0) batch_stage_item<T, N, 0>(B.stage[member], first, count);
    else if (layout == 1) batch_stage_item<T, N, 1>(B.stage[member], first, count);
    else if constexpr (std::is_same<T, double>::value) batch_stage_item<T, N, 2>(B.stage[member], first, count);
  }
}

template <class T>
__device__ __forceinline__ void batch_dispatch(const BatchArgs& B, int kind, int layout, int N, int member,
                                               int64_t first, int count) {
  switch (N) {
    case 1: batch_dispatch_n<T, 1>(B, kind, layout, member, first, count); break;
    case 2: batch_dispatch_n<T, 2>(B, kind, layout, member, first, count); break;
    case 3: batch_dispatch_n<T, 3>(B, kind, layout, member, first, count); break;
    case 4: batch_dispatch_n<T, 4>(B, kind, layout, member, first, count); break;
    case 5: batch_dispatch_n<T, 5>(B, kind, layout, member, first, count); break;
    case 6: batch_dispatch_n<T, 6>(B, kind, layout, member, first, count); break;
    case 7: batch_dispatch_n<T, 7>(B, kind, layout, member, first, count); break;
    case 8: batch_dispatch_n<T, 8>(B, kind, layout, member, first, count); break;
    default: break;
  }
}

// The persistent kernel: MINB is the register budget's occupancy target (launch bounds), one
// of the choices of dg_batch_autotune.
template <int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB) batch_stage_kernel(const __grid_constant__ BatchArgs B) {
  __shared__ int s_item;
  for (;;) {
    __syncthreads();   // every thread is done with the previous item's shared memory and s_item
    if (threadIdx.x == 0) s_item = atomicAdd(B.fetch, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= B.nitems) return;
    const int4 w = B.items[it];
    const int kind = w.x & 3, layout = (w.x >> 2) & 3, prec32 = (w.x >> 4) & 1, N = w.x >> 5;
    if (prec32) batch_dispatch<float>(B, kind, layout, N, w.y, (int64_t)w.z, w.w);
    else        batch_dispatch<double>(B, kind, layout, N, w.y, (int64_t)w.z, w.w);
  }
}

// Dynamic shared memory of the bodies per (precision, N, layout 0 node / 1 column / 2 mortar /
// 3 column with the face buffer); a launch takes the largest over the bodies its items use
// (face items use none).
template <class T, int N>
constexpr size_t batch_body_smem(int layout) {
  return layout == 0 ? node_smem_bytes<T, 2, N, batch_epb_node(N)>()
         : layout == 1 ? async_smem_bytes<T, 2, N, batch_epb_col(N)>()
         : layout == 3 ? fb_smem_bytes<T, 2, N, batch_epb_col(N)>()
                       : batch_mortar_smem_bytes<T, N>();
}

inline size_t batch_body_smem_any(int prec32, int N, int layout) {
  switch (N) {
#define DG_BATCH_SMEM_CASE(n) \
    case n: return prec32 ? batch_body_smem<float, n>(layout) : batch_body_smem<double, n>(layout);
    DG_BATCH_SMEM_CASE(1) DG_BATCH_SMEM_CASE(2) DG_BATCH_SMEM_CASE(3) DG_BATCH_SMEM_CASE(4)
    DG_BATCH_SMEM_CASE(5) DG_BATCH_SMEM_CASE(6) DG_BATCH_SMEM_CASE(7) DG_BATCH_SMEM_CASE(8)
#undef DG_BATCH_SMEM_CASE
    default: return 0;
  }
}

// The largest dynamic shared memory any body needs: the kernel's attribute is raised to it once
// per device, and each launch passes what its own items need.
inline size_t batch_smem_limit() {
  size_t mx = 0;
  for (int p = 0; p < 2; ++p)
    for (int N = 1; N <= 8; ++N)
      for (int l = 0; l < 4; ++l) {
        const size_t b = batch_body_smem_any(p, N, l);
        if (b > mx) mx = b;
      }
  return mx;
}

template <int MINB>
cudaError_t launch_batch(const BatchArgs& B, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = configure_kernel((const void*)batch_stage_kernel<MINB>, batch_smem_limit(), true);
  if (e != cudaSuccess) return e;
  if (grid <= 0 || B.nitems <= 0) return cudaSuccess;
  batch_stage_kernel<MINB><<<grid, kBatchThreads, smem, s>>>(B);
  return cudaGetLastError();
}

template <int MINB>
cudaError_t occupancy_batch(size_t smem, int* ctas_per_sm) {
  cudaError_t e = configure_kernel((const void*)batch_stage_kernel<MINB>, batch_smem_limit(), true);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, batch_stage_kernel<MINB>, kBatchThreads, smem);
}

}  // namespace dgk
