// Instantiates the stage and mortar kernels of one (precision, dimension) for N = 1..8.
// Included by stage_<prec>_<dim>.cu with DG_T and DG_D defined.
#include "dg_face.cuh"
#include "dg_launch.hpp"
#include "dg_stage_fb.cuh"
#include "dg_stage_half.cuh"
#include "dg_stage_line.cuh"

namespace dgk {
namespace {

template <class T, int D, int N>
void run_stage_node(const StageArgs& A, cudaStream_t s) {
  constexpr int NP = ipow(N + 1, D);
  constexpr int EPB = epb_node(D, N);
  constexpr size_t smem = node_smem_bytes<T, D, N, EPB>();
  const unsigned blocks = (unsigned)((A.E - A.e_begin + EPB - 1) / EPB);
  if (blocks) stage_kernel<T, D, N, EPB><<<blocks, EPB * NP, smem, s>>>(A);
}

template <class T, int D, int N>
cudaError_t run_stage_col(const StageArgs& A, cudaStream_t s) {
  constexpr int NF = ipow(N + 1, D - 1);
  constexpr int EPB = epb_col(D, N);
  constexpr size_t smem = col_smem_bytes<T, D, N, EPB>();
  {
    cudaError_t e = configure_kernel((const void*)stage_kernel_col<T, D, N, EPB>, smem, false);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((A.E - A.e_begin + EPB - 1) / EPB);
  if (blocks) stage_kernel_col<T, D, N, EPB><<<blocks, EPB * NF, smem, s>>>(A);
  return cudaSuccess;
}

// A column-mapped stage kernel (EPB elements per CTA, one thread per column), as the
// programmatic dependent of the kernel before it when A.after_mortar is set.
template <int D, int N, int EPB>
cudaError_t launch_col_kernel(void (*kernel)(StageArgs), size_t smem, const StageArgs& A, cudaStream_t s) {
  constexpr int NF = ipow(N + 1, D - 1);
  {
    cudaError_t e = configure_kernel((const void*)kernel, smem, false);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((A.E - A.e_begin + EPB - 1) / EPB);
  if (!blocks) return cudaSuccess;
  if (!A.after_mortar) {
    kernel<<<blocks, EPB * NF, smem, s>>>(A);
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(EPB * NF);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, A);
}

// Layout 2 (after the mortar kernel: see the hanging-face staging of stage_body_async).
template <class T, int D, int N>
cudaError_t run_stage_async(const StageArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_col(D, N);
  return launch_col_kernel<D, N, EPB>(stage_kernel_async<T, D, N, EPB>, async_smem_bytes<T, D, N, EPB>(), A, s);
}

// Layout 5 (after the face kernel: see the staging of stage_body_fb).
template <class T, int D, int N>
cudaError_t run_stage_fb(const StageArgs& A, cudaStream_t s) {
  constexpr int EPB = epb_col(D, N);
  return launch_col_kernel<D, N, EPB>(stage_kernel_fb<T, D, N, EPB>, fb_smem_bytes<T, D, N, EPB>(), A, s);
}

// Layout 3 (3D, odd N); other shapes take layout 2.
template <class T, int D, int N>
cudaError_t run_stage_half(const StageArgs& A, cudaStream_t s) {
  if constexpr (D == 3 && N % 2 == 1) {
    constexpr size_t smem = half_smem_bytes<T, N>();
    {
      cudaError_t e = configure_kernel((const void*)stage_kernel_half<T, N>, smem, false);
      if (e != cudaSuccess) return e;
    }
    if (A.E > A.e_begin)
      stage_kernel_half<T, N><<<(unsigned)(A.E - A.e_begin), HalfCfg<N>::THREADS, smem, s>>>(A);
    return cudaSuccess;
  } else {
    return run_stage_async<T, D, N>(A, s);
  }
}

// Layout 4 (3D, odd N); other shapes take layout 2.
template <class T, int D, int N>
cudaError_t run_stage_line(const StageArgs& A, cudaStream_t s) {
  if constexpr (D == 3 && N % 2 == 1) {
    constexpr size_t smem = line_smem_bytes<T, N>();
    {
      // all of the unified L1/shared capacity as shared memory: 7 CTAs of the FP32 N = 7 kernel
      cudaError_t e = configure_kernel((const void*)stage_kernel_line<T, N>, smem, true);
      if (e != cudaSuccess) return e;
    }
    if (A.E <= A.e_begin) return cudaSuccess;
    if (!A.after_mortar) {
      stage_kernel_line<T, N><<<(unsigned)(A.E - A.e_begin), LineCfg<N>::THREADS, smem, s>>>(A);
      return cudaSuccess;
    }
    // programmatic dependent launch after the mortar kernel (see stage_body_line)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(A.E - A.e_begin));
    cfg.blockDim = dim3(LineCfg<N>::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stage_kernel_line<T, N>, A);
  } else {
    return run_stage_async<T, D, N>(A, s);
  }
}

// Batched launch over many meshes: layout 1 (node) or 2 (column, asynchronous staging).
template <class T, int D, int N>
cudaError_t run_stage_batched(int layout, const StageArgs* tab, const int2* map, int nblocks,
                              cudaStream_t s) {
  if (layout == 1) {
    constexpr int EPB = epb_node(D, N);
    constexpr size_t smem = node_smem_bytes<T, D, N, EPB>();
    if (nblocks <= 0) return cudaSuccess;
    stage_kernel_batched<T, D, N, EPB><<<nblocks, EPB * ipow(N + 1, D), smem, s>>>(tab, map);
    return cudaGetLastError();
  }
  constexpr int NF = ipow(N + 1, D - 1);
  constexpr int EPB = epb_col(D, N);
  constexpr size_t smem = async_smem_bytes<T, D, N, EPB>();
  {   // done on the first call, also with nblocks == 0 (before a capture)
    cudaError_t e = configure_kernel((const void*)stage_kernel_async_batched<T, D, N, EPB>, smem, false);
    if (e != cudaSuccess) return e;
  }
  if (nblocks <= 0) return cudaSuccess;
  stage_kernel_async_batched<T, D, N, EPB><<<nblocks, EPB * NF, smem, s>>>(tab, map);
  return cudaGetLastError();
}

template <class T, int D>
cudaError_t batched_dispatch(int N, int layout, const StageArgs* tab, const int2* map, int nblocks,
                             cudaStream_t s) {
  switch (N) {
    case 1: return run_stage_batched<T, D, 1>(layout, tab, map, nblocks, s);
    case 2: return run_stage_batched<T, D, 2>(layout, tab, map, nblocks, s);
    case 3: return run_stage_batched<T, D, 3>(layout, tab, map, nblocks, s);
    case 4: return run_stage_batched<T, D, 4>(layout, tab, map, nblocks, s);
    case 5: return run_stage_batched<T, D, 5>(layout, tab, map, nblocks, s);
    case 6: return run_stage_batched<T, D, 6>(layout, tab, map, nblocks, s);
    case 7: return run_stage_batched<T, D, 7>(layout, tab, map, nblocks, s);
    case 8: return run_stage_batched<T, D, 8>(layout, tab, map, nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, int D, int N>
void run_stage(const StageArgs& A, cudaStream_t s) {
  if (A.variant == 1) run_stage_node<T, D, N>(A, s);
  else if (A.variant == 2) run_stage_async<T, D, N>(A, s);
  else if (A.variant == 3) run_stage_half<T, D, N>(A, s);
  else if (A.variant == 4) run_stage_line<T, D, N>(A, s);
  else if (A.variant == 5) run_stage_fb<T, D, N>(A, s);
  else run_stage_col<T, D, N>(A, s);
}

// Face kernel of layout 5 (dg_face.cuh); pdl: launched as the programmatic dependent of the
// mortar kernel just before it.
template <class T, int D, int N>
cudaError_t run_face(const FaceArgs& F, bool pdl, cudaStream_t s) {
  constexpr int FPB = face_per_block<D, N>();
  constexpr int NF = ipow(N + 1, D - 1);
  const int64_t n = (int64_t)F.C + F.B;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + FPB - 1) / FPB);
  if (!pdl) {
    face_kernel<T, D, N><<<blocks, FPB * NF, 0, s>>>(F);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(FPB * NF);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, face_kernel<T, D, N>, F);
}

template <class T, int D>
cudaError_t face_dispatch(int N, const FaceArgs& F, bool pdl, cudaStream_t s) {
  switch (N) {
    case 1: return run_face<T, D, 1>(F, pdl, s);
    case 2: return run_face<T, D, 2>(F, pdl, s);
    case 3: return run_face<T, D, 3>(F, pdl, s);
    case 4: return run_face<T, D, 4>(F, pdl, s);
    case 5: return run_face<T, D, 5>(F, pdl, s);
    case 6: return run_face<T, D, 6>(F, pdl, s);
    case 7: return run_face<T, D, 7>(F, pdl, s);
    case 8: return run_face<T, D, 8>(F, pdl, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T, int D, int N>
void run_mortar(const MortarArgs& A, cudaStream_t s) {
  if (A.G) mortar_kernel<T, D, N><<<A.G, (1 << (D - 1)) * ipow(N + 1, D - 1), 0, s>>>(A);
}

template <class T, int D>
bool stage_dispatch(int N, const StageArgs& A, cudaStream_t s) {
  switch (N) {
    case 1: run_stage<T, D, 1>(A, s); return true;
    case 2: run_stage<T, D, 2>(A, s); return true;
    case 3: run_stage<T, D, 3>(A, s); return true;
    case 4: run_stage<T, D, 4>(A, s); return true;
    case 5: run_stage<T, D, 5>(A, s); return true;
    case 6: run_stage<T, D, 6>(A, s); return true;
    case 7: run_stage<T, D, 7>(A, s); return true;
    case 8: run_stage<T, D, 8>(A, s); return true;
    default: return false;
  }
}

template <class T, int D>
bool mortar_dispatch(int N, const MortarArgs& A, cudaStream_t s) {
  switch (N) {
    case 1: run_mortar<T, D, 1>(A, s); return true;
    case 2: run_mortar<T, D, 2>(A, s); return true;
    case 3: run_mortar<T, D, 3>(A, s); return true;
    case 4: run_mortar<T, D, 4>(A, s); return true;
    case 5: run_mortar<T, D, 5>(A, s); return true;
    case 6: run_mortar<T, D, 6>(A, s); return true;
    case 7: run_mortar<T, D, 7>(A, s); return true;
    case 8: run_mortar<T, D, 8>(A, s); return true;
    default: return false;
  }
}

}  // namespace
}  // namespace dgk
