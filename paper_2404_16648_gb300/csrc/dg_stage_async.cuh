// Column-mapped fused stage kernel with asynchronous staging (layout 2).
//
// Same operator and thread layout as stage_kernel_col (one thread per vertical node column),
// but every global read of the CTA is issued up front as cp.async copies into shared memory:
// the element's state and P' planes (contiguous, 16-byte chunks), its background column, the
// neighbour traces of its conforming faces and the mortar fluxes of its hanging faces.  The
// column's q^n values (Shu-Osher combination) are loaded into registers before the face terms
// and consumed at the end.  The computation runs from shared memory, so a CTA waits on memory
// once instead of once per dependent load chain, and the resident CTAs of an SM overlap one
// another's copies with their arithmetic.  One horizontal flux tile serves both horizontal
// axes (the y fluxes are recomputed from the staged state), which keeps the CTA at 32 KB.
#pragma once
#include "dg_stage_col.cuh"

namespace dgk {

__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Waits until at most one committed group of this thread is still in flight.
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copies `count` elements of T from a global run to shared memory with the threads
// [tid0, tid0 + nthr) of the CTA; 16-byte copies when both ends allow it.
template <class T>
__device__ __forceinline__ void stage_run(T* dst, const T* src, int count, int lane, int nthr) {
  constexpr int per16 = 16 / sizeof(T);
  const bool aligned = ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) == 0 && (count % per16) == 0;
  if (aligned) {
    for (int c = lane; c < count / per16; c += nthr) cp_async_bytes(dst + c * per16, src + c * per16, 16);
  } else {
    for (int c = lane; c < count; c += nthr) cp_async_bytes(dst + c, src + c, (int)sizeof(T));
  }
}

// Shared memory of the asynchronous kernel per CTA (bytes), per element:
//   region A  max(one horizontal flux tile, face lifts)
//   sQ        (NV + 1) x NP     state and P'
//   sNb       2d x (NV + 1) x NF  neighbour traces / mortar fluxes per face
//   sBg       n1 x 4            background column (T)
//   sBc       n1 doubles        gamma p_bar / Theta_bar per z-level (FP32 path's P')
// plus the derivative matrix once.
template <class T, int D, int N>
__host__ __device__ constexpr int async_region_a() {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2, NT = D - 1;
  constexpr int tile = NV * NP;
  constexpr int lifts = 2 * NT * NV * NF;
  return ((tile > lifts ? tile : lifts) + 3) / 4 * 4;
}
template <class T, int D, int N>
__host__ __device__ constexpr int async_elem_words() {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  return async_region_a<T, D, N>() + ((NV + 1) * NP + 3) / 4 * 4 + (2 * D * (NV + 1) * NF + 3) / 4 * 4 + n1 * 4 +
         ((n1 * (int)(8 / sizeof(T))) + 3) / 4 * 4;
}
template <class T, int D, int N, int EPB>
__host__ __device__ constexpr size_t async_smem_bytes() {
  return sizeof(T) * ((size_t)EPB * async_elem_words<T, D, N>() + (size_t)(N + 1) * (N + 1));
}

// Body for the EPB elements e0, e0 + 1, ... of mesh A.
template <class T, int D, int N, int EPB>
__device__ __forceinline__ void stage_body_async(const StageArgs& A, int64_t e0) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  constexpr int NT = D - 1;
  constexpr int RA = async_region_a<T, D, N>();
  constexpr int RQ = ((NV + 1) * NP + 3) / 4 * 4;
  constexpr int RN = (2 * D * (NV + 1) * NF + 3) / 4 * 4;
  constexpr int EW = async_elem_words<T, D, N>();
  constexpr bool VEC = (sizeof(T) == 4) && (n1 % 4 == 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int le = tid / NF, t = tid - le * NF;
  T* base = reinterpret_cast<T*>(smem_raw) + le * EW;
  T* sA = base;                       // one horizontal flux tile; later the lifts [2NT][NV][NF]
  T* sQ = base + RA;                  // [NV + 1][NP]
  T* sNb = base + RA + RQ;            // [2D][NV + 1][NF]
  T* sBg = base + RA + RQ + RN;       // [n1][4]
  double* sBc = reinterpret_cast<double*>(sBg + n1 * 4);   // [n1] (FP32 path)
  T* sDh = reinterpret_cast<T*>(smem_raw) + EPB * EW;
  const int64_t e = e0 + le;
  // threads beyond EPB columns (a persistent block of a fixed size) only take part in the
  // barriers and write no shared memory
  const bool inblk = le < EPB;
  const bool valid = inblk && e < A.E;
  const int ci = t % n1, cj = (D == 3) ? t / n1 : 0;
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + (valid ? e : 0) * NP;
  // ---- stage 1: own state, P', background column (contiguous runs)
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) stage_run<T>(sQ + v * NP, qe + v * P, NP, t, NF);
    stage_run<T>(sQ + NV * NP, (const T*)A.pp_in + e * NP, NP, t, NF);
    stage_run<T>(sBg, (const T*)A.bgt + e * n1 * 4, n1 * 4, t, NF);
    if (sizeof(T) == 4) stage_run<double>(sBc, A.bgc + e * n1, n1, t, NF);
  }
  const T* ops = (const T*)A.ops;
  for (int x = tid; x < n1 * n1; x += blockDim.x) sDh[x] = ops[x];
  // ---- neighbour traces of conforming faces, mortar fluxes of hanging faces
  int kinds[2 * D];
  if (valid) {
#pragma unroll
    for (int f = 0; f < 2 * D; ++f) {
      const int32_t* c = A.conn + ((size_t)e * 2 * D + f) * 5;
      const int kind = c[0];
      kinds[f] = kind;
      const int a = f >> 1, s = f & 1;
      T* dst = sNb + f * (NV + 1) * NF;
      if (kind == FACE_CONF) {
        const int no = face_node<D, N>(a, 1 - s, t);
        const T* qb = (const T*)A.qs + (int64_t)c[1] * NP;
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + t, qb + v * P + no, (int)sizeof(T));
        cp_async_bytes(dst + NV * NF + t, (const T*)A.pp_in + (int64_t)c[1] * NP + no, (int)sizeof(T));
      } else if (kind == FACE_FINE || kind == FACE_COARSE) {
        // launched as the programmatic dependent of this stage's mortar kernel: only the
        // elements that read its fluxes wait for it, before they read them
        if (A.after_mortar) asm volatile("griddepcontrol.wait;\n" ::: "memory");
        const int64_t gg = (kind == FACE_FINE) ? c[2] : c[1];
        const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
        const T* src = (const T*)A.mbuf + (((size_t)gg * (1 + NSUB) + slot) * NV) * NF;
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + t, src + v * NF + t, (int)sizeof(T));
      }
    }
  }
  cp_async_commit();
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  const T g = sizeof(T) == 4 ? (T)A.gf : (T)A.ph.g;
  T inv2h[D];
  const int level = valid ? A.elem[e * 4] : 0;
#pragma unroll
  for (int a = 0; a < D; ++a) inv2h[a] = valid ? inv2h_of<T>(A, level, a) : (T)0;
  cp_async_wait_all();
  __syncthreads();
  // ---- column fluxes; horizontal ones to the tiles, the vertical one kept in registers
  T acc[NV][n1];
  T Fz[NV][n1];
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    const int n = t + NF * k;
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = valid ? sQ[v * NP + n] : (T)0;
    const T pp = valid ? sQ[NV * NP + n] : (T)0;
    const NodeBg<T> bg = valid ? NodeBg<T>{sBg[k * 4], sBg[k * 4 + 1], sBg[k * 4 + 2]}
                               : NodeBg<T>{(T)1, (T)1, (T)1};
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v][k] = (T)0;
    acc[D][k] = -(q[0] * g);               // buoyancy -rho' g on the vertical momentum
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    T F[NV];
    flux_axis<T, D>(q, nd, pp, 0, F);
    if (inblk) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sA[v * NP + n] = F[v];
    }
    flux_axis<T, D>(q, nd, pp, D - 1, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fz[v][k] = F[v];
  }
  if constexpr (n1 % 2 == 0) {
    // the whole vertical line is this thread's: the even/odd split of the antisymmetric
    // derivative, 2 K2^2 multiply-adds and 2 n1 adds per line instead of n1^2 multiply-adds
    constexpr int K2 = n1 / 2;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T Ev[K2], Ov[K2];
#pragma unroll
      for (int m = 0; m < K2; ++m) {
        Ev[m] = add_rn(Fz[v][m], Fz[v][N - m]);
        Ov[m] = sub_rn(Fz[v][m], Fz[v][N - m]);
      }
#pragma unroll
      for (int i = 0; i < K2; ++i) {
        T se = (T)0, so = (T)0;
#pragma unroll
        for (int m = 0; m < K2; ++m) {
          se = fma(dtab_eo<T>(dtab_offset(N) + i * K2 + m), Ev[m], se);
          so = fma(dtab_eo<T>(dtab_offset(N) + K2 * K2 + i * K2 + m), Ov[m], so);
        }
        acc[v][i] = fma(-inv2h[D - 1], add_rn(se, so), acc[v][i]);
        acc[v][N - i] = fma(-inv2h[D - 1], sub_rn(so, se), acc[v][N - i]);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < n1; ++k) {
        T s = (T)0;
#pragma unroll
        for (int m = 0; m < n1; ++m) s = fma(dtab<T>(dtab_offset(N) + k * n1 + m), Fz[v][m], s);
        acc[v][k] = fma(-inv2h[D - 1], s, acc[v][k]);
      }
  }
  __syncthreads();
  // acc + sum_m Dr[m] row[m], the rows Dr already scaled by -2/h
  auto line_dot = [&](const T* row, const T* Dr, T s) {
    if constexpr (VEC) {
#pragma unroll
      for (int m = 0; m < n1; m += 4) {
        const float4 f = *reinterpret_cast<const float4*>(row + m);
        s = fma(Dr[m], (T)f.x, s);
        s = fma(Dr[m + 1], (T)f.y, s);
        s = fma(Dr[m + 2], (T)f.z, s);
        s = fma(Dr[m + 3], (T)f.w, s);
      }
    } else {
#pragma unroll
      for (int m = 0; m < n1; ++m) s = fma(Dr[m], row[m], s);
    }
    return s;
  };
  if (valid) {
    T Dr[n1];
#pragma unroll
    for (int m = 0; m < n1; ++m) Dr[m] = mul_rn(-inv2h[0], sDh[ci * n1 + m]);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < n1; ++k) acc[v][k] = line_dot(&sA[v * NP + NF * k + n1 * cj], Dr, acc[v][k]);
  }
  if (D == 3) {
    // y fluxes recomputed from the staged state into the same tile, transposed so that the
    // y lines are contiguous
    __syncthreads();
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      const int n = t + NF * k;
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = valid ? sQ[v * NP + n] : (T)0;
      const T pp = valid ? sQ[NV * NP + n] : (T)0;
      const NodeBg<T> bg = valid ? NodeBg<T>{sBg[k * 4], sBg[k * 4 + 1], sBg[k * 4 + 2]}
                                 : NodeBg<T>{(T)1, (T)1, (T)1};
      T F[NV];
      flux_axis<T, D>(q, node_der<T, D>(q, bg), pp, 1, F);
      if (inblk) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sA[v * NP + NF * k + n1 * ci + cj] = F[v];
      }
    }
    __syncthreads();
    if (valid) {
      T Dr[n1];
#pragma unroll
      for (int m = 0; m < n1; ++m) Dr[m] = mul_rn(-inv2h[1], sDh[cj * n1 + m]);
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < n1; ++k) acc[v][k] = line_dot(&sA[v * NP + NF * k + n1 * ci], Dr, acc[v][k]);
    }
  }
  __syncthreads();
  // ---- the tile is free for the lifts; q^n of this column is requested now and used last
  T* sLift = sA;                           // [2NT][NV][NF]
  const bool first = A.first != 0;
  T qn_col[NV][n1];
  if (valid && A.mode == 1 && !first) {
    const T* qne = (const T*)A.qn + e * NP;
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) qn_col[v][k] = qne[v * P + t + NF * k];
  }
  // ---- face terms, all operands in shared memory
  auto face_lift = [&](int a, int s, int fn, int own_node, int k, T* L) {
    const int f = 2 * a + s;
    const int kind = kinds[f];
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = sQ[v * NP + own_node];
    const T pp = sQ[NV * NP + own_node];
    const NodeBg<T> bg{sBg[k * 4], sBg[k * 4 + 1], sBg[k * 4 + 2]};
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    const T* nb = sNb + f * (NV + 1) * NF;
    T Fo[NV], Fs[NV];
    flux_axis<T, D>(q, nd, pp, a, Fo);
    if (kind == FACE_WALL || kind == FACE_CONF) {
      const T so = wave_speed<T>(q, nd, bg, pp, a, gamma);
      T qo[NV], Fn[NV], sn;
      if (kind == FACE_WALL) {
#pragma unroll
        for (int v = 0; v < NV; ++v) qo[v] = q[v];
        qo[1 + a] = -q[1 + a];
        flux_axis<T, D>(qo, nd, pp, a, Fn);
        sn = so;
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) qo[v] = nb[v * NF + fn];
        sn = face_side<T, D>(qo, bg, nb[NV * NF + fn], a, gamma, Fn);
      }
      if (s) rusanov<T, D>(q, Fo, so, qo, Fn, sn, Fs);
      else   rusanov<T, D>(qo, Fn, sn, q, Fo, so, Fs);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fs[v] = nb[v * NF + fn];
    }
    // the flux jump; its lift factor (2/h)/w0, signed by the side, is applied by the caller
#pragma unroll
    for (int v = 0; v < NV; ++v) L[v] = sub_rn(Fs[v], Fo[v]);
  };
  if (valid) {
#pragma unroll
    for (int a = 0; a < NT; ++a) {
      const int u = (D == 3) ? t % n1 : 0;
      const int k = (D == 3) ? t / n1 : t;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int ii, jj;
        if (a == 0) { ii = s ? N : 0; jj = u; } else { ii = u; jj = s ? N : 0; }
        T L[NV];
        face_lift(a, s, t, ii + n1 * jj + NF * k, k, L);
#pragma unroll
        for (int v = 0; v < NV; ++v) sLift[((2 * a + s) * NV + v) * NF + t] = L[v];
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int k = s ? N : 0;
      T L[NV];
      face_lift(D - 1, s, t, t + NF * k, k, L);
      const T coef = s ? -lift_of<T>(A, level, D - 1) : lift_of<T>(A, level, D - 1);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v][k] = fma(coef, L[v], acc[v][k]);
    }
  }
  __syncthreads();
  if (!valid) return;
#pragma unroll
  for (int a = 0; a < NT; ++a) {
    const int own = (a == 0) ? ci : cj;
    const int u = (a == 0) ? cj : ci;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (own != (s ? N : 0)) continue;
      const T coef = s ? -lift_of<T>(A, level, a) : lift_of<T>(A, level, a);
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < n1; ++k)
          acc[v][k] = fma(coef, sLift[((2 * a + s) * NV + v) * NF + (D == 3 ? u : 0) + (D == 3 ? n1 : 1) * k],
                          acc[v][k]);
    }
  }
  // ---- output
  T* oute = (T*)A.out + e * NP;
  if (A.mode == 0) {
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) oute[v * P + t + NF * k] = acc[v][k];
    return;
  }
  const StageCoef<T> scf = stage_coef<T>(A);
  const T dt = scf.dt, ca = scf.ca, cb = scf.cb;
  T* ppo = (T*)A.pp_out + e * NP;
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    const int n = t + NF * k;
    T qnew[NV];
    if (first) {   // uniform over the grid
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = fma(dt, acc[v][k], sQ[v * NP + n]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = fma(ca, qn_col[v][k], cb * fma(dt, acc[v][k], sQ[v * NP + n]));
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
    ppo[n] = pprime_of<T>(qnew[D + 1], sBg[k * 4 + 3], A.bg + ((size_t)e * n1 + k) * 4, sBc + k, A.ph);
  }
}

template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D - 1))
stage_kernel_async(const __grid_constant__ StageArgs A) {
  stage_body_async<T, D, N, EPB>(A, (int64_t)A.e_begin + (int64_t)blockIdx.x * EPB);
}

// Batched form: block b works on mesh tab[map[b].x], elements from map[b].y.
template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D - 1))
stage_kernel_async_batched(const StageArgs* __restrict__ tab, const int2* __restrict__ map) {
  const int2 bm = map[blockIdx.x];
  stage_body_async<T, D, N, EPB>(tab[bm.x], (int64_t)bm.y);
}

}  // namespace dgk
