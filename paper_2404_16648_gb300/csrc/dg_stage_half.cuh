// Half-column fused stage kernel (layout 3; 3D, odd N so that N + 1 is even).
//
// The operator is the one of the other layouts: volume term of the strong form (Sec. 2.2) with
// the derivative applied along each axis, face lifts with the Rusanov flux on conforming faces
// and walls and the precomputed mortar fluxes on hanging faces (Sec. 3.3), the Shu-Osher
// combination and P' of the new state.  The thread mapping differs: two threads share each
// vertical node column, each owning (N+1)/2 of its nodes, so a CTA of one element has twice
// the threads of the column layout at the same shared memory and the SM holds twice the warps
// to hide load and pipeline latency.
//
// Mapping: 16 columns per warp; lane l of warp w works on column t = 16 w + (l & 15) and half
// h = l >> 4, i.e. the two halves of a column sit in lanes l and l ^ 16 of one warp.  Half 0
// owns rows k = 0 .. K2-1, half 1 rows N, N-1, .. K2 (row r of a thread is k = r or N - r), so
// the row of the thread's vertical face is r = 0 for both halves.  The vertical derivative
// exchanges the two halves' fluxes with one warp shuffle per value; each half applies a
// permuted copy of D (its output rows, own rows first) from shared memory, stored where layout
// 2 keeps D, so the CTA needs exactly the shared memory of layout 2.
//
// Bank layout for N + 1 = 8 (64-word k-slabs).  The two halves of a warp touch the same
// in-slab positions of two slabs of opposite parity, so the state, P' and the x-flux tile flip
// bit 4 of the word index in odd slabs (whole 8-word rows move, rows stay contiguous): the two
// half-warps then use disjoint banks.  The state also swaps the two 16-byte halves of rows
// j >= 4, which spreads the nodes of an x face over 8 banks instead of 4.  The transposed
// y-flux tile (row ci holds the y line) stores column cj at cj ^ 4 (ci >= 4) ^ 2 (odd slab),
// which spreads a warp's stores over all 32 banks; the y derivative applies D with the same
// permutation.  The D rows of the horizontal derivatives come from constant memory.
#pragma once
#include <type_traits>

#include "dg_stage_async.cuh"

namespace dgk {

template <int N>
struct HalfCfg {
  static constexpr int n1 = N + 1, NF = n1 * n1, NP = NF * n1, K2 = n1 / 2;
  static constexpr int THREADS = 32 * ((NF + 15) / 16);
};

// Shared memory: the per-element regions of the asynchronous kernel and the permuted D
// (2 halves x (N+1)/2 rows x (N+1) = (N+1)^2 entries, the size of D itself).
template <class T, int N>
__host__ __device__ constexpr size_t half_smem_bytes() {
  return async_smem_bytes<T, 3, N, 1>();
}

// Row k of half h's r-th output row.
template <int N>
__device__ __forceinline__ int half_row(int h, int r) { return h ? N - r : r; }

// Word index of natural node index n in the x-flux tile (N + 1 = 8: slab-parity flip) and in
// the staged state (additionally the 16-byte halves of rows j >= 4 swapped).
template <int N>
__device__ __forceinline__ int tile_swz(int n) {
  if constexpr (N == 7) return n ^ ((n >> 2) & 16);
  else return n;
}
template <int N>
__device__ __forceinline__ int half_swz(int n) {
  if constexpr (N == 7) return n ^ ((n >> 2) & 16) ^ ((n >> 3) & 4);
  else return n;
}

// Background row (rho_bar, Theta_bar, p_bar, 1/Theta_bar) of z-level k from shared memory.
__device__ __forceinline__ void load_bg_row(const float* sBg, int k, float* b) {
  const float4 v = *reinterpret_cast<const float4*>(sBg + k * 4);
  b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
}
__device__ __forceinline__ void load_bg_row(const double* sBg, int k, double* b) {
  const double2 v0 = *reinterpret_cast<const double2*>(sBg + k * 4);
  const double2 v1 = *reinterpret_cast<const double2*>(sBg + k * 4 + 2);
  b[0] = v0.x; b[1] = v0.y; b[2] = v1.x; b[3] = v1.y;
}

// Copies `count` words of T to shared memory at swizzled positions; 16-byte copies when both
// ends allow it (the swizzle keeps 4-word chunks together).
template <class T, int N>
__device__ __forceinline__ void stage_run_swz(T* dst, const T* src, int count, int lane, int nthr) {
  constexpr int per16 = 16 / sizeof(T);
  const bool aligned = ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) == 0 && (count % per16) == 0;
  if (aligned) {
    for (int c = lane; c < count / per16; c += nthr)
      cp_async_bytes(dst + half_swz<N>(c * per16), src + c * per16, 16);
  } else {
    for (int c = lane; c < count; c += nthr) cp_async_bytes(dst + half_swz<N>(c), src + c, (int)sizeof(T));
  }
}

template <class T, int N>
__device__ __forceinline__ void stage_body_half(const StageArgs& A, int64_t e) {
  constexpr int D = 3, n1 = N + 1, NP = ipow(n1, 3), NF = n1 * n1, NV = 5;
  constexpr int K2 = n1 / 2;
  constexpr int NSUB = 4;
  constexpr int THREADS = HalfCfg<N>::THREADS;
  constexpr int RA = async_region_a<T, D, N>();
  constexpr int RQ = ((NV + 1) * NP + 3) / 4 * 4;
  constexpr int RN = (2 * D * (NV + 1) * NF + 3) / 4 * 4;
  constexpr bool VEC = (sizeof(T) == 4) && (n1 % 4 == 0);
  static_assert(n1 % 2 == 0, "layout 3 needs an even number of nodes per line");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (e >= A.E) return;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int h = lane >> 4;
  const int t = 16 * (tid >> 5) + (lane & 15);
  const bool colok = t < NF;
  const int tc = colok ? t : 0;
  const int ci = tc % n1, cj = tc / n1;
  T* sA = reinterpret_cast<T*>(smem_raw);     // flux tile; later the horizontal lifts [4][NV][NF]
  T* sQ = sA + RA;                            // [NV + 1][NP]
  T* sNb = sA + RA + RQ;                      // [2D][NV + 1][NF]
  T* sBg = sA + RA + RQ + RN;                 // [n1][4]
  double* sBc = reinterpret_cast<double*>(sBg + n1 * 4);
  T* sDz = sA + async_elem_words<T, D, N>();  // [2][K2][n1]: per half, its output rows
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + e * NP;
  // ---- q^n of the Shu-Osher combination is read only in the epilogue: one thread asks the L2
  // for the element's planes now (bulk prefetch, no registers or shared memory held)
  if (tid == 0 && A.mode == 1 && !A.first) {
    const T* qne = (const T*)A.qn + e * NP;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* src = qne + (int64_t)v * P;
      if ((((uintptr_t)src) & 15) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"((int)(NP * sizeof(T)))
                     : "memory");
    }
  }
  // ---- own state, P', background column: contiguous runs over all threads
#pragma unroll
  for (int v = 0; v < NV; ++v) stage_run_swz<T, N>(sQ + v * NP, qe + v * P, NP, tid, THREADS);
  stage_run_swz<T, N>(sQ + NV * NP, (const T*)A.pp_in + e * NP, NP, tid, THREADS);
  stage_run<T>(sBg, (const T*)A.bgt + e * n1 * 4, n1 * 4, tid, THREADS);
  if (sizeof(T) == 4) stage_run<double>(sBc, A.bgc + e * n1, n1, tid, THREADS);
  const T* ops = (const T*)A.ops;
  for (int x = tid; x < 2 * K2 * n1; x += THREADS) {
    // sDz[hh][r][j]: output row k = half_row(hh, r); j < K2 the column of own row j, j >= K2
    // the column of the other half's row j - K2
    const int hh = x / (K2 * n1), r = (x / n1) % K2, j = x % n1;
    const int k = half_row<N>(hh, r);
    const int m = j < K2 ? half_row<N>(hh, j) : half_row<N>(1 - hh, j - K2);
    sDz[x] = ops[k * n1 + m];
  }
  // ---- neighbour data of the faces this thread evaluates: horizontal face item j = tid of
  // each axis (side j / NF, face node j % NF) and the vertical face (2, h) at column t
  const int hs = tid / NF, hfn = tid - hs * NF;     // horizontal item
  const bool hok = tid < 2 * NF;
  int kindH[2], kindV = FACE_WALL;
  auto stage_face = [&](int a, int s, int fn) -> int {
    const int f = 2 * a + s;
    const int32_t* c = A.conn + ((size_t)e * 2 * D + f) * 5;
    const int kind = c[0];
    T* dst = sNb + f * (NV + 1) * NF;
    if (kind == FACE_CONF) {
      const int no = face_node<D, N>(a, 1 - s, fn);
      const T* qb = (const T*)A.qs + (int64_t)c[1] * NP;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + fn, qb + v * P + no, (int)sizeof(T));
      cp_async_bytes(dst + NV * NF + fn, (const T*)A.pp_in + (int64_t)c[1] * NP + no, (int)sizeof(T));
    } else if (kind == FACE_FINE || kind == FACE_COARSE) {
      const int64_t gg = (kind == FACE_FINE) ? c[2] : c[1];
      const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
      const T* src = (const T*)A.mbuf + (((size_t)gg * (1 + NSUB) + slot) * NV) * NF;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + fn, src + v * NF + fn, (int)sizeof(T));
    }
    return kind;
  };
#pragma unroll
  for (int a = 0; a < 2; ++a) kindH[a] = hok ? stage_face(a, hs, hfn) : FACE_WALL;
  if (colok) kindV = stage_face(2, h, t);
  cp_async_commit();
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  const T g = sizeof(T) == 4 ? (T)A.gf : (T)A.ph.g;
  const int level = A.elem[e * 4];
  T inv2h[D];
#pragma unroll
  for (int a = 0; a < D; ++a) inv2h[a] = inv2h_of<T>(A, level, a);
  T lc[D];                                 // lift factors (2/h_a) / w0
#pragma unroll
  for (int a = 0; a < D; ++a) lc[a] = lift_of<T>(A, level, a);
  // F* - F(own) on face (a, s) at face node fn, given the own node's state and normal flux Fo;
  // returns the lift n_a (2/h_a)/w0 (F* - F(own)).
  auto face_lift = [&](auto axis, int s, int kind, int fn, const T* q, T pp, const NodeBg<T>& bg,
                       const NodeDer<T>& nd, const T* Fo, T* L) {
    constexpr int a = decltype(axis)::value;
    const T* nb = sNb + (2 * a + s) * (NV + 1) * NF;
    T Fs[NV];
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
    const T coef = s ? -lc[a] : lc[a];
#pragma unroll
    for (int v = 0; v < NV; ++v) L[v] = coef * (Fs[v] - Fo[v]);
  };
  cp_async_wait_all();
  __syncthreads();
  // ---- node fluxes of the thread's rows: x to the tile, z kept in registers; the row r = 0
  // lies on the thread's vertical face (bottom for half 0, top for half 1), whose lift is
  // taken here from the same registers
  T acc[NV][K2];
  T Fz[NV][K2];
#pragma unroll
  for (int r = 0; r < K2; ++r) {
    const int k = half_row<N>(h, r);
    const int nn = tc + NF * k;
    const int n = half_swz<N>(nn);
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = sQ[v * NP + n];
    const T pp = sQ[NV * NP + n];
    T b4[4];
    load_bg_row(sBg, k, b4);
    const NodeBg<T> bg{b4[0], b4[1], b4[2]};
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v][r] = (T)0;
    acc[D][r] = -(q[0] * g);               // buoyancy -rho' g on the vertical momentum
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    T F[NV];
    flux_axis<T, D>(q, nd, pp, 0, F);
    if (colok) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sA[v * NP + tile_swz<N>(nn)] = F[v];
    }
    flux_axis<T, D>(q, nd, pp, D - 1, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fz[v][r] = F[v];
    if (r == 0 && colok) {
      T L[NV];
      face_lift(std::integral_constant<int, 2>{}, h, kindV, t, q, pp, bg, nd, F, L);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v][0] += L[v];
    }
  }
  // ---- vertical derivative: the other half's fluxes by shuffle, permuted D rows from smem
  {
    T Fo[NV][K2];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int r = 0; r < K2; ++r) Fo[v][r] = __shfl_xor_sync(0xffffffffu, Fz[v][r], 16);
#pragma unroll
    for (int r = 0; r < K2; ++r) {
      T Dr[n1];
      const T* row = sDz + (h * K2 + r) * n1;
      if constexpr (VEC) {
#pragma unroll
        for (int j = 0; j < n1; j += 4) {
          const float4 d4 = *reinterpret_cast<const float4*>(row + j);
          Dr[j] = (T)d4.x; Dr[j + 1] = (T)d4.y; Dr[j + 2] = (T)d4.z; Dr[j + 3] = (T)d4.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < n1; ++j) Dr[j] = row[j];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T s = (T)0;
#pragma unroll
        for (int j = 0; j < K2; ++j) s = fma(Dr[j], Fz[v][j], s);
#pragma unroll
        for (int j = 0; j < K2; ++j) s = fma(Dr[K2 + j], Fo[v][j], s);
        acc[v][r] = fma(-inv2h[D - 1], s, acc[v][r]);
      }
    }
  }
  __syncthreads();
  auto d_at = [&](int k, int m) -> T { return dtab<T>(dtab_offset(N) + k * n1 + m); };
  auto line_dot = [&](const T* row, const T* Dr) {
    T s = (T)0;
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
  if (colok) {
    T Dr[n1];
#pragma unroll
    for (int m = 0; m < n1; ++m) Dr[m] = d_at(ci, m);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int r = 0; r < K2; ++r) {
        const int k = half_row<N>(h, r);
        acc[v][r] = fma(-inv2h[0], line_dot(&sA[v * NP + tile_swz<N>(NF * k + n1 * cj)], Dr), acc[v][r]);
      }
  }
  __syncthreads();
  // ---- y fluxes recomputed into the tile, transposed so that the y lines are contiguous
  if (colok) {
#pragma unroll
    for (int r = 0; r < K2; ++r) {
      const int k = half_row<N>(h, r);
      const int n = half_swz<N>(tc + NF * k);
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = sQ[v * NP + n];
      const T pp = sQ[NV * NP + n];
      T b4[4];
      load_bg_row(sBg, k, b4);
      const NodeBg<T> bg{b4[0], b4[1], b4[2]};
      T F[NV];
      flux_axis<T, D>(q, node_der<T, D>(q, bg), pp, 1, F);
      const int col = (N == 7) ? (cj ^ ((ci >> 2) << 2) ^ ((k & 1) << 1)) : cj;
#pragma unroll
      for (int v = 0; v < NV; ++v) sA[v * NP + NF * k + n1 * ci + col] = F[v];
    }
  }
  __syncthreads();
  if (colok) {
    // position p of a stored y line holds column p ^ G, G = 4 (ci >= 4) ^ 2 (odd slab)
    T Dr0[n1], Dr1[n1];
    const int g = (N == 7) ? ((ci >> 2) << 2) : 0;
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      Dr0[m] = d_at(cj, m ^ g);
      Dr1[m] = d_at(cj, (N == 7) ? (m ^ g ^ 2) : m);
    }
#pragma unroll
    for (int r = 0; r < K2; ++r) {
      const int k = half_row<N>(h, r);
      T Dr[n1];
#pragma unroll
      for (int m = 0; m < n1; ++m) Dr[m] = (k & 1) ? Dr1[m] : Dr0[m];
#pragma unroll
      for (int v = 0; v < NV; ++v)
        acc[v][r] = fma(-inv2h[1], line_dot(&sA[v * NP + NF * k + n1 * ci], Dr), acc[v][r]);
    }
  }
  __syncthreads();
  // ---- horizontal face terms; the tile now holds their lifts [4][NV][NF]
  T* sLift = sA;
  const bool first = A.first != 0;
  auto horizontal = [&](auto axis, int own_node, int k) {
    constexpr int a = decltype(axis)::value;
    const int n = half_swz<N>(own_node);
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = sQ[v * NP + n];
    const T pp = sQ[NV * NP + n];
    T b4[4];
    load_bg_row(sBg, k, b4);
    const NodeBg<T> bg{b4[0], b4[1], b4[2]};
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    T Fo[NV], L[NV];
    flux_axis<T, D>(q, nd, pp, a, Fo);
    face_lift(axis, hs, kindH[a], hfn, q, pp, bg, nd, Fo, L);
#pragma unroll
    for (int v = 0; v < NV; ++v) sLift[((2 * a + hs) * NV + v) * NF + hfn] = L[v];
  };
  if (hok) {
    const int u = hfn % n1, k = hfn / n1;
    horizontal(std::integral_constant<int, 0>{}, (hs ? N : 0) + n1 * u + NF * k, k);
    horizontal(std::integral_constant<int, 1>{}, u + n1 * (hs ? N : 0) + NF * k, k);
  }
  __syncthreads();
  if (!colok) return;
  // ---- horizontal lifts onto the owners' rows
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int own = (a == 0) ? ci : cj;
    const int u = (a == 0) ? cj : ci;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (own != (s ? N : 0)) continue;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int r = 0; r < K2; ++r)
          acc[v][r] += sLift[((2 * a + s) * NV + v) * NF + u + n1 * half_row<N>(h, r)];
    }
  }
  // ---- output
  T* oute = (T*)A.out + e * NP;
  if (A.mode == 0) {
#pragma unroll
    for (int r = 0; r < K2; ++r)
#pragma unroll
      for (int v = 0; v < NV; ++v) oute[v * P + t + NF * half_row<N>(h, r)] = acc[v][r];
    return;
  }
  const StageCoef<T> scf = stage_coef<T>(A);
  const T dt = scf.dt, ca = scf.ca, cb = scf.cb;
  const T* qne = (const T*)A.qn + e * NP;
  T* ppo = (T*)A.pp_out + e * NP;
#pragma unroll
  for (int r = 0; r < K2; ++r) {
    const int k = half_row<N>(h, r);
    const int n = t + NF * k;
    T qnew[NV];
    if (first) {   // uniform over the grid: stage 1 reads no q^n
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = sQ[v * NP + half_swz<N>(n)] + dt * acc[v][r];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v)
        qnew[v] = ca * qne[v * P + n] + cb * (sQ[v * NP + half_swz<N>(n)] + dt * acc[v][r]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
    ppo[n] = pprime_of<T>(qnew[D + 1], sBg[k * 4 + 3], A.bg + ((size_t)e * n1 + k) * 4, sBc + k, A.ph);
  }
}

// FP32, N = 7: 128-thread CTAs of 32 KB shared memory, 7 per SM when the registers allow it
// (72 per thread; ptxas keeps the spill to a few bytes).
template <class T, int N>
constexpr int half_min_blocks() { return (sizeof(T) == 4 && N == 7) ? 7 : 1; }

template <class T, int N>
__global__ void __launch_bounds__(HalfCfg<N>::THREADS, half_min_blocks<T, N>())
stage_kernel_half(const __grid_constant__ StageArgs A) {
  stage_body_half<T, N>(A, (int64_t)A.e_begin + (int64_t)blockIdx.x);
}

}  // namespace dgk
