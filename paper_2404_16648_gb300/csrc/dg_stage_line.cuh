// Line fused stage kernel (layout 4; 3D, odd N).
//
// The operator is the one of the other layouts: volume term of the strong form (Sec. 2.2) with
// the derivative applied along each axis, face lifts with the Rusanov flux on conforming faces
// and walls and the precomputed mortar fluxes on hanging faces (Sec. 3.3), the Shu-Osher
// combination and P' of the new state.  The order of work differs: one pass per axis, and in
// the pass along axis a every thread owns half of one line of nodes along a.  Lanes l and
// l ^ 16 of warp w hold the two halves of line L = 16 w + (l & 15) (K2 = (N+1)/2 nodes each):
// local row r is node r of the line for half 0 and node N - r for half 1, so row 0 lies on the
// line's face for both.  A pass loads the thread's nodes from the staged state, forms their
// flux along a in registers and takes the other half's fluxes by warp shuffle.  The derivative
// uses the antisymmetry of the LGL matrix under reflection, D[N-m][N-i] = -D[m][i]: in these
// local orders both halves apply the same rows r < K2 to their own and the other half's
// fluxes, half 1 with the opposite sign, so every coefficient is the same for all lanes and
// reaches the multiply-adds as a constant operand.  Row 0 adds the lift of the face from the
// same registers.  The x pass stores its part of the right-hand side to shared memory, the y
// pass adds to it, and the z pass (with the buoyancy term) reads it and finishes the stage: the
// Shu-Osher combination with q^n, the output and P' of the new state.  No flux passes through
// shared memory: per node the kernel reads the state three times and the partial right-hand
// side twice and writes it twice.
//
// Bank layout for N + 1 = 8 (32 banks of 4 bytes): node (i, j, k) sits at word
// 64 k + 8 (j ^ 2 (k & 1)) + (i ^ (j & 4)).  The x pass moves a half line as one 16-byte access,
// the y and z passes one word per node; every such access of a warp, and the 16-byte staging
// copies, reach the minimum number of shared-memory wavefronts (one per 128 bytes).  The face
// table's faces are 16 words apart for the same reason.
#pragma once
#include <type_traits>

#include "dg_stage_half.cuh"

namespace dgk {

template <int N>
struct LineCfg {
  static constexpr int n1 = N + 1, NF = n1 * n1, NP = NF * n1, K2 = n1 / 2, NV = 5;
  static constexpr int THREADS = 32 * ((NF + 15) / 16);
  static constexpr int RQ = ((NV + 1) * NP + 3) / 4 * 4;           // state and P'
  static constexpr int RR = (NV * NP + 3) / 4 * 4;                 // partial right-hand side
  static constexpr int NBS = (NV + 1) * NF + (N == 7 ? 16 : 0);    // face stride of sNb
  static constexpr int RN = (5 * NBS + (NV + 1) * NF + 3) / 4 * 4;  // no pad after the last face
};

template <class T, int N>
__host__ __device__ constexpr size_t line_smem_bytes() {
  using C = LineCfg<N>;
  return sizeof(T) * (size_t)(C::RQ + C::RR + C::RN + C::n1 * 4) + sizeof(double) * (size_t)C::n1;
}

// Word of node (i, j, k) in the staged state and the partial right-hand side.
template <int N>
__device__ __forceinline__ int line_swz(int i, int j, int k) {
  if constexpr (N == 7) {
    return 64 * k + 8 * (j ^ ((k & 1) << 1)) + (i ^ (j & 4));
  } else {
    constexpr int n1 = N + 1;
    return i + n1 * (j + n1 * k);
  }
}
template <int N>
__device__ __forceinline__ int line_swz_n(int n) {
  constexpr int n1 = N + 1;
  return line_swz<N>(n % n1, (n / n1) % n1, n / (n1 * n1));
}

// Copies `count` words to shared memory at line_swz positions (16-byte pieces when both ends
// allow it; the layout keeps aligned groups of 4 words together for N = 7).
template <class T, int N>
__device__ __forceinline__ void stage_run_line(T* dst, const T* src, int count, int tid, int nthr) {
  constexpr int per16 = 16 / sizeof(T);
  const bool aligned = N == 7 && ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) == 0 && (count % per16) == 0;
  if (aligned) {
    for (int c = tid; c < count / per16; c += nthr)
      cp_async_bytes(dst + line_swz_n<N>(c * per16), src + c * per16, 16);
  } else {
    for (int c = tid; c < count; c += nthr) cp_async_bytes(dst + line_swz_n<N>(c), src + c, (int)sizeof(T));
  }
}

// Packed FP32 pairs (two floats in one 64-bit register) for fma.rn.f32x2.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t x, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// What a pass needs from the CTA: staged data, the thread's line and the element constants.
// Elements between a CTA and the one whose data it asks the L2 for: 7 resident CTAs on each of
// 152 SMs.
constexpr int kLineAhead = 7 * 152;

template <class T>
struct LineCtx {
  const T* sQ;
  const T* sNb;
  const T* sBg;
  int h, la, lb, L;
  bool lok;
  int kind[3];
  T inv2h[3], lc[3], gamma;
};

// Node (i, j, k) of local row r of half h of line (la, lb) along axis a.
template <int N>
__device__ __forceinline__ void line_node(int a, int h, int la, int lb, int r, int* ijk) {
  const int p = h ? N - r : r;
  if (a == 0) { ijk[0] = p; ijk[1] = la; ijk[2] = lb; }
  else if (a == 1) { ijk[0] = la; ijk[1] = p; ijk[2] = lb; }
  else { ijk[0] = la; ijk[1] = lb; ijk[2] = p; }
}

// One pass along axis a: out[r][v] = -(2/h_a) (D F_a) at the thread's row r, plus the lift of
// the face (a, h) on row 0 (node 0 of the line for half 0, node N for half 1).
template <class T, int N, int a>
__device__ __forceinline__ void line_pass(const LineCtx<T>& C, T (&out)[(N + 1) / 2][5]) {
  constexpr int D = 3, n1 = N + 1, NP = n1 * n1 * n1, NF = n1 * n1, NV = 5, K2 = n1 / 2;
  constexpr int NBS = LineCfg<N>::NBS;
  constexpr bool VEC = sizeof(T) == 4 && N == 7;
  const int h = C.h, la = C.la, lb = C.lb, L = C.L;
  T F[K2][NV];
  T qf[NV], ppf = (T)0, Ff[NV];
  T bgf0 = (T)0, bgf1 = (T)0, bgf2 = (T)0, rinvf = (T)0, thf = (T)0;
  T qv[NV + 1][K2];
  if constexpr (a == 0 && VEC) {
    // one 16-byte access per plane: nodes 4 h .. 4 h + 3, i.e. rows 0..3 (half 0) or 3..0
    const int w0 = line_swz<N>(K2 * h, la, lb);
#pragma unroll
    for (int v = 0; v <= NV; ++v) {
      const float4 x = *reinterpret_cast<const float4*>(C.sQ + v * NP + w0);
      qv[v][0] = h ? x.w : x.x; qv[v][1] = h ? x.z : x.y;
      qv[v][2] = h ? x.y : x.z; qv[v][3] = h ? x.x : x.w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < K2; ++r) {
      int ijk[3];
      line_node<N>(a, h, la, lb, r, ijk);
      const int w = line_swz<N>(ijk[0], ijk[1], ijk[2]);
#pragma unroll
      for (int v = 0; v <= NV; ++v) qv[v][r] = C.sQ[v * NP + w];
    }
  }
#pragma unroll
  for (int r = 0; r < K2; ++r) {
    int ijk[3];
    line_node<N>(a, h, la, lb, r, ijk);
    T q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = qv[v][r];
    const T pp = qv[NV][r];
    T b4[4];
    load_bg_row(C.sBg, ijk[2], b4);
    const NodeBg<T> bg{b4[0], b4[1], b4[2]};
    const NodeDer<T> nd = node_der<T, D>(q, bg);
    flux_axis<T, D>(q, nd, pp, a, F[r]);
    if (r == 0) {   // the face row
#pragma unroll
      for (int v = 0; v < NV; ++v) { qf[v] = q[v]; Ff[v] = F[r][v]; }
      ppf = pp; bgf0 = bg.rb; bgf1 = bg.Tb; bgf2 = bg.pb; rinvf = nd.rinv; thf = nd.Theta;
    }
  }
  // the other half's fluxes in its local order
  T G[K2][NV];
#pragma unroll
  for (int r = 0; r < K2; ++r)
#pragma unroll
    for (int v = 0; v < NV; ++v) G[r][v] = __shfl_xor_sync(0xffffffffu, F[r][v], 16);
  // row r: node r (half 0) takes D[r][c] on node c = own row c and D[r][K2 + c] on node K2 + c
  // = other row K2 - 1 - c; node N - r (half 1) takes -D[r][c] on node N - c = own row c and
  // -D[r][K2 + c] on node K2 - 1 - c = other row K2 - 1 - c
  const T sc = h ? C.inv2h[a] : -C.inv2h[a];
  if constexpr (VEC) {
    // FP32: packed pairs, one fma.rn.f32x2 for two multiply-adds, each lane rounded as fmaf, so
    // every sum is that of the scalar form below: variables 0-1 and 2-3 of one row share the
    // coefficient (c_dtab_af2), variable 4 of rows r, r + 1 shares the flux (c_dtab_afr)
    uint64_t Fp[K2][2], Gp[K2][2], F4[K2], G4[K2];
#pragma unroll
    for (int c = 0; c < K2; ++c) {
      Fp[c][0] = f2_pack(F[c][0], F[c][1]); Fp[c][1] = f2_pack(F[c][2], F[c][3]);
      Gp[c][0] = f2_pack(G[c][0], G[c][1]); Gp[c][1] = f2_pack(G[c][2], G[c][3]);
      F4[c] = f2_pack(F[c][4], F[c][4]); G4[c] = f2_pack(G[c][4], G[c][4]);
    }
    const uint64_t sc2 = f2_pack(sc, sc);
#pragma unroll
    for (int r = 0; r < K2; ++r) {
      uint64_t s01 = 0, s23 = 0;
#pragma unroll
      for (int c = 0; c < K2; ++c) {
        const uint64_t dd = c_dtab_af2[dtab_offset(N) + r * n1 + c];
        s01 = f2_fma(dd, Fp[c][0], s01);
        s23 = f2_fma(dd, Fp[c][1], s23);
      }
#pragma unroll
      for (int c = 0; c < K2; ++c) {
        const uint64_t dd = c_dtab_af2[dtab_offset(N) + r * n1 + K2 + c];
        s01 = f2_fma(dd, Gp[K2 - 1 - c][0], s01);
        s23 = f2_fma(dd, Gp[K2 - 1 - c][1], s23);
      }
      f2_unpack(f2_mul(sc2, s01), out[r][0], out[r][1]);
      f2_unpack(f2_mul(sc2, s23), out[r][2], out[r][3]);
    }
#pragma unroll
    for (int r = 0; r < K2; r += 2) {
      uint64_t s4 = 0;
#pragma unroll
      for (int c = 0; c < K2; ++c) s4 = f2_fma(c_dtab_afr[dtab_offset(N) + r * n1 + c], F4[c], s4);
#pragma unroll
      for (int c = 0; c < K2; ++c)
        s4 = f2_fma(c_dtab_afr[dtab_offset(N) + r * n1 + K2 + c], G4[K2 - 1 - c], s4);
      f2_unpack(f2_mul(sc2, s4), out[r][4], out[r + 1][4]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < K2; ++r)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T s = (T)0;
#pragma unroll
        for (int c = 0; c < K2; ++c) s = fma(dtab_anti<T>(dtab_offset(N) + r * n1 + c), F[c][v], s);
#pragma unroll
        for (int c = 0; c < K2; ++c)
          s = fma(dtab_anti<T>(dtab_offset(N) + r * n1 + K2 + c), G[K2 - 1 - c][v], s);
        out[r][v] = sc * s;
      }
  }
  if (!C.lok) return;
  if constexpr (a == 0) cp_async_wait_all();   // this thread's face copies
  // lift of the thread's face (a, h) at face node L
  const NodeBg<T> bgf{bgf0, bgf1, bgf2};
  const NodeDer<T> ndf{rinvf, thf};
  const T* nb = C.sNb + (2 * a + h) * NBS;
  const int kd = C.kind[a];
  const T coef = h ? -C.lc[a] : C.lc[a];
  if (kd == FACE_WALL || kd == FACE_CONF) {
    const T so = wave_speed<T>(qf, ndf, bgf, ppf, a, C.gamma);
    T qo[NV], Fn[NV], sn;
    if (kd == FACE_WALL) {
#pragma unroll
      for (int v = 0; v < NV; ++v) qo[v] = qf[v];
      qo[1 + a] = -qf[1 + a];
      flux_axis<T, D>(qo, ndf, ppf, a, Fn);
      sn = so;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qo[v] = nb[v * NF + L];
      sn = face_side<T, D>(qo, bgf, nb[NV * NF + L], a, C.gamma, Fn);
    }
    // Rusanov flux F* = (Ff + Fn)/2 - (lambda/2) s (qo - qf), s = +1 with the thread's side as
    // the low one (h = 1), -1 as the high one (h = 0); its lift coef (F* - Ff), coef = -s lc,
    // is (coef/2) (Fn - Ff) + lc (lambda/2) (qo - qf): two differences and two fma per
    // variable, the same expression for both halves of the warp
    const T cA = mul_rn((T)0.5, coef);
    const T cB = mul_rn(C.lc[a], mul_rn((T)0.5, so > sn ? so : sn));
#pragma unroll
    for (int v = 0; v < NV; ++v)
      out[0][v] = fma(cB, sub_rn(qo[v], qf[v]), fma(cA, sub_rn(Fn[v], Ff[v]), out[0][v]));
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[0][v] = fma(coef, nb[v * NF + L] - Ff[v], out[0][v]);
  }
}

template <class T, int N>
__device__ __forceinline__ void stage_body_line(const StageArgs& A, int64_t e) {
  using C = LineCfg<N>;
  constexpr int D = 3, n1 = C::n1, NP = C::NP, NF = C::NF, NV = C::NV, K2 = C::K2, NSUB = 4;
  constexpr int THREADS = C::THREADS, NBS = C::NBS;
  constexpr bool VEC = sizeof(T) == 4 && N == 7;
  static_assert(n1 % 2 == 0, "layout 4 needs an even number of nodes per line");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (e >= A.E) return;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int h = lane >> 4;
  const int L0 = 16 * (tid >> 5) + (lane & 15);
  const bool lok = L0 < NF;
  const int L = lok ? L0 : 0;
  const int la = L % n1, lb = L / n1;       // the line's coordinates, lower axis first
  T* sQ = reinterpret_cast<T*>(smem_raw);   // [NV + 1][NP] state and P' (line_swz)
  T* sR = sQ + C::RQ;                       // [NV][NP] partial right-hand side (line_swz)
  T* sNb = sR + C::RR;                      // [2D][NBS] neighbour traces / mortar fluxes
  T* sBg = sNb + C::RN;                     // [n1][4]
  double* sBc = reinterpret_cast<double*>(sBg + n1 * 4);
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + e * NP;
  // ---- q^n is read only in the epilogue: ask the L2 for the element's planes now.  The CTA
  // that starts one resident wave later (kLineAhead elements on) finds its state, P' and face
  // table in L2 as well, so its staging waits for L2 instead of DRAM.
  auto prefetch_l2 = [](const void* src, int bytes) {
    if ((((uintptr_t)src) & 15) == 0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
  };
  if (tid == 0) {
    if (A.mode == 1 && !A.first) {
      const T* qne = (const T*)A.qn + e * NP;
#pragma unroll
      for (int v = 0; v < NV; ++v) prefetch_l2(qne + (int64_t)v * P, (int)(NP * sizeof(T)));
    }
    const int64_t ea = e + kLineAhead;
    if (ea < A.E) {
      const T* qa = (const T*)A.qs + ea * NP;
#pragma unroll
      for (int v = 0; v < NV; ++v) prefetch_l2(qa + (int64_t)v * P, (int)(NP * sizeof(T)));
      prefetch_l2((const T*)A.pp_in + ea * NP, (int)(NP * sizeof(T)));
      // the 120-byte conn row widened to 16-byte bounds (a bulk prefetch needs them); the conn
      // buffer is allocated with a quarter of headroom, so the widened end stays inside it
      const uintptr_t c0 = (uintptr_t)(A.conn + (size_t)ea * 2 * D * 5);
      const uintptr_t c1 = c0 + 2 * D * 5 * sizeof(int32_t);
      const uintptr_t a0 = c0 & ~(uintptr_t)15, a1 = (c1 + 15) & ~(uintptr_t)15;
      prefetch_l2((const void*)a0, (int)(a1 - a0));
      prefetch_l2(A.elem + (size_t)ea * 4, 16);
    }
  }
  // ---- own state, P', background column
#pragma unroll
  for (int v = 0; v < NV; ++v) stage_run_line<T, N>(sQ + v * NP, qe + v * P, NP, tid, THREADS);
  stage_run_line<T, N>(sQ + NV * NP, (const T*)A.pp_in + e * NP, NP, tid, THREADS);
  stage_run<T>(sBg, (const T*)A.bgt + e * n1 * 4, n1 * 4, tid, THREADS);
  if (sizeof(T) == 4) stage_run<double>(sBc, A.bgc + e * n1, n1, tid, THREADS);
  cp_async_commit();
  // ---- the faces this thread lifts: (a, h) at face node L of each axis a; only this thread
  // reads them, so they form a group of their own that it waits for before its first lift
  auto stage_face = [&](int a, int s, int fn) -> int {
    const int f = 2 * a + s;
    const int32_t* c = A.conn + ((size_t)e * 2 * D + f) * 5;
    const int kind = c[0];
    T* dst = sNb + f * NBS;
    if (kind == FACE_CONF) {
      const int no = face_node<D, N>(a, 1 - s, fn);
      const T* qb = (const T*)A.qs + (int64_t)c[1] * NP;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + fn, qb + v * P + no, (int)sizeof(T));
      cp_async_bytes(dst + NV * NF + fn, (const T*)A.pp_in + (int64_t)c[1] * NP + no, (int)sizeof(T));
    } else if (kind == FACE_FINE || kind == FACE_COARSE) {
      // the mortar fluxes are written by the mortar kernel of this stage, which may still run
      // when this grid was launched as its programmatic dependent: only a thread that reads
      // them waits for it (everything else this kernel reads comes from the previous stage,
      // complete before the mortar kernel began)
      if (A.after_mortar) asm volatile("griddepcontrol.wait;\n" ::: "memory");
      const int64_t gg = (kind == FACE_FINE) ? c[2] : c[1];
      const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
      const T* src = (const T*)A.mbuf + (((size_t)gg * (1 + NSUB) + slot) * NV) * NF;
#pragma unroll
      for (int v = 0; v < NV; ++v) cp_async_bytes(dst + v * NF + fn, src + v * NF + fn, (int)sizeof(T));
    }
    return kind;
  };
  int kind[D];
#pragma unroll
  for (int a = 0; a < D; ++a) kind[a] = lok ? stage_face(a, h, L) : FACE_WALL;
  cp_async_commit();
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  const T g = sizeof(T) == 4 ? (T)A.gf : (T)A.ph.g;
  const int level = A.elem[e * 4];
  T inv2h[D], lc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    inv2h[a] = inv2h_of<T>(A, level, a);
    lc[a] = lift_of<T>(A, level, a);   // (2/h_a) / w0
  }
  cp_async_wait_one();
  __syncthreads();
  // FP32 path: c of each z-level as two FP32 parts, in place of the double (read before the
  // epilogue, two barriers later)
  float2* sC2 = reinterpret_cast<float2*>(sBc);
  if (sizeof(T) == 4 && tid < n1) {
    const double c = sBc[tid];
    const float chi = (float)c;
    sC2[tid] = make_float2(chi, (float)(c - (double)chi));
  }

  LineCtx<T> ctx;
  ctx.sQ = sQ; ctx.sNb = sNb; ctx.sBg = sBg;
  ctx.h = h; ctx.la = la; ctx.lb = lb; ctx.L = L; ctx.lok = lok;
#pragma unroll
  for (int a = 0; a < D; ++a) { ctx.kind[a] = kind[a]; ctx.inv2h[a] = inv2h[a]; ctx.lc[a] = lc[a]; }
  ctx.gamma = gamma;
  auto node_of = [&](int a, int r, int* ijk) { line_node<N>(a, h, la, lb, r, ijk); };

  // ---- x pass: partial right-hand side to shared memory
  {
    T out[K2][NV];
    line_pass<T, N, 0>(ctx, out);
    if (lok) {
      if constexpr (VEC) {
        const int w0 = line_swz<N>(K2 * h, la, lb);
#pragma unroll
        for (int v = 0; v < NV; ++v)
          *reinterpret_cast<float4*>(sR + v * NP + w0) =
              h ? make_float4(out[3][v], out[2][v], out[1][v], out[0][v])
                : make_float4(out[0][v], out[1][v], out[2][v], out[3][v]);
      } else {
#pragma unroll
        for (int r = 0; r < K2; ++r) {
          int ijk[3];
          node_of(0, r, ijk);
          const int w = line_swz<N>(ijk[0], ijk[1], ijk[2]);
#pragma unroll
          for (int v = 0; v < NV; ++v) sR[v * NP + w] = out[r][v];
        }
      }
    }
  }
  __syncthreads();
  // ---- y pass: added to it
  {
    T out[K2][NV];
    line_pass<T, N, 1>(ctx, out);
    if (lok) {
#pragma unroll
      for (int r = 0; r < K2; ++r) {
        int ijk[3];
        node_of(1, r, ijk);
        const int w = line_swz<N>(ijk[0], ijk[1], ijk[2]);
#pragma unroll
        for (int v = 0; v < NV; ++v) sR[v * NP + w] += out[r][v];
      }
    }
  }
  __syncthreads();
  // ---- z pass, buoyancy and the epilogue
  T out[K2][NV];
  line_pass<T, N, 2>(ctx, out);
  if (!lok) return;
  T* oute = (T*)A.out + e * NP;
  const bool first = A.first != 0;
  const StageCoef<T> scf = stage_coef<T>(A);
  const T dt = scf.dt, ca = scf.ca, cb = scf.cb;
  const T* qne = (const T*)A.qn + e * NP;
  T* ppo = (T*)A.pp_out + e * NP;
#pragma unroll
  for (int r = 0; r < K2; ++r) {
    int ijk[3];
    node_of(2, r, ijk);
    const int k = ijk[2];
    const int w = line_swz<N>(ijk[0], ijk[1], k);
    const int n = ijk[0] + n1 * (ijk[1] + n1 * k);
    T rhs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) rhs[v] = sR[v * NP + w] + out[r][v];
    rhs[D] -= sQ[w] * g;                 // buoyancy -rho' g on the vertical momentum
    if (A.mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) oute[v * P + n] = rhs[v];
      continue;
    }
    T qnew[NV];
    if (first) {   // uniform over the grid: stage 1 reads no q^n
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = fma(dt, rhs[v], sQ[v * NP + w]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = fma(ca, qne[v * P + n], cb * fma(dt, rhs[v], sQ[v * NP + w]));
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
    if constexpr (sizeof(T) == 4) {
      const float2 c2 = sC2[k];
      ppo[n] = pressure_pert_f32ff(qnew[D + 1], sBg[k * 4 + 3], c2.x, c2.y, A.bg + ((size_t)e * n1 + k) * 4, A.ph);
    } else {
      ppo[n] = pprime_of<T>(qnew[D + 1], sBg[k * 4 + 3], A.bg + ((size_t)e * n1 + k) * 4, sBc + k, A.ph);
    }
  }
}

// FP32, N = 7: 128-thread CTAs of 32,256 bytes of shared memory (33,280 with the driver's
// reserve, allocated in 128-byte units), 7 per SM in its 233,472 bytes; 72 registers a thread.
template <class T, int N>
constexpr int line_min_blocks() { return (sizeof(T) == 4 && N == 7) ? 7 : 1; }

template <class T, int N>
__global__ void __launch_bounds__(LineCfg<N>::THREADS, line_min_blocks<T, N>())
stage_kernel_line(const __grid_constant__ StageArgs A) {
  stage_body_line<T, N>(A, (int64_t)A.e_begin + (int64_t)blockIdx.x);
}

}  // namespace dgk
