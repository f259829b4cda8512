// Stage body of layout 5: every face flux comes from a buffer (conforming and wall faces from
// face_kernel, hanging faces from mortar_kernel), and the volume term runs as one column pass
// and one line pass per horizontal axis.
//
// The operator is the one of the other layouts (volume term of the strong form, Sec. 2.2; face
// lifts (2/h)/w0 (F* - F) with the Rusanov flux or the mortar flux, Sec. 3.3; the Shu-Osher
// combination and P' of the new state).  The CTA stages the element's state, its background
// and the F* of its horizontal faces into shared memory (each column thread keeps its P' and
// the F* of its two vertical faces in registers, which holds the FP64 N = 7 CTA to 52.8 KB, 4
// per SM), then:
//   column pass  - one thread per vertical node line (column): the fluxes of its nodes along
//                  x to a shared tile and along the vertical axis in registers; the vertical
//                  derivative by the even/odd split of the antisymmetric LGL matrix, and the
//                  lifts of the two vertical faces from those registers;
//   x line pass  - one thread per node line along x: the line's x fluxes from the tile, the
//                  derivative of the line (even/odd split), and the lifts of the line's two end
//                  nodes from the same values, written back over the line; the column threads
//                  then add it, scaled by -2/h_x, to their accumulators;
//   y line pass  - (3D) the same for y, on y fluxes the column threads recompute into the tile.
// Each thread of a line pass lifts exactly the two face nodes at the ends of its line, so no
// warp runs a face branch for a few of its lanes, and the lift uses the flux the derivative
// already read instead of evaluating it again at the face node.  The lifts enter the line's
// derivative unscaled, as -(1/w0)(F* - F) on the low face and +(1/w0)(F* - F) on the high one,
// so that the -2/h_a scaling of the line makes them (2/h_a)/w0 (F* - F) with the face's sign;
// for odd N their -F parts sit in the derivative table itself (the summation-by-parts form
// D - M^-1 B, still centro-antisymmetric), so a line adds only its two F* terms.
//
// The tile stores node (i, j, k) at ((k n1 + j) (n1 + 1) + i) (3D) or (k (n1 + 1) + i) (2D):
// one padding word per x line.  For N = 7 in FP64 that makes the x line pass (each lane reading
// its own line) and the y line pass (lanes reading neighbouring columns) reach the minimum
// number of shared-memory wavefronts.
#pragma once
#include "dg_stage_async.cuh"

namespace dgk {

template <class T, int D, int N>
__host__ __device__ constexpr int fb_tile_words() {
  constexpr int n1 = N + 1, NV = D + 2;
  return ((D == 3 ? n1 * n1 : n1) * (n1 + 1) * NV + 3) / 4 * 4;
}
// Words of T per element: tile, state, fluxes of the 2(d-1) horizontal faces [NV][NF] each,
// background, FP64 c.  P' and the vertical faces' fluxes go to registers.
template <class T, int D, int N>
__host__ __device__ constexpr int fb_elem_words() {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  return fb_tile_words<T, D, N>() + (NV * NP + 3) / 4 * 4 + (2 * (D - 1) * NV * NF + 3) / 4 * 4 + n1 * 4 +
         ((n1 * (int)(8 / sizeof(T))) + 3) / 4 * 4;
}
template <class T, int D, int N, int EPB>
__host__ __device__ constexpr size_t fb_smem_bytes() {
  return sizeof(T) * (size_t)EPB * fb_elem_words<T, D, N>();
}

// The even/odd split (the layout of c_dtab_eo_*) of A + (1/w0) (e_0 e_0^T - e_N e_N^T), with A
// the antisymmetric part of the LGL derivative: the derivative with the -(1/w0) F_0 and +(1/w0)
// F_N parts of the two end-node lifts folded in (the summation-by-parts form D - M^-1 B).  The
// added diagonal keeps the centro-antisymmetry, so only Ae[0][0] and Ao[0][0] differ from the
// plain split, each by 1/(2 w0), and a line adds -(1/w0) F*_lo and +(1/w0) F*_hi alone.  Odd N
// only; per translation unit, filled by upload_dtab_fb() of the unit before its first launch.
static __constant__ float c_dtab_eob_f[kDTabSize];
static __constant__ double c_dtab_eob_d[kDTabSize];

static inline cudaError_t upload_dtab_fb(const double* all) {
  double eo[kDTabSize];
  float eof[kDTabSize];
  for (int i = 0; i < kDTabSize; ++i) eo[i] = 0.0;
  for (int N = 1; N <= 8; N += 2) {
    const int o = dtab_offset(N), n1 = N + 1, K2 = n1 / 2;
    auto anti = [&](int m, int i) {
      return 0.5 * (all[o + m * n1 + i] - all[o + (N - m) * n1 + (N - i)]);
    };
    for (int i = 0; i < K2; ++i)
      for (int m = 0; m < K2; ++m) {
        eo[o + i * K2 + m] = 0.5 * (anti(i, m) + anti(i, N - m));
        eo[o + K2 * K2 + i * K2 + m] = 0.5 * (anti(i, m) - anti(i, N - m));
      }
    // w0 = 2 / (N (N+1)), rounded as the LGL weights are, so that 1/w0 here is the 1/w0 the
    // kernels multiply F* by
    const double half_rw0 = 0.5 * (1.0 / (2.0 / (N * (N + 1.0))));
    eo[o] += half_rw0;
    eo[o + K2 * K2] += half_rw0;
  }
  for (int i = 0; i < kDTabSize; ++i) eof[i] = (float)eo[i];
  cudaError_t e = cudaMemcpyToSymbol(c_dtab_eob_d, eo, sizeof(eo));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dtab_eob_f, eof, sizeof(eof));
}
template <class T> __device__ __forceinline__ T dtab_eob(int i);
template <> __device__ __forceinline__ float dtab_eob<float>(int i) { return c_dtab_eob_f[i]; }
template <> __device__ __forceinline__ double dtab_eob<double>(int i) { return c_dtab_eob_d[i]; }

// P' of the new state (Sec. 2.1, P' = P_bar ((1 + x)^gamma - 1), x = Theta'/Theta_bar), FP64:
// the binomial series of pressure_pert with as many terms K as |x| needs instead of six for all
// |x| < 2^-10 and eleven up to 2^-5.  For 1 < gamma <= 2, |binom(gamma, K+1)| / gamma <=
// 1 / (K (K+1)), so the first omitted term, relative to the leading one gamma x, stays below
// 2^-54 / 6 (K = 2, |x| < 2^-27), 2^-54 / 12 (K = 3, < 2^-18), 2^-52 / 20 (K = 4, < 2^-13),
// 2^-50 / 30 (K = 5, < 2^-10), 2^-54 / 42 (K = 6, < 2^-9), 2^-49 / 56 (K = 7, < 2^-7), all under
// a third of the result's rounding; |x| >= 2^-7 (and a gamma outside (1, 2], tiers = false)
// take pressure_pert itself.  The tier is picked from the high word of x by integer compares,
// which leaves the FP64 pipe to the series.  pb is P_bar at the node's height.
__device__ __forceinline__ double pprime_tiered(double tp, double invTb, double pb, bool tiers,
                                                const PhysC& ph) {
  const double x = __dmul_rn(tp, invTb);
  const int hx = __double2hiint(x) & 0x7fffffff;   // |x| < 2^-m  <=>  hx < (1023 - m) << 20
  if (!tiers || hx >= 0x3F800000) return pressure_pert<kSeries>(tp, invTb, pb, ph);   // 2^-7
  const double* b = ph.binom;                      // b[k - 1] = binom(gamma, k)
  double p;                                        // sum_{k=1..K} b[k - 1] x^(k - 1)
  if (hx < 0x3E400000) {                           // 2^-27
    p = fma(b[1], x, b[0]);
  } else if (hx < 0x3ED00000) {                    // 2^-18
    p = fma(fma(b[2], x, b[1]), x, b[0]);
  } else if (hx < 0x3F200000) {                    // 2^-13
    p = fma(fma(fma(b[3], x, b[2]), x, b[1]), x, b[0]);
  } else if (hx < 0x3F500000) {                    // 2^-10
    p = fma(fma(fma(fma(b[4], x, b[3]), x, b[2]), x, b[1]), x, b[0]);
  } else if (hx < 0x3F600000) {                    // 2^-9
    p = fma(fma(fma(fma(fma(b[5], x, b[4]), x, b[3]), x, b[2]), x, b[1]), x, b[0]);
  } else {
    p = fma(fma(fma(fma(fma(fma(b[6], x, b[5]), x, b[4]), x, b[3]), x, b[2]), x, b[1]), x, b[0]);
  }
  return __dmul_rn(pb, __dmul_rn(p, x));
}

template <class T> __device__ __forceinline__ T rw0_of(const StageArgs& A);
template <> __device__ __forceinline__ float rw0_of<float>(const StageArgs& A) { return A.rw0f; }
template <> __device__ __forceinline__ double rw0_of<double>(const StageArgs& A) { return A.rw0d; }

// Derivative of one line of n1 values r (unscaled, D r) into out, with the lifts of its two end
// nodes, -rw0 (Flo - r[0]) and +rw0 (Fhi - r[N]).  For even n1 the -rw0 r[0] and +rw0 r[N] parts
// come with the derivative from the boundary-folded even/odd table, and only the F* terms are
// added here.
template <class T, int N>
__device__ __forceinline__ void fb_line(const T (&r)[N + 1], T Flo, T Fhi, T rw0, T (&out)[N + 1]) {
  constexpr int n1 = N + 1;
  if constexpr (n1 % 2 == 0) {
    constexpr int K2 = n1 / 2;
    T Ev[K2], Ov[K2];
#pragma unroll
    for (int m = 0; m < K2; ++m) {
      Ev[m] = add_rn(r[m], r[N - m]);
      Ov[m] = sub_rn(r[m], r[N - m]);
    }
#pragma unroll
    for (int i = 0; i < K2; ++i) {
      T se = (T)0, so = (T)0;
#pragma unroll
      for (int m = 0; m < K2; ++m) {
        se = fma(dtab_eob<T>(dtab_offset(N) + i * K2 + m), Ev[m], se);
        so = fma(dtab_eob<T>(dtab_offset(N) + K2 * K2 + i * K2 + m), Ov[m], so);
      }
      out[i] = add_rn(se, so);
      out[N - i] = sub_rn(so, se);
    }
    out[0] = fma(-rw0, Flo, out[0]);
    out[N] = fma(rw0, Fhi, out[N]);
  } else {
#pragma unroll
    for (int i = 0; i < n1; ++i) {
      T s = (T)0;
#pragma unroll
      for (int m = 0; m < n1; ++m) s = fma(dtab<T>(dtab_offset(N) + i * n1 + m), r[m], s);
      out[i] = s;
    }
    out[0] = fma(-rw0, sub_rn(Flo, r[0]), out[0]);
    out[N] = fma(rw0, sub_rn(Fhi, r[N]), out[N]);
  }
}

template <class T, int D, int N, int EPB>
__device__ __forceinline__ void stage_body_fb(const StageArgs& A, int64_t e0) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  constexpr int RS = n1 + 1;                       // tile stride of an x line
  constexpr int TV = (D == 3 ? n1 * n1 : n1) * RS; // tile words per variable
  constexpr int RA = fb_tile_words<T, D, N>();
  constexpr int RQ = (NV * NP + 3) / 4 * 4;
  constexpr int RN = (2 * (D - 1) * NV * NF + 3) / 4 * 4;
  constexpr int EW = fb_elem_words<T, D, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int le = tid / NF, t = tid - le * NF;
  T* base = reinterpret_cast<T*>(smem_raw) + (le < EPB ? le : 0) * EW;
  T* sA = base;                       // [NV][TV] flux tile, then line derivatives
  T* sQ = base + RA;                  // [NV][NP] state
  T* sF = base + RA + RQ;             // [2 (D - 1)][NV][NF] F* of the horizontal faces
  T* sBg = base + RA + RQ + RN;       // [n1][4]
  double* sBc = reinterpret_cast<double*>(sBg + n1 * 4);   // [n1] (FP32 path)
  const int64_t e = e0 + le;
  // threads beyond EPB columns (a persistent block of a fixed size) only take part in the
  // barriers and write no shared memory
  const bool inblk = le < EPB;
  const bool valid = inblk && e < A.E;
  // the column of this thread, and its line in the line passes: (j, k) along x, (i, k) along y
  // in 3D, k along x in 2D -- in every case the line's tangential index on its end faces is t
  const int ci = t % n1, cj = (D == 3) ? t / n1 : 0;
  const int la = t % n1, lk = (D == 3) ? t / n1 : t;
  auto tix = [&](int i, int j, int k) { return (D == 3 ? (k * n1 + j) : k) * RS + i; };
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + (valid ? e : 0) * NP;
  // ---- staging: own state and background column to shared memory, the fluxes of the
  // horizontal faces too; this column's P' and the vertical faces' fluxes to registers
  T ppc[n1], Fv[2][NV];
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) stage_run<T>(sQ + v * NP, qe + v * P, NP, t, NF);
    stage_run<T>(sBg, (const T*)A.bgt + e * n1 * 4, n1 * 4, t, NF);
    if (sizeof(T) == 4) stage_run<double>(sBc, A.bgc + e * n1, n1, t, NF);
    const T* ppe = (const T*)A.pp_in + e * NP;
#pragma unroll
    for (int k = 0; k < n1; ++k) ppc[k] = ppe[t + NF * k];
    // launched as the programmatic dependent of this stage's face kernel, which completes only
    // after the mortar kernel: wait for it before reading either buffer
    if (A.after_mortar) asm volatile("griddepcontrol.wait;\n" ::: "memory");
#pragma unroll
    for (int f = 0; f < 2 * D; ++f) {
      const int32_t* c = A.conn + ((size_t)e * 2 * D + f) * 5;
      const int kind = c[0];
      const T* src;
      if (kind == FACE_FINE || kind == FACE_COARSE) {
        const int64_t gg = (kind == FACE_FINE) ? c[2] : c[1];
        const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
        src = (const T*)A.mbuf + (((size_t)gg * (1 + NSUB) + slot) * NV) * NF;
      } else {
        src = (const T*)A.fbuf + (size_t)c[2] * NV * NF;
      }
      if (f < 2 * (D - 1)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) cp_async_bytes(sF + (f * NV + v) * NF + t, src + v * NF + t, (int)sizeof(T));
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) Fv[f - 2 * (D - 1)][v] = src[v * NF + t];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < n1; ++k) ppc[k] = (T)0;
#pragma unroll
    for (int v = 0; v < NV; ++v) { Fv[0][v] = (T)0; Fv[1][v] = (T)0; }
  }
  cp_async_commit();
  // the accumulators hold the right-hand side times sc, the factor the Shu-Osher combination
  // applies to it (1 for a plain right-hand side, dt in the first stage, cb dt after it): the
  // scale rides on the -2/h factors and on g, and the combination saves a multiply per value
  const StageCoef<T> scf = stage_coef<T>(A);
  const bool first = scf.first;
  const T sc = A.mode == 0 ? (T)1 : (first ? scf.dt : scf.cb * scf.dt);
  const T g = (sizeof(T) == 4 ? (T)A.gf : (T)A.ph.g) * sc;
  const T rw0 = rw0_of<T>(A);
  T inv2h[D];
  const int level = valid ? A.elem[e * 4] : 0;
#pragma unroll
  for (int a = 0; a < D; ++a) inv2h[a] = valid ? inv2h_of<T>(A, level, a) * sc : (T)0;
  cp_async_wait_all();
  __syncthreads();
  // ---- column pass: x fluxes to the tile, the vertical derivative and the vertical lifts
  T acc[NV][n1];
  T rinvc[n1];   // 1/rho of the column's nodes, kept for the y fluxes
  {
    T Fz[NV][n1];
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      const int n = t + NF * k;
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = valid ? sQ[v * NP + n] : (T)0;
      const T pp = ppc[k];
      const NodeBg<T> bg = valid ? NodeBg<T>{sBg[k * 4], sBg[k * 4 + 1], sBg[k * 4 + 2]}
                                 : NodeBg<T>{(T)1, (T)1, (T)1};
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v][k] = (T)0;
      acc[D][k] = -(q[0] * g);               // buoyancy -rho' g (times sc) on the vertical momentum
      const NodeDer<T> nd = node_der<T, D>(q, bg);
      rinvc[k] = nd.rinv;
      T F[NV];
      flux_axis<T, D>(q, nd, pp, 0, F);
      if (inblk) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sA[v * TV + tix(ci, cj, k)] = F[v];
      }
      flux_axis<T, D>(q, nd, pp, D - 1, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fz[v][k] = F[v];
    }
    // the vertical faces' fluxes at this column: face (D - 1, s), tangential index t
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T dz[n1];
      fb_line<T, N>(Fz[v], Fv[0][v], Fv[1][v], rw0, dz);
#pragma unroll
      for (int k = 0; k < n1; ++k) acc[v][k] = fma(-inv2h[D - 1], dz[k], acc[v][k]);
    }
  }
  __syncthreads();
  // ---- x line pass: line (la, lk) of the tile, in place
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T r[n1], d[n1];
#pragma unroll
      for (int m = 0; m < n1; ++m) r[m] = sA[v * TV + tix(m, la, lk)];
      fb_line<T, N>(r, sF[(0 * NV + v) * NF + t], sF[(1 * NV + v) * NF + t], rw0, d);
#pragma unroll
      for (int m = 0; m < n1; ++m) sA[v * TV + tix(m, la, lk)] = d[m];
    }
  }
  __syncthreads();
  // ---- the x derivative into the column accumulators; in 3D the y fluxes into the tile (the
  // positions this thread just read, so no barrier between)
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < n1; ++k) acc[v][k] = fma(-inv2h[0], sA[v * TV + tix(ci, cj, k)], acc[v][k]);
  }
  // q^n of this column is requested now and used last
  T qn_col[NV][n1];
  if (valid && A.mode == 1 && !first) {
    const T* qne = (const T*)A.qn + e * NP;
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) qn_col[v][k] = qne[v * P + t + NF * k];
  }
  if constexpr (D == 3) {
#pragma unroll
    for (int k = 0; k < n1; ++k) {
      const int n = t + NF * k;
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = valid ? sQ[v * NP + n] : (T)0;
      const NodeBg<T> bg = valid ? NodeBg<T>{sBg[k * 4], sBg[k * 4 + 1], sBg[k * 4 + 2]}
                                 : NodeBg<T>{(T)1, (T)1, (T)1};
      T F[NV];
      flux_axis<T, D>(q, NodeDer<T>{rinvc[k], add_rn(bg.Tb, q[D + 1])}, ppc[k], 1, F);
      if (inblk) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sA[v * TV + tix(ci, cj, k)] = F[v];
      }
    }
    __syncthreads();
    // ---- y line pass: line (la, lk) = (i, k) along y, in place
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T r[n1], d[n1];
#pragma unroll
        for (int m = 0; m < n1; ++m) r[m] = sA[v * TV + tix(la, m, lk)];
        fb_line<T, N>(r, sF[(2 * NV + v) * NF + t], sF[(3 * NV + v) * NF + t], rw0, d);
#pragma unroll
        for (int m = 0; m < n1; ++m) sA[v * TV + tix(la, m, lk)] = d[m];
      }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < n1; ++k) acc[v][k] = fma(-inv2h[1], sA[v * TV + tix(ci, cj, k)], acc[v][k]);
    }
  }
  if (!valid) return;
  // ---- output
  T* oute = (T*)A.out + e * NP;
  if (A.mode == 0) {
#pragma unroll
    for (int k = 0; k < n1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) oute[v * P + t + NF * k] = acc[v][k];
    return;
  }
  const T ca = scf.ca, cb = scf.cb;
  // 1 < gamma <= 2 by the bit patterns (positive doubles order as their integers)
  const long long gbits = __double_as_longlong(A.ph.gamma);
  const bool tiers = gbits > 0x3FF0000000000000LL && gbits <= 0x4000000000000000LL;
  T* ppo = (T*)A.pp_out + e * NP;
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    const int n = t + NF * k;
    T qnew[NV];
    if (first) {   // uniform over the grid
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = add_rn(sQ[v * NP + n], acc[v][k]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qnew[v] = fma(ca, qn_col[v][k], fma(cb, sQ[v * NP + n], acc[v][k]));
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
    if constexpr (sizeof(T) == 8)
      ppo[n] = pprime_tiered(qnew[D + 1], sBg[k * 4 + 3], sBg[k * 4 + 2], tiers, A.ph);
    else
      ppo[n] = pprime_of<T>(qnew[D + 1], sBg[k * 4 + 3], A.bg + ((size_t)e * n1 + k) * 4, sBc + k, A.ph);
  }
}

template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D - 1))
stage_kernel_fb(const __grid_constant__ StageArgs A) {
  stage_body_fb<T, D, N, EPB>(A, (int64_t)A.e_begin + (int64_t)blockIdx.x * EPB);
}

}  // namespace dgk
