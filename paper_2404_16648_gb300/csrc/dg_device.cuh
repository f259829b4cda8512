// Device kernels of the GB300 tree-based dGSEM hot path (sm_103a).
//
// Per SSP-RK3 stage two launches:
//  * mortar_kernel: one CTA per hanging face (Sec. 3.3 mortar method).  Projects the coarse
//    trace onto the 2^(d-1) mortars (P = M^{-1} S, exact interpolation), solves the Rusanov
//    problem on every mortar node against the fine traces (the fine face is the mortar:
//    identity projection), stores F* for the fine sides and the back-projection
//    sum_m s M^{-1} S^T F*_m (s = 1/2 per tangential axis) for the coarse side.
//  * stage_kernel: one thread per LGL node, EPB elements per CTA.  Volume term of the strong
//    form (Sec. 2.2): flux at the node, D applied along each axis through shared memory
//    (sum factorisation), buoyancy source; face terms: Rusanov on conforming faces and walls
//    (mirror state), precomputed mortar fluxes on hanging faces, lifted with 2/(h w_0); then the
//    Shu-Osher stage combination.  The epilogue also evaluates the pressure perturbation P' of
//    the new state in FP64 and stores it as an extra plane, so that the next stage reads P' of
//    its own node and of its face neighbours instead of recomputing it.
//
// Face fluxes use explicitly rounded arithmetic (__dadd_rn etc.), so the two elements that
// share a conforming face compute bit-identical F* and the scheme conserves mass and Theta
// to the rounding of the update itself.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dgk {

constexpr int kMaxLevels = 13;   // DG_MAX_LEVEL + 1
constexpr int kSeries = 11;      // binomial-series terms kept for the FP64 pressure perturbation

struct PhysC {
  double theta0, p0, g, R, cp, cv, gamma;
  double binom[kSeries];         // binom(gamma, k) for k = 1..kSeries
  float rel[3];                  // binom(gamma, k) / gamma for k = 2..4 (FP32 path's correction)
};

enum { FACE_WALL = 0, FACE_CONF = 1, FACE_FINE = 2, FACE_COARSE = 3 };

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Elements per CTA of the node-per-thread layout and of the column layouts.
__host__ __device__ constexpr int epb_node(int D, int N) {
  return ipow(N + 1, D) >= 128 ? 1 : 256 / ipow(N + 1, D);
}
__host__ __device__ constexpr int epb_col(int D, int N) {
  return ipow(N + 1, D - 1) >= 64 ? 1 : (128 / ipow(N + 1, D - 1) > 0 ? 128 / ipow(N + 1, D - 1) : 1);
}

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }

// Pressure perturbation P(Theta_bar + Theta') - P(Theta_bar) of the EOS of Sec. 2.1, in FP64,
// through the exact identity P' = P_bar ((1 + x)^gamma - 1), x = Theta' / Theta_bar, which has
// no cancellation between two ~1e5 Pa values.  For |x| <= 2^-5 the binomial series
// sum_{k=1..K} binom(gamma, k) x^k is summed by Horner's rule: K = 11 keeps the truncation below
// 1e-19 relative (FP64 path, integrals), K = 4 below 8e-9 relative, under the FP32 rounding of
// the result (FP32 path).  Larger |x| take expm1(gamma log1p(x)).
template <int K>
__device__ __forceinline__ double pressure_pert(double tp, double invTb, double pb,
                                                const PhysC& ph) {
  const double x = tp * invTb;
  if (fabs(x) <= 0.0009765625) {
    // |x| <= 2^-10: six terms; the first term left out, binom(gamma, 7) x^7 with
    // |binom(gamma, 7)| < 5e-3, is below 4e-24 P_bar, i.e. 3e-21 of P', far under its rounding
    constexpr int K6 = K < 6 ? K : 6;
    double p = ph.binom[K6 - 1];
#pragma unroll
    for (int k = K6 - 2; k >= 0; --k) p = fma(p, x, ph.binom[k]);
    return __dmul_rn(pb, __dmul_rn(p, x));
  }
  if (fabs(x) <= 0.03125) {
    double p = ph.binom[K - 1];
#pragma unroll
    for (int k = K - 2; k >= 0; --k) p = fma(p, x, ph.binom[k]);
    return __dmul_rn(pb, __dmul_rn(p, x));
  }
  return __dmul_rn(pb, expm1(__dmul_rn(ph.gamma, log1p(x))));
}

// P' for the FP32 path, stored in FP32: with c = gamma P_bar / Theta_bar (FP64, per z-level),
//   P' = A (1 + s),  A = Theta' c,  s = sum_{k=2..4} binom(gamma, k)/gamma x^(k-1),
// A and A + A s in FP64, s in FP32.  |s| < 0.7 % for |x| <= 2^-5, so the FP32 rounding of s
// moves P' by < 1e-9 relative and the truncation after x^4 by < 8e-9, both below the FP32
// rounding (6e-8) of the stored result: the value is the FP64 evaluation rounded to FP32 up to
// rare one-ulp ties, with 5 FP64 operations instead of 9.  Larger |x| use the full FP64 form
// with the row bd = (rho_bar, Theta_bar, p_bar, 1/Theta_bar) of the FP64 background.
__device__ __forceinline__ float pressure_pert_f32(float tp, float invTbf, double c, const double* bd,
                                                   const PhysC& ph) {
  const float x = __fmul_rn(tp, invTbf);
  if (fabsf(x) <= 0.03125f) {
    const float s = __fmul_rn(x, __fmaf_rn(x, __fmaf_rn(x, ph.rel[2], ph.rel[1]), ph.rel[0]));
    const double A = __dmul_rn((double)tp, c);
    return (float)__fma_rn(A, (double)s, A);
  }
  return (float)pressure_pert<kSeries>((double)tp, bd[3], bd[2], ph);
}

// The same P' with the product A = Theta' c in FP32 pieces instead of FP64: c = chi + clo (its
// FP32 rounding and the rounding of the rest, within 2^-48 of c), A = ahi + alo with ahi the FP32
// product and alo the exact rounding error of tp chi (one fma) plus tp clo, so that ahi + alo is
// within about 2^-46 of A; then P' = fl(ahi + fl(ahi s + alo)).  The inner sum is below 0.7 %
// of A, so its rounding and the omitted alo s move the result by about 1e-9 relative, 1/60 of
// the final rounding: the value is the FP64 evaluation rounded to FP32 up to a one-ulp difference
// where it lies that close to a rounding boundary.  No FP64 operation on this branch.
// The large-|x| branch, out of line: it is rarely taken, and inlined at every use its FP64
// series and expm1/log1p would crowd the hot code out of the instruction cache.
static __device__ __noinline__ float pressure_pert_f32_full(float tp, const double* bd, const PhysC& ph) {
  return (float)pressure_pert<kSeries>((double)tp, bd[3], bd[2], ph);
}
__device__ __forceinline__ float pressure_pert_f32ff(float tp, float invTbf, float chi, float clo,
                                                     const double* bd, const PhysC& ph) {
  const float x = __fmul_rn(tp, invTbf);
  if (fabsf(x) <= 0.03125f) {
    const float s = __fmul_rn(x, __fmaf_rn(x, __fmaf_rn(x, ph.rel[2], ph.rel[1]), ph.rel[0]));
    const float ahi = __fmul_rn(tp, chi);
    const float alo = __fmaf_rn(tp, clo, __fmaf_rn(tp, chi, -ahi));
    return __fadd_rn(ahi, __fmaf_rn(ahi, s, alo));
  }
  return pressure_pert_f32_full(tp, bd, ph);
}

// P' of a node in the arithmetic type T: FP64 series (T = double) or the form above.  invTb is
// 1/Theta_bar in T (the background table of the path), bd the FP64 background row, bc -> c.
template <class T>
__device__ __forceinline__ T pprime_of(T tp, T invTb, const double* bd, const double* bc, const PhysC& ph);
template <>
__device__ __forceinline__ double pprime_of<double>(double tp, double invTb, const double* bd, const double*,
                                                    const PhysC& ph) {
  return pressure_pert<kSeries>(tp, invTb, bd[2], ph);
}
template <>
__device__ __forceinline__ float pprime_of<float>(float tp, float invTb, const double* bd, const double* bc,
                                                  const PhysC& ph) {
  return pressure_pert_f32(tp, invTb, *bc, bd, ph);
}

// Background and pressure at one node, in the flux arithmetic type T.
template <class T>
struct NodeBg {
  T rb, Tb, pb;
};

// Reciprocal and square root used by the fluxes.  Deterministic (the same inputs give the same
// bits wherever they are evaluated), so the two elements of a face agree bit for bit.  FP64:
// Newton-Raphson from the hardware approximation, within about one ulp (not always correctly
// rounded: the 1e-12 FP64 parity bound is far above that, and the FP64 pipe, which bounds the
// FP64 kernels, does less work than for the correctly rounded forms).  FP32: the hardware
// approximations (about 1 ulp; rho is never subnormal), far below the FP32 path's stated error
// bound.
//
// 1/x: Newton's iteration for f(r) = 1/r - x, r <- r + r (1 - x r), the residual by one fma.
// Each step squares the relative error of r, so two steps from the hardware seed (relative error
// below 2^-20) reach the rounding of the last one.
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// sqrt(a) for a > 0: Newton's iteration for the inverse square root, y <- y (3/2 - (a/2) y^2),
// once from the hardware seed, then s = a y corrected once by Newton's step for s^2 = a,
// s <- s + (y/2) (a - s^2), the residual by one fma: each step squares the relative error.
__device__ __forceinline__ double sqrt_fast(double a) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  y = y * fma(-(0.5 * a) * y, y, 1.5);
  const double s = a * y;
  return fma(0.5 * y, fma(-s, s, a), s);
}
__device__ __forceinline__ float sqrt_fast(float x) { return __fmul_rn(x, rsqrtf(x)); }

// Quantities of one node's state that every flux component needs, computed once.
template <class T>
struct NodeDer {
  T rinv;    // 1 / (rho_bar + rho')
  T Theta;   // Theta_bar + Theta'
};

template <class T, int D>
__device__ __forceinline__ NodeDer<T> node_der(const T* q, const NodeBg<T>& bg) {
  return NodeDer<T>{recip(add_rn(bg.rb, q[0])), add_rn(bg.Tb, q[D + 1])};
}

// Component `a` of the Euler flux (Sec. 2.1, Eq. "eulervector") at one node, perturbation form:
// rho': U_a;  U_b: U_b u_a + P' delta_ab;  Theta': (Theta_bar + Theta') u_a, with u_a = U_a / rho.
template <class T, int D>
__device__ __forceinline__ void flux_axis(const T* q, const NodeDer<T>& nd, T pp, int a, T* F) {
  const T ua = mul_rn(q[1 + a], nd.rinv);
  F[0] = q[1 + a];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    T f = mul_rn(q[1 + b], ua);
    if (b == a) f = add_rn(f, pp);
    F[1 + b] = f;
  }
  F[D + 1] = mul_rn(nd.Theta, ua);
}

// Wave speed |u_a| + c, c = sqrt(gamma P / rho) of the total state (P = P_bar + P').
template <class T>
__device__ __forceinline__ T wave_speed(const T* q, const NodeDer<T>& nd, const NodeBg<T>& bg, T pp,
                                        int a, T gamma) {
  const T ua = mul_rn(q[1 + a], nd.rinv);
  const T c = sqrt_fast(mul_rn(mul_rn(gamma, add_rn(bg.pb, pp)), nd.rinv));
  return add_rn(ua < (T)0 ? -ua : ua, c);
}

// Rusanov flux along +axis a (Sec. 2.2): F* = (F(qm) + F(qp))/2 - lambda/2 (qp - qm),
// lambda = max(|u_a| + c) over both sides; qm is the low side, qp the high side, with their
// fluxes Fm, Fp and wave speeds sm, sp already evaluated.
template <class T, int D>
__device__ __forceinline__ void rusanov(const T* qm, const T* Fm, T sm, const T* qp, const T* Fp,
                                        T sp, T* Fs) {
  constexpr int NV = D + 2;
  const T hl = mul_rn((T)0.5, sm > sp ? sm : sp);
#pragma unroll
  for (int v = 0; v < NV; ++v)
    Fs[v] = fma(-hl, sub_rn(qp[v], qm[v]), mul_rn((T)0.5, add_rn(Fm[v], Fp[v])));
}

// Flux and wave speed of a face state in one call.
template <class T, int D>
__device__ __forceinline__ T face_side(const T* q, const NodeBg<T>& bg, T pp, int a, T gamma, T* F) {
  const NodeDer<T> nd = node_der<T, D>(q, bg);
  flux_axis<T, D>(q, nd, pp, a, F);
  return wave_speed<T>(q, nd, bg, pp, a, gamma);
}

struct StageArgs {
  const void* qs;        // stage input state (T), NV planes of `plane` entries
  const void* pp_in;     // P' of qs (T), one plane
  const void* qn;        // q^n for the Shu-Osher combination (T)
  void* out;             // output (T): dq/dt (mode 0) or the next stage state (mode 1)
  void* pp_out;          // mode 1: P' of the output state (T), one plane
  const void* mbuf;      // mortar fluxes [G][1 + 2^(d-1)][NV][NF] (T)
  int64_t plane;         // entries per variable plane (elements x nodes)
  int32_t E;
  const int32_t* elem;   // [E][4]: level, c0, c1, c2
  const int32_t* conn;   // [E][2d][5] (see tree.cpp)
  const double* bg;      // [E][N+1][4]: rho_bar, Theta_bar, p_bar, 1/Theta_bar (FP64)
  const void* bgt;       // [E][N+1][4]: the same in T (the FP64 array itself when T = double)
  const double* bgc;     // [E][N+1]: gamma p_bar / Theta_bar (FP32 path's P'; null for FP64)
  const void* ops;       // (T) D, P0, P1, C0, C1 (n1 x n1 each), w (n1)
  float inv2hf[kMaxLevels][3];    // 2/h per level and axis
  double inv2hd[kMaxLevels][3];
  float liftf[kMaxLevels][3];     // face lift factor (2/h) / w0 per level and axis
  double liftd[kMaxLevels][3];
  double dt, ca, cb;
  int32_t mode;
  int32_t variant;       // 0: column kernel, 1: node-per-thread kernel, 2: column kernel with async staging
  int32_t plane32;       // `plane` as int32 (the host guarantees (NV+1) * plane < 2^31)
  float gammaf, gf;      // gamma and g in FP32
  PhysC ph;
  // layout 4: the launch directly follows the mortar kernel of the same stage and may begin
  // before it ends (programmatic dependent launch); the kernel waits for it before reading mbuf
  int32_t after_mortar;
  // the launch covers elements e_begin .. E - 1 (a part of an SFC partition; 0 otherwise)
  int32_t e_begin;
  // layout 5: F* of conforming and wall faces, one slot per face (dg_face.cuh); the slot of a
  // face is the third field of its connectivity row
  const void* fbuf;
  // 1 / w0 (w0 the LGL weight of an end node): layout 5 adds the lifts to the unscaled
  // derivative of a line, which is then scaled by -2/h, so the lift enters as (1/w0)(F* - F)
  double rw0d;
  float rw0f;
  // dt, ca, cb rounded to FP32 on the host (the FP32 kernels read them without an FP64
  // conversion, which the FP64 pipe would carry), and ca == 0 (the first stage)
  float dtf, caf, cbf;
  int32_t first;
};

// The stage's Shu-Osher coefficients in T and whether it is the first stage.
template <class T>
struct StageCoef {
  T dt, ca, cb;
  bool first;
};
template <class T> __device__ __forceinline__ StageCoef<T> stage_coef(const StageArgs& A);
template <> __device__ __forceinline__ StageCoef<float> stage_coef<float>(const StageArgs& A) {
  return StageCoef<float>{A.dtf, A.caf, A.cbf, A.first != 0};
}
template <> __device__ __forceinline__ StageCoef<double> stage_coef<double>(const StageArgs& A) {
  return StageCoef<double>{A.dt, A.ca, A.cb, A.first != 0};
}

struct MortarArgs {
  const void* qs;
  const void* pp_in;
  void* mbuf;
  int64_t plane;
  int32_t G;
  const int32_t* groups; // [G][7]: coarse element, axis, side, fine elements (Morton order)
  const double* bg;
  const void* bgt;
  const double* bgc;
  const void* ops;
  float gammaf;
  PhysC ph;
  const int32_t* glist;  // the launch's mortar groups (a part of an SFC partition); null: 0 .. G-1
};

template <class T> __device__ __forceinline__ T gamma_of(const PhysC& ph, float gf) {
  return sizeof(T) == 4 ? (T)gf : (T)ph.gamma;
}

template <class T> __device__ __forceinline__ T lift_of(const StageArgs& A, int level, int a);
template <> __device__ __forceinline__ float lift_of<float>(const StageArgs& A, int level, int a) {
  return A.liftf[level][a];
}
template <> __device__ __forceinline__ double lift_of<double>(const StageArgs& A, int level, int a) {
  return A.liftd[level][a];
}

template <class T> __device__ __forceinline__ T inv2h_of(const StageArgs& A, int level, int a);
template <> __device__ __forceinline__ float inv2h_of<float>(const StageArgs& A, int level, int a) {
  return A.inv2hf[level][a];
}
template <> __device__ __forceinline__ double inv2h_of<double>(const StageArgs& A, int level, int a) {
  return A.inv2hd[level][a];
}

template <int D, int N>
__device__ __forceinline__ int face_node(int a, int side, int t) {
  // element node index of tangential position t on face (a, side); tangential axes ascending,
  // the lower one fastest
  constexpr int n1 = N + 1;
  int idx[3] = {0, 0, 0};
  idx[a] = side ? N : 0;
  int r = t;
#pragma unroll
  for (int b = 0; b < D; ++b)
    if (b != a) { idx[b] = r % n1; r /= n1; }
  return idx[0] + n1 * (idx[1] + n1 * idx[2]);
}

// Dynamic shared memory of the node-per-thread layout: D, then the flux tile [EPB][NV][NP].
template <class T, int D, int N, int EPB>
__host__ __device__ constexpr size_t node_smem_bytes() {
  return sizeof(T) * ((size_t)(N + 1) * (N + 1) + (size_t)EPB * (D + 2) * ipow(N + 1, D));
}

// Body of the node-per-thread stage kernel for the EPB elements e0, e0 + 1, ... of mesh A.
// Threads beyond EPB (N+1)^d (a persistent block of a fixed size) only take part in the
// barriers.
template <class T, int D, int N, int EPB>
__device__ __forceinline__ void stage_body_node(const StageArgs& A, int64_t e0) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);             // [n1 * n1]
  T* sF = sD + n1 * n1;                                // [EPB][NV][NP]
  const int tid = threadIdx.x;
  const T* ops = (const T*)A.ops;
  for (int i = tid; i < n1 * n1; i += blockDim.x) sD[i] = ops[i];
  const T gamma = gamma_of<T>(A.ph, A.gammaf);
  const int le = tid / NP, n = tid - le * NP;
  const bool inblk = le < EPB;
  const int64_t e = e0 + le;
  const bool valid = inblk && e < A.E;
  int idx[3];
  idx[0] = n % n1;
  idx[1] = (n / n1) % n1;
  idx[2] = (D == 3) ? n / (n1 * n1) : 0;
  const int P = A.plane32;
  const T* qe = (const T*)A.qs + (valid ? e : 0) * NP;
  const T* ppe = (const T*)A.pp_in + (valid ? e : 0) * NP;
  T q[NV], acc[NV], inv2h[D];
  T pp = (T)0;
  NodeBg<T> bg{(T)1, (T)1, (T)1};
#pragma unroll
  for (int v = 0; v < NV; ++v) { q[v] = (T)0; acc[v] = (T)0; }
#pragma unroll
  for (int a = 0; a < D; ++a) inv2h[a] = (T)0;
  int level = 0;
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = qe[v * P + n];
    pp = ppe[n];
    level = A.elem[e * 4];
#pragma unroll
    for (int a = 0; a < D; ++a) inv2h[a] = inv2h_of<T>(A, level, a);
    const T* b = (const T*)A.bgt + ((size_t)e * n1 + idx[D - 1]) * 4;
    bg.rb = b[0]; bg.Tb = b[1]; bg.pb = b[2];
    acc[D] = -(q[0] * (T)A.ph.g);   // buoyancy -rho' g on the vertical momentum
  }
  const NodeDer<T> nd = node_der<T, D>(q, bg);
  __syncthreads();
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T F[NV];
    flux_axis<T, D>(q, nd, pp, a, F);
    if (inblk) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sF[(le * NV + v) * NP + n] = F[v];
    }
    __syncthreads();
    if (valid) {
      const int stride = ipow(n1, a);
      const int ia = idx[a];
      const int b0 = n - ia * stride;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T s = (T)0;
#pragma unroll
        for (int m = 0; m < n1; ++m) s = fma(sD[ia * n1 + m], sF[(le * NV + v) * NP + b0 + m * stride], s);
        acc[v] = fma(-inv2h[a], s, acc[v]);
      }
    }
    __syncthreads();
  }
  if (!valid) return;
  const T* mbuf = (const T*)A.mbuf;
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (idx[a] != (s ? N : 0)) continue;
      const int32_t* c = A.conn + ((size_t)e * 2 * D + 2 * a + s) * 5;
      const int kind = c[0];
      int t = 0, mul = 1;
#pragma unroll
      for (int b = 0; b < D; ++b)
        if (b != a) { t += idx[b] * mul; mul *= n1; }
      T Fo[NV], Fs[NV];
      flux_axis<T, D>(q, nd, pp, a, Fo);
      if (kind == FACE_WALL || kind == FACE_CONF) {
        const T so = wave_speed<T>(q, nd, bg, pp, a, gamma);
        T qo[NV], Fn[NV], sn;
        if (kind == FACE_WALL) {
          // mirror state: same Theta, rho and P', normal momentum negated
#pragma unroll
          for (int v = 0; v < NV; ++v) qo[v] = q[v];
          qo[1 + a] = -q[1 + a];
          flux_axis<T, D>(qo, nd, pp, a, Fn);
          sn = so;
        } else {
          // the neighbour's matching node: same tangential indices, opposite face; its z (hence
          // its background) is bit-identical to this node's
          const int stride_a = (a == 0) ? 1 : (a == 1 ? n1 : n1 * n1);
          const int no = n + ((s ? 0 : N) - idx[a]) * stride_a;
          const T* qb = (const T*)A.qs + (int64_t)c[1] * NP;
#pragma unroll
          for (int v = 0; v < NV; ++v) qo[v] = qb[v * P + no];
          const T ppo = ((const T*)A.pp_in)[(int64_t)c[1] * NP + no];
          sn = face_side<T, D>(qo, bg, ppo, a, gamma, Fn);
        }
        if (s) rusanov<T, D>(q, Fo, so, qo, Fn, sn, Fs);
        else   rusanov<T, D>(qo, Fn, sn, q, Fo, so, Fs);
      } else {
        const int64_t g = (kind == FACE_FINE) ? c[2] : c[1];
        const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
        const T* src = mbuf + (((size_t)g * (1 + NSUB) + slot) * NV) * NF + t;
#pragma unroll
        for (int v = 0; v < NV; ++v) Fs[v] = src[(size_t)v * NF];
      }
      const T coef = s ? -lift_of<T>(A, level, a) : lift_of<T>(A, level, a);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += coef * (Fs[v] - Fo[v]);
    }
  }
  T* oute = (T*)A.out + e * NP;
  if (A.mode == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) oute[v * P + n] = acc[v];
    return;
  }
  T qnew[NV];
  const StageCoef<T> sc = stage_coef<T>(A);
  const T dt = sc.dt;
  if (sc.first) {
#pragma unroll
    for (int v = 0; v < NV; ++v) qnew[v] = q[v] + dt * acc[v];
  } else {
    const T ca = sc.ca, cb = sc.cb;
    const T* qne = (const T*)A.qn + e * NP;
#pragma unroll
    for (int v = 0; v < NV; ++v) qnew[v] = ca * qne[v * P + n] + cb * (q[v] + dt * acc[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) oute[v * P + n] = qnew[v];
  const size_t zk = (size_t)e * n1 + idx[D - 1];
  ((T*)A.pp_out)[e * NP + n] =
      pprime_of<T>(qnew[D + 1], ((const T*)A.bgt)[zk * 4 + 3], A.bg + zk * 4, A.bgc + zk, A.ph);
}

template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D))
stage_kernel(const __grid_constant__ StageArgs A) {
  stage_body_node<T, D, N, EPB>(A, (int64_t)A.e_begin + (int64_t)blockIdx.x * EPB);
}

// Batched form: block b works on mesh tab[map[b].x], elements from map[b].y.
template <class T, int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D))
stage_kernel_batched(const StageArgs* __restrict__ tab, const int2* __restrict__ map) {
  const int2 bm = map[blockIdx.x];
  stage_body_node<T, D, N, EPB>(tab[bm.x], (int64_t)bm.y);
}

// P' of every node of a state (FP64 evaluation, stored in T): used when a state enters from
// outside the time loop (set_state, initial condition, transfer, dg_rhs input).
template <class T>
__global__ void pprime_kernel(int64_t total, int NP, int n1, int D, const T* theta_plane,
                              const double* bg, const double* bgc, PhysC ph, T* pp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int k = D == 3 ? n / (n1 * n1) : n / n1;
  const int64_t zk = e * n1 + k;
  pp[i] = pprime_of<T>(theta_plane[i], (T)bg[zk * 4 + 3], bg + zk * 4, bgc + zk, ph);
}

// One CTA per mortar group; NSUB * NF threads: thread (m, t) owns mortar node t of mortar m.
template <class T, int D, int N>
__global__ void __launch_bounds__((1 << (D - 1)) * ipow(N + 1, D - 1))
mortar_kernel(const __grid_constant__ MortarArgs A) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  __shared__ T sP[2][n1 * n1], sC[2][n1 * n1];
  __shared__ T sQc[NV][NF];
  __shared__ T sT[NSUB][NV][NF];
  __shared__ T sM[NSUB][NV][NF];
  const int tid = threadIdx.x;
  // a stage kernel launched after this one may start now; it waits for this grid's completion
  // before it reads the mortar buffer
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const T* ops = (const T*)A.ops;
  for (int i = tid; i < n1 * n1; i += blockDim.x) {
    sP[0][i] = ops[1 * n1 * n1 + i];
    sP[1][i] = ops[2 * n1 * n1 + i];
    sC[0][i] = ops[3 * n1 * n1 + i];
    sC[1][i] = ops[4 * n1 * n1 + i];
  }
  const int g = A.glist ? A.glist[blockIdx.x] : (int)blockIdx.x;
  const int32_t* row = A.groups + (size_t)g * 7;
  const int64_t ec = row[0];
  const int a = row[1], side = row[2];
  const int m = tid / NF, t = tid - m * NF;
  const T* qs = (const T*)A.qs;
  // the fine trace and background of this thread's mortar node, requested together with the
  // coarse trace below rather than after the projections (one memory round trip instead of two)
  const int64_t ef = row[3 + m];
  const int nf = face_node<D, N>(a, 1 - side, t);
  T qf[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) qf[v] = qs[(size_t)v * A.plane + (size_t)ef * NP + nf];
  const int kf = (D == 3) ? nf / (n1 * n1) : nf / n1;
  const size_t zf = (size_t)ef * n1 + kf;
  const T* bt = (const T*)A.bgt + zf * 4;
  const NodeBg<T> bgf{bt[0], bt[1], bt[2]};
  const T invTbf = bt[3];
  const T ppf = ((const T*)A.pp_in)[(size_t)ef * NP + nf];
  for (int i = tid; i < NV * NF; i += blockDim.x) {
    const int v = i / NF, tt = i - v * NF;
    sQc[v][tt] = qs[(size_t)v * A.plane + (size_t)ec * NP + face_node<D, N>(a, side, tt)];
  }
  __syncthreads();
  // sub-face bits of mortar m over the tangential axes (lower axis first)
  const int b0 = m & 1, b1 = (m >> 1) & 1;
  const int t0 = t % n1, t1 = t / n1;
  // coarse trace -> mortar m, first tangential axis
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T s = (T)0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s = fma(sP[b0][t0 * n1 + j], sQc[v][j + n1 * t1], s);
    sT[m][v][t] = s;
  }
  __syncthreads();
  if (D == 3) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T s = (T)0;
#pragma unroll
      for (int j = 0; j < n1; ++j) s = fma(sP[b1][t1 * n1 + j], sT[m][v][t0 + n1 * j], s);
      sM[m][v][t] = s;
    }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) sM[m][v][t] = sT[m][v][t];
  }
  __syncthreads();
  // Rusanov on mortar node (m, t); the fine face is the mortar (identity projection), and the
  // projected coarse state takes the fine side's background (the mortar points' heights)
  T qc[NV], Fs[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) qc[v] = sM[m][v][t];
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
    sM[m][v][t] = Fs[v];
  }
  __syncthreads();
  // back to the coarse face: sum_m (C_b1 x C_b0) F*_m
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T s = (T)0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s = fma(sC[b0][t0 * n1 + j], sM[m][v][j + n1 * t1], s);
    sT[m][v][t] = s;
  }
  __syncthreads();
  if (m == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = (T)0;
      for (int mm = 0; mm < NSUB; ++mm) {
        if (D == 3) {
          const int c1 = (mm >> 1) & 1;
          T s = (T)0;
#pragma unroll
          for (int j = 0; j < n1; ++j) s = fma(sC[c1][t1 * n1 + j], sT[mm][v][t0 + n1 * j], s);
          acc += s;
        } else {
          acc += sT[mm][v][t];
        }
      }
      mb[(size_t)v * NF + t] = acc;
    }
  }
}

}  // namespace dgk
