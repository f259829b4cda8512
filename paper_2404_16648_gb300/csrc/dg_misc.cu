// Helper kernels of the GB300 dGSEM library that run once per regrid or per diagnostic:
// hydrostatic background (FP64), initial bubble, refinement indicator, compensated integrals
// and the conservative parent<->child transfer of Sec. 3.3.
#include "dg_launch.hpp"
#include "../../include/dg.h"

#include <cmath>

namespace dgk {
namespace {

__device__ __forceinline__ double node_coord(int c, double xi, double h) {
  // (c + (xi + 1)/2) h: faces shared by two elements get bit-identical coordinates
  return (c + (xi + 1.0) * 0.5) * h;
}

// Hydrostatic neutral background at the z-nodes of every element (Sec. 4.3):
// pi = 1 - g z / (cp theta0), rho_bar = p0 pi^(cv/R) / (R theta0), Theta_bar = rho_bar theta0,
// p_bar := P(Theta_bar) = p0 (R Theta_bar / p0)^gamma so that a fluid at rest has P' = 0.
__global__ void background_kernel(int32_t E, int n1, int D, const int32_t* elem,
                                  const double* xi, double root_hz, PhysC ph, double* bg,
                                  float* bgf, double* bgc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)E * n1) return;
  const int64_t e = i / n1;
  const int k = (int)(i - e * n1);
  const int level = elem[e * 4];
  const double hz = ldexp(root_hz, -level);
  const double z = node_coord(elem[e * 4 + D], xi[k], hz);
  const double pi = 1.0 - ph.g * z / (ph.cp * ph.theta0);
  const double rb = ph.p0 * pow(pi, ph.cv / ph.R) / (ph.R * ph.theta0);
  const double Tb = rb * ph.theta0;
  const double pb = ph.p0 * pow(ph.R * Tb / ph.p0, ph.gamma);
  double* o = bg + i * 4;
  o[0] = rb; o[1] = Tb; o[2] = pb; o[3] = 1.0 / Tb;
  if (bgf) {
    float* f = bgf + i * 4;
    f[0] = (float)rb; f[1] = (float)Tb; f[2] = (float)pb; f[3] = (float)(1.0 / Tb);
    bgc[i] = ph.gamma * pb / Tb;
  }
}

template <class T>
__global__ void bubble_kernel(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                              double rh0, double rh1, double rh2, const double* bg,
                              double c0, double c1, double c2, double r0, double r1, double r2,
                              double amp, int n_rff, double rff_scale, const double* rff_k,
                              const double* rff_phase, double theta0, T* q, int64_t plane,
                              double* theta_out) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)E * NP) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
  const int level = elem[e * 4];
  const double rh[3] = {rh0, rh1, rh2}, cen[3] = {c0, c1, c2}, rad[3] = {r0, r1, r2};
  double x[3] = {0.0, 0.0, 0.0};
  double r2s = 0.0;
  for (int a = 0; a < D; ++a) {
    x[a] = node_coord(elem[e * 4 + 1 + a], xi[idx[a]], ldexp(rh[a], -level));
    const double s = (x[a] - cen[a]) / rad[a];
    r2s = r2s + s * s;
  }
  const double r = sqrt(r2s);
  double th = r <= 1.0 ? amp * (1.0 + cos(M_PI * r)) : 0.0;
  if (n_rff > 0) {
    double acc = 0.0;
    for (int m = 0; m < n_rff; ++m) {
      double arg = rff_phase[m];
      for (int a = 0; a < D; ++a) arg = arg + rff_k[m * 3 + a] * x[a];
      acc = acc + cos(arg);
    }
    th = th + rff_scale * acc;
  }
  if (theta_out) { theta_out[i] = th; return; }
  const double rb = bg[(e * n1 + idx[D - 1]) * 4];
  q[i] = (T)(-rb * th / (theta0 + th));
  for (int v = 1; v < D + 2; ++v) q[(int64_t)v * plane + i] = (T)0;
}

// max over the element's nodes of |theta'|, theta' = (Theta_bar + Theta') / (rho_bar + rho')
// - theta0, in FP64 (refinement criterion of Sec. 4.3, tagging by potential temperature).
//
// One warp per element.  With A = Theta_bar + Theta' and B = rho_bar + rho' as FP64 forms them,
// fl(A/B) and then fl(fl(A/B) - theta0) are monotone in the exact quotient A/B = theta0 + D/B,
// D = A - theta0 B, so the largest |theta'| sits at the node of largest or of smallest D/B.  A
// first pass bounds every D/B in FP32 (indicator_screen: an estimate t and an interval
// [lo, hi] that holds D/B); a node can hold the largest D/B only if hi >= max(lo) and the
// smallest only if lo <= min(hi).  Only those nodes take the FP64 division, and the result is
// the value the division at every node gives.  D is formed from per-layer constants
// C = fl64(Theta_bar - theta0 rho_bar) and the perturbations, so the interval is as narrow
// relative to theta' as to theta: elements near the background need no more divisions than
// the rest.  An element with a node outside the bounds' range (a non-finite value, the FP32
// density estimate outside [1e-6, 1e30] or within 4 error bounds of zero) takes the division
// at every node instead.
constexpr int kIndWarps = 8;

struct IndScreen {
  float lo, hi;
  bool ok;
};

// FP32 interval [lo, hi] around D/B for one node.  c, b0f, b1f: C, rho_bar, Theta_bar rounded to
// FP32; thf = fl32(theta0) and dth >= |thf - theta0|.  Every FP32 operation is rounded once
// (no contraction) and contributes at most 2^-24 of its result, every FP32 conversion 2^-24 of
// its value, the FP64 sums 2^-53; the terms below bound these with a factor of 4 to spare.
// Underflow adds at most 2^-126 per operation, which the 1e-36 terms cover once the density
// estimate is at least 1e-6.  __fdividef is within 2 ulp for divisors in [2^-126, 2^126].
template <class T>
__device__ __forceinline__ IndScreen indicator_screen(float c, float b0f, float b1f, T q0, T q3,
                                                      float thf, float dth) {
  const float q0f = (float)q0, q3f = (float)q3;
  const float p = __fmul_rn(thf, q0f);
  const float Qh = __fsub_rn(q3f, p);
  const float Dh = __fadd_rn(c, Qh);
  const float bh = __fadd_rn(b0f, q0f);
  const float a0 = fabsf(q0f), a3 = fabsf(q3f);
  // |Dh - D| <= eD
  float eD = __fadd_rn(__fadd_rn(fabsf(c), a3), __fmul_rn(thf, a0));
  eD = __fadd_rn(eD, __fadd_rn(__fadd_rn(fabsf(p), fabsf(Qh)), fabsf(Dh)));
  eD = __fmul_rn(eD, 0x1p-21f);
  eD = __fadd_rn(eD, __fmul_rn(dth, a0));
  // FP64 rounding of A and B: none where the perturbation is zero
  const float rA = q3 == T(0) ? 0.0f : __fadd_rn(fabsf(b1f), a3);
  const float rB = q0 == T(0) ? 0.0f : __fadd_rn(fabsf(b0f), a0);
  const float big = __fadd_rn(rA, __fmul_rn(thf, rB));
  eD = __fadd_rn(__fadd_rn(eD, __fmul_rn(big, 0x1p-50f)), 1e-36f);
  // |bh - B| <= eB
  float eB = __fmul_rn(__fadd_rn(__fadd_rn(fabsf(b0f), a0), fabsf(bh)), 0x1p-21f);
  eB = __fadd_rn(__fadd_rn(eB, __fmul_rn(rB, 0x1p-50f)), 1e-36f);
  // |t - D/B| <= 2^-21 |t| + (eD + (|D| + eD) eB / (3/4 bh)) / bh, doubled
  const float t = __fdividef(Dh, bh);
  float e = __fmul_rn(__fmul_rn(__fadd_rn(fabsf(Dh), eD), eB), __fdividef(2.0f, bh));
  e = __fdividef(__fadd_rn(eD, e), bh);
  e = __fadd_rn(__fadd_rn(__fmul_rn(fabsf(t), 0x1p-20f), e), 1e-36f);
  e = __fmul_rn(e, 2.0f);
  IndScreen r;
  r.lo = __fsub_rn(t, e);
  r.hi = __fadd_rn(t, e);
  r.ok = bh >= 1e-6f && bh <= 1e30f && bh >= __fmul_rn(4.0f, eB) && isfinite(r.lo) && isfinite(r.hi);
  return r;
}

template <class T>
__global__ void indicator_kernel(int32_t E, int n1, int D, const double* bg, const T* q,
                                 int64_t plane, double theta0, float thf, float dth, double* out) {
  __shared__ float lay[kIndWarps][DG_MAX_N + 1][3];
  __shared__ uint16_t cand[kIndWarps][(DG_MAX_N + 1) * (DG_MAX_N + 1) * (DG_MAX_N + 1)];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kIndWarps + w;
  if (e >= E) return;   // whole warps leave together; no block-wide barrier below
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int layer = D == 3 ? n1 * n1 : n1;
  // node n lies in layer (n * M) >> 20, M = ceil(2^20 / layer): exact for n < 729, layer <= 81
  const uint32_t M = ((1u << 20) + (uint32_t)layer - 1) / (uint32_t)layer;
  const T* q0 = q + e * NP;
  const T* q3 = q + (int64_t)(D + 1) * plane + e * NP;
  const double* be = bg + e * n1 * 4;
  if (lane < n1) {
    const double b0 = be[lane * 4], b1 = be[lane * 4 + 1];
    lay[w][lane][0] = (float)fma(-theta0, b0, b1);
    lay[w][lane][1] = (float)b0;
    lay[w][lane][2] = (float)b1;
  }
  __syncwarp();
  float L = -INFINITY, U = INFINITY;
  bool fast = true;
  for (int n = lane; n < NP; n += 32) {
    const int k = (int)(((uint32_t)n * M) >> 20);
    const IndScreen s = indicator_screen<T>(lay[w][k][0], lay[w][k][1], lay[w][k][2], q0[n], q3[n], thf, dth);
    fast = fast && s.ok;
    L = fmaxf(L, s.lo);
    U = fminf(U, s.hi);
  }
  for (int o = 16; o > 0; o >>= 1) {
    L = fmaxf(L, __shfl_xor_sync(0xffffffffu, L, o));
    U = fminf(U, __shfl_xor_sync(0xffffffffu, U, o));
  }
  fast = __all_sync(0xffffffffu, fast);
  double m;
  if (fast) {
    // candidates: nodes with both perturbations zero share fl(A/B) = fl(Theta_bar / rho_bar)
    // with their layer and are marked per layer; the others are packed into a per-warp list
    // {node, may be the largest, may be the smallest} so the divisions take ceil(count / 32)
    // rounds of the warp
    uint32_t cmask = 0, xmask = 0, nmask = 0, lmax = 0, lmin = 0;
    for (int j = 0, n = lane; n < NP; ++j, n += 32) {
      const int k = (int)(((uint32_t)n * M) >> 20);
      const IndScreen s = indicator_screen<T>(lay[w][k][0], lay[w][k][1], lay[w][k][2], q0[n], q3[n], thf, dth);
      const bool cmax = s.hi >= L, cmin = s.lo <= U;
      if (!(cmax || cmin)) continue;
      if (q0[n] == T(0) && q3[n] == T(0)) {
        lmax |= (uint32_t)cmax << k;
        lmin |= (uint32_t)cmin << k;
      } else {
        cmask |= 1u << j;
        xmask |= (uint32_t)cmax << j;
        nmask |= (uint32_t)cmin << j;
      }
    }
    const int cnt = __popc(cmask);
    int off = cnt;   // inclusive scan over lanes, then exclusive
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, off, o);
      if (lane >= o) off += v;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;
    for (uint32_t b = cmask; b; b &= b - 1) {
      const int j = __ffs(b) - 1;
      cand[w][off++] = (uint16_t)((lane + 32 * j) | (((xmask >> j) & 1u) << 14) | (((nmask >> j) & 1u) << 15));
    }
    lmax = __reduce_or_sync(0xffffffffu, lmax);
    lmin = __reduce_or_sync(0xffffffffu, lmin);
    __syncwarp();
    double vmax = -INFINITY, vmin = INFINITY;
    for (int c = lane; c < total; c += 32) {
      const uint32_t x = cand[w][c];
      const int n = (int)(x & 0x3fffu);
      const int k = (int)(((uint32_t)n * M) >> 20);
      const double v = (be[k * 4 + 1] + (double)q3[n]) / (be[k * 4] + (double)q0[n]);
      if (x & (1u << 14)) vmax = fmax(vmax, v);
      if (x & (1u << 15)) vmin = fmin(vmin, v);
    }
    if (lane < n1 && (((lmax | lmin) >> lane) & 1u)) {
      const double v = (be[lane * 4 + 1] + 0.0) / (be[lane * 4] + 0.0);
      if ((lmax >> lane) & 1u) vmax = fmax(vmax, v);
      if ((lmin >> lane) & 1u) vmin = fmin(vmin, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    }
    m = fmax(fabs(vmax - theta0), fabs(vmin - theta0));
  } else {
    m = 0.0;
    for (int n = lane; n < NP; n += 32) {
      const int k = (int)(((uint32_t)n * M) >> 20);
      m = fmax(m, fabs((be[k * 4 + 1] + (double)q3[n]) / (be[k * 4] + (double)q0[n]) - theta0));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if (lane == 0) out[e] = m;
}

// Refinement tags of the theta' criterion: tag[e] = (the indicator of element e > thr), with
// the indicator as indicator_kernel returns it, decided without forming it where the FP32
// intervals of indicator_screen settle the comparison.  |fl(fl(A/B) - theta0)| differs from
// |D/B| by the two FP64 roundings, below 2^-52 (|A/B| + |theta0|), which the margin `del`
// (host: 2^-30 (|theta0| + |thr|)) covers many times over: a node is certainly above the
// threshold when its interval lies beyond +-fh >= thr + del, certainly below when it lies
// within +-fl <= thr - del.  Only an element with no node certainly above and some node that
// is neither takes FP64 divisions, at those nodes; an element outside the bounds' range, or a
// threshold too small for the margins (screen == 0), takes them at every node.  Non-finite
// values compare false, as the indicator's fmax leaves them out.
template <class T>
__global__ void tag_kernel(int32_t E, int n1, int D, const double* bg, const T* q, int64_t plane,
                           double theta0, float thf, float dth, double thr, float fh, float fl, int screen,
                           uint8_t* tag) {
  __shared__ float lay[kIndWarps][DG_MAX_N + 1][3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kIndWarps + w;
  if (e >= E) return;   // whole warps leave together; no block-wide barrier below
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int layer = D == 3 ? n1 * n1 : n1;
  const uint32_t M = ((1u << 20) + (uint32_t)layer - 1) / (uint32_t)layer;
  const T* q0 = q + e * NP;
  const T* q3 = q + (int64_t)(D + 1) * plane + e * NP;
  const double* be = bg + e * n1 * 4;
  if (lane < n1) {
    const double b0 = be[lane * 4], b1 = be[lane * 4 + 1];
    lay[w][lane][0] = (float)fma(-theta0, b0, b1);
    lay[w][lane][1] = (float)b0;
    lay[w][lane][2] = (float)b1;
  }
  __syncwarp();
  auto exceeds = [&](int n) {
    const int k = (int)(((uint32_t)n * M) >> 20);
    return fabs((be[k * 4 + 1] + (double)q3[n]) / (be[k * 4] + (double)q0[n]) - theta0) > thr;
  };
  bool above = false, unsure = false;
  if (screen) {
    bool ok = true;
    for (int n = lane; n < NP; n += 32) {
      const int k = (int)(((uint32_t)n * M) >> 20);
      const IndScreen s = indicator_screen<T>(lay[w][k][0], lay[w][k][1], lay[w][k][2], q0[n], q3[n], thf, dth);
      ok = ok && s.ok;
      above = above || s.lo > fh || s.hi < -fh;
      unsure = unsure || !(s.hi < fl && s.lo > -fl);
    }
    if (__all_sync(0xffffffffu, ok)) {
      above = __any_sync(0xffffffffu, above);
      unsure = __any_sync(0xffffffffu, unsure);
      if (!above && unsure) {
        bool hit = false;
        for (int n = lane; n < NP; n += 32) {
          const int k = (int)(((uint32_t)n * M) >> 20);
          const IndScreen s = indicator_screen<T>(lay[w][k][0], lay[w][k][1], lay[w][k][2], q0[n], q3[n], thf, dth);
          if (!(s.hi < fl && s.lo > -fl)) hit = hit || exceeds(n);
        }
        above = __any_sync(0xffffffffu, hit);
      }
      if (lane == 0) tag[e] = above ? 1 : 0;
      return;
    }
  }
  bool hit = false;
  for (int n = lane; n < NP; n += 32) hit = hit || exceeds(n);
  hit = __any_sync(0xffffffffu, hit);
  if (lane == 0) tag[e] = hit ? 1 : 0;
}

// Primitive diagnostics per node in FP64: out[a] = U_a / rho (a < D), out[D] = theta'
// = (Theta_bar + Theta') / (rho_bar + rho') - theta0; planes of length E * NP.
template <class T>
__global__ void primitives_kernel(int32_t E, int n1, int D, const double* bg, const T* q,
                                  int64_t plane, double theta0, double* out) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t e = i / NP;
  const int n = (int)(i - e * NP);
  const int k = D == 3 ? n / (n1 * n1) : n / n1;
  const double* b = bg + (e * n1 + k) * 4;
  const double rho = b[0] + (double)q[i];
  for (int a = 0; a < D; ++a) out[a * total + i] = (double)q[(int64_t)(1 + a) * plane + i] / rho;
  out[D * total + i] = (b[1] + (double)q[(int64_t)(D + 1) * plane + i]) / rho - theta0;
}

// Neumaier-compensated accumulator.
struct Comp {
  double s, c;
  __device__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ void merge(const Comp& o) { add(o.s); c += o.c; }
};

constexpr int kIntBlocks = 1216;    // 8 per SM
constexpr int kIntThreads = 256;
constexpr int kMaxNP = 729;          // (N + 1)^3 for N = 8

// Compensated partial sums over the nodes, weights w_i w_j (w_k) |J|.  The total energy
// p cv/R + |U|^2/(2 rho) + rho g z splits into a part of the background alone and a part that
// carries the state, and so does the mass:
//   BG = true:  {int rho_bar, int (p_bar cv/R + rho_bar g z), int 1}   (once per mesh)
//   BG = false: {int rho', int (P' cv/R + |U|^2/(2 rho) + rho' g z), int |U|^2/(2 rho)}
// Each thread sums its nodes of one element in plain FP64 and adds that subtotal to its
// Neumaier accumulator; blocks then reduce in a fixed tree order, and a final pass walks the
// block partials in order, so the result is deterministic.  Node weights and z-levels come
// from per-block tables, so no node needs an integer division.
template <class T, bool BG>
__global__ void __launch_bounds__(kIntThreads)
integrals_partial(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                  const double* w, double rh0, double rh1, double rh2, const double* bg,
                  const T* q, int64_t plane, PhysC ph, double* partial, int* bad) {
  __shared__ double sW[kMaxNP];
  __shared__ double sXh[9];
  __shared__ unsigned char sK[kMaxNP];
  const int tid = threadIdx.x;
  const int NF = D == 3 ? n1 * n1 : n1;
  const int NP = NF * n1;
  for (int n = tid; n < NP; n += blockDim.x) {
    const int i = n % n1, k = n / NF;
    double wn = w[i];
    if (D == 3) wn = wn * w[(n / n1) % n1];
    sW[n] = wn * w[k];
    sK[n] = (unsigned char)k;
  }
  if (tid < n1) sXh[tid] = (xi[tid] + 1.0) * 0.5;
  __syncthreads();
  const int epi = NP >= (int)blockDim.x ? 1 : (int)blockDim.x / NP;   // elements per pass
  const int le = epi > 1 ? tid / NP : 0;
  const int n0 = epi > 1 ? tid - le * NP : tid;
  const int nstride = epi > 1 ? NP : (int)blockDim.x;
  const double rh[3] = {rh0, rh1, rh2};
  const double cvR = ph.cv / ph.R;
  Comp acc[3];
  for (int k = 0; k < 3; ++k) acc[k] = Comp{0.0, 0.0};
  int nonfinite = 0;
  for (int64_t eb = (int64_t)blockIdx.x * epi; eb < E; eb += (int64_t)gridDim.x * epi) {
    const int64_t e = eb + le;
    if (le >= epi || e >= E) continue;
    const int level = elem[e * 4];
    double J = 1.0;
    for (int a = 0; a < D; ++a) J = J * (ldexp(rh[a], -level) * 0.5);
    const double hz = ldexp(rh[D - 1], -level);
    const double cz = (double)elem[e * 4 + D];
    double l0 = 0.0, l1 = 0.0, l2 = 0.0;
    for (int n = n0; n < NP; n += nstride) {
      const int k = sK[n];
      const double W = sW[n] * J;
      const double* b = bg + (e * n1 + k) * 4;
      const double z = (cz + sXh[k]) * hz;
      if (BG) {
        const double rb = b[0];
        l0 += W * rb;
        l1 += W * (b[2] * cvR + rb * ph.g * z);
        l2 += W;
      } else {
        const int64_t i = e * NP + n;
        const double rp = (double)q[i];
        const double rho = b[0] + rp;
        double u2 = 0.0;
        for (int a = 0; a < D; ++a) {
          const double U = (double)q[(int64_t)(1 + a) * plane + i];
          u2 = u2 + U * U;
        }
        const double ke = 0.5 * u2 / rho;
        const double pp = pressure_pert<kSeries>((double)q[(int64_t)(D + 1) * plane + i], b[3], b[2], ph);
        const double ep = pp * cvR + ke + rp * ph.g * z;
        if (!isfinite(rho) || !isfinite(ep)) nonfinite = 1;
        l0 += W * rp;
        l1 += W * ep;
        l2 += W * ke;
      }
    }
    acc[0].add(l0);
    acc[1].add(l1);
    acc[2].add(l2);
  }
  if (nonfinite) atomicOr(bad, 1);
  __shared__ double ss[3][kIntThreads], sc[3][kIntThreads];
  for (int k = 0; k < 3; ++k) { ss[k][tid] = acc[k].s; sc[k][tid] = acc[k].c; }
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (tid < st)
      for (int k = 0; k < 3; ++k) {
        Comp a{ss[k][tid], sc[k][tid]};
        a.merge(Comp{ss[k][tid + st], sc[k][tid + st]});
        ss[k][tid] = a.s; sc[k][tid] = a.c;
      }
    __syncthreads();
  }
  if (tid == 0)
    for (int k = 0; k < 3; ++k) {
      partial[(blockIdx.x * 3 + k) * 2] = ss[k][0];
      partial[(blockIdx.x * 3 + k) * 2 + 1] = sc[k][0];
    }
}

// Final pass, one CTA of kIntThreads: thread t merges a fixed contiguous run of block partials
// in order, then the threads reduce in a fixed tree (deterministic).  out[k] = s + c rounded,
// out[3 + k] its rounding error, so that a later sum of two such results loses nothing.
__global__ void __launch_bounds__(kIntThreads) integrals_final(int nblocks, const double* partial, double* out) {
  __shared__ double ss[3][kIntThreads], sc[3][kIntThreads];
  const int tid = threadIdx.x;
  const int run = (nblocks + kIntThreads - 1) / kIntThreads;
  const int b0 = tid * run, b1 = min(nblocks, b0 + run);
  for (int k = 0; k < 3; ++k) {
    Comp a{0.0, 0.0};
    for (int b = b0; b < b1; ++b) a.merge(Comp{partial[(b * 3 + k) * 2], partial[(b * 3 + k) * 2 + 1]});
    ss[k][tid] = a.s; sc[k][tid] = a.c;
  }
  __syncthreads();
  for (int st = kIntThreads / 2; st > 0; st >>= 1) {
    if (tid < st)
      for (int k = 0; k < 3; ++k) {
        Comp a{ss[k][tid], sc[k][tid]};
        a.merge(Comp{ss[k][tid + st], sc[k][tid + st]});
        ss[k][tid] = a.s; sc[k][tid] = a.c;
      }
    __syncthreads();
  }
  if (tid < 3) {
    const double t = ss[tid][0] + sc[tid][0];
    out[tid] = t;
    out[3 + tid] = sc[tid][0] - (t - ss[tid][0]);   // |s| >= |c| for a compensated sum
  }
}

// The integrals' last step on the device (dg_integrals_async): the state sums S (three sums and
// their rounding errors) added to the background sums B with their rounding errors (TwoSum,
// explicitly rounded, so the bits are those of the host combination in dg_integrals):
//   res = {mass, total energy, kinetic energy, volume, perturbation mass, non-finite flag}.
__device__ __forceinline__ double two_sum_rn(double a, double b, double* err) {
  const double t = __dadd_rn(a, b);
  const double bb = __dsub_rn(t, a);
  *err = __dadd_rn(__dsub_rn(a, __dsub_rn(t, bb)), __dsub_rn(b, bb));
  return t;
}

__global__ void integrals_combine(const double* S, const double* B, const int* bad, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e0, e1;
  const double t0 = two_sum_rn(B[0], S[0], &e0);
  const double t1 = two_sum_rn(B[1], S[1], &e1);
  res[0] = __dadd_rn(t0, __dadd_rn(e0, __dadd_rn(B[3], S[3])));
  res[1] = __dadd_rn(t1, __dadd_rn(e1, __dadd_rn(B[4], S[4])));
  res[2] = S[2];
  res[3] = B[2];
  res[4] = S[0];
  res[5] = *bad ? 1.0 : 0.0;
}


// Conservative transfer after a regrid (Sec. 3.3), one CTA per new element, FP64 arithmetic:
//   keep:   copy;
//   child:  (P_{c_2} x P_{c_1} x P_{c_0}) parent, P_c the half-interval interpolation;
//   parent: sum_c (C_{c_2} x C_{c_1} x C_{c_0}) child_c, C_c = (1/2) M^{-1} S_c^T.
template <class T>
__global__ void transfer_kernel(int32_t Enew, int n1, int D, const int32_t* tmap,
                                const double* ops, const T* qold, int64_t plane_old, T* qnew,
                                int64_t plane_new, int nv) {
  extern __shared__ double sm[];
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int nn = n1 * n1;
  double* sP = sm;              // P0, P1, C0, C1
  double* s0 = sm + 4 * nn;
  double* s1 = s0 + NP;
  double* sacc = s1 + NP;
  for (int i = threadIdx.x; i < 4 * nn; i += blockDim.x) sP[i] = ops[nn + i];
  const int64_t e = blockIdx.x;
  const int32_t* row = tmap + e * 9;
  const int kind = row[0];
  const int n = threadIdx.x;
  int idx[3] = {n % n1, (n / n1) % n1, D == 3 ? n / (n1 * n1) : 0};
  __syncthreads();
  for (int v = 0; v < nv; ++v) {
    if (kind == 0) {
      if (n < NP) qnew[(int64_t)v * plane_new + e * NP + n] = qold[(int64_t)v * plane_old + (int64_t)row[1] * NP + n];
      continue;
    }
    const int nsrc = kind == 1 ? 1 : (1 << D);
    if (n < NP) sacc[n] = 0.0;
    for (int c = 0; c < nsrc; ++c) {
      const int64_t src = kind == 1 ? row[1] : row[1 + c];
      const int ci = kind == 1 ? row[2] : c;
      const double* mats = kind == 1 ? sP : sP + 2 * nn;
      __syncthreads();
      if (n < NP) s0[n] = (double)qold[(int64_t)v * plane_old + src * NP + n];
      __syncthreads();
      double* in = s0;
      double* out = s1;
      for (int a = 0; a < D; ++a) {
        const double* M = mats + ((ci >> a) & 1) * nn;
        const int stride = a == 0 ? 1 : (a == 1 ? n1 : nn);
        if (n < NP) {
          const int ia = idx[a];
          const int b0 = n - ia * stride;
          double s = 0.0;
          for (int m = 0; m < n1; ++m) s += M[ia * n1 + m] * in[b0 + m * stride];
          out[n] = s;
        }
        __syncthreads();
        double* t = in; in = out; out = t;
      }
      if (n < NP) sacc[n] += in[n];
    }
    __syncthreads();
    if (n < NP) qnew[(int64_t)v * plane_new + e * NP + n] = (T)sacc[n];
  }
}

}  // namespace

cudaError_t launch_background(int32_t E, int n1, int D, const int32_t* elem, const double* xi,
                              double root_hz, const PhysC& ph, double* bg, float* bgf,
                              double* bgc, cudaStream_t s) {
  const int64_t n = (int64_t)E * n1;
  if (n == 0) return cudaSuccess;
  background_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, n1, D, elem, xi, root_hz, ph, bg, bgf, bgc);
  return cudaGetLastError();
}

cudaError_t launch_pprime(int prec, int32_t E, int n1, int D, const void* theta_plane,
                          const double* bg, const double* bgc, const PhysC& ph, void* pp, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t n = (int64_t)E * NP;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 0)
    pprime_kernel<double><<<blocks, 256, 0, s>>>(n, NP, n1, D, (const double*)theta_plane, bg, bgc, ph, (double*)pp);
  else
    pprime_kernel<float><<<blocks, 256, 0, s>>>(n, NP, n1, D, (const float*)theta_plane, bg, bgc, ph, (float*)pp);
  return cudaGetLastError();
}

// Isentropic vortex of Sec. 4.1 (nondimensional: p0 = R = theta0 = 1, g = 0) moved to time t:
// T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) e^(1-r^2), rho = T^(1/(gamma-1)), theta = 1,
// (u, v) = (U, V) + beta/(2 pi) e^((1-r^2)/2) (-dy, dx); dx, dy nearest-image on joined axes.
template <class T>
__global__ void vortex_kernel(int32_t E, int n1, const int32_t* elem, const double* xi, double hx0,
                              double hy0, double lx, double ly, int perx, int pery, double cx,
                              double cy, double beta, double ux, double uy, double gamma,
                              const double* bg, T* q, int64_t plane) {
  const int NP = n1 * n1;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)E * NP) return;
  const int64_t e = k / NP;
  const int n = (int)(k - e * NP);
  const int i = n % n1, j = n / n1;
  const int level = elem[e * 4];
  const double x = node_coord(elem[e * 4 + 1], xi[i], ldexp(hx0, -level));
  const double y = node_coord(elem[e * 4 + 2], xi[j], ldexp(hy0, -level));
  double dx = x - cx, dy = y - cy;
  if (perx) dx = dx - lx * floor((dx + 0.5 * lx) / lx);
  if (pery) dy = dy - ly * floor((dy + 0.5 * ly) / ly);
  const double r2 = dx * dx + dy * dy;
  const double Tt = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * M_PI * M_PI) * exp(1.0 - r2);
  const double rho = pow(Tt, 1.0 / (gamma - 1.0));
  const double amp = beta / (2.0 * M_PI) * exp(0.5 * (1.0 - r2));
  const double u = ux - amp * dy, v = uy + amp * dx;
  const double* b = bg + (e * n1 + j) * 4;
  q[k] = (T)(rho - b[0]);
  q[plane + k] = (T)(rho * u);
  q[2 * plane + k] = (T)(rho * v);
  q[3 * plane + k] = (T)(rho - b[1]);
}

cudaError_t launch_vortex(int prec, int32_t E, int n1, const int32_t* elem, const double* xi,
                          const double* root_h, const double* length, const int* periodic,
                          const double* center, double beta, const double* uinf, double t,
                          double gamma, const double* bg, void* q, int64_t plane, cudaStream_t s) {
  const int64_t total = (int64_t)E * n1 * n1;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  const double cx = center[0] + uinf[0] * t, cy = center[1] + uinf[1] * t;
  if (prec == 0)
    vortex_kernel<double><<<grid, 256, 0, s>>>(E, n1, elem, xi, root_h[0], root_h[1], length[0], length[1],
                                               periodic[0], periodic[1], cx, cy, beta, uinf[0], uinf[1],
                                               gamma, bg, (double*)q, plane);
  else
    vortex_kernel<float><<<grid, 256, 0, s>>>(E, n1, elem, xi, root_h[0], root_h[1], length[0], length[1],
                                              periodic[0], periodic[1], cx, cy, beta, uinf[0], uinf[1],
                                              gamma, bg, (float*)q, plane);
  return cudaGetLastError();
}

cudaError_t launch_bubble(int prec, int32_t E, int n1, int D, const int32_t* elem,
                          const double* xi, const double* root_h, const double* bg,
                          const double* center, const double* radius, double amp, int n_rff,
                          double rff_scale, const double* rff_k, const double* rff_phase,
                          double theta0, void* q, int64_t plane, double* theta_out,
                          cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t n = (int64_t)E * NP;
  if (n == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == 0)
    bubble_kernel<double><<<blocks, 256, 0, s>>>(E, n1, D, elem, xi, root_h[0], root_h[1], root_h[2], bg,
        center[0], center[1], center[2], radius[0], radius[1], radius[2], amp, n_rff, rff_scale,
        rff_k, rff_phase, theta0, (double*)q, plane, theta_out);
  else
    bubble_kernel<float><<<blocks, 256, 0, s>>>(E, n1, D, elem, xi, root_h[0], root_h[1], root_h[2], bg,
        center[0], center[1], center[2], radius[0], radius[1], radius[2], amp, n_rff, rff_scale,
        rff_k, rff_phase, theta0, (float*)q, plane, theta_out);
  return cudaGetLastError();
}

cudaError_t launch_indicator(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                             int64_t plane, double theta0, double* out, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  const int grid = (int)((E + kIndWarps - 1) / kIndWarps);   // one warp per element
  // theta0 in FP32 and a bound on its rounding error, rounded up
  const float thf = (float)theta0;
  const float dth = (float)(std::fabs((double)thf - theta0) * (1.0 + 0x1p-20));
  if (prec == 0)
    indicator_kernel<double><<<grid, 32 * kIndWarps, 0, s>>>(E, n1, D, bg, (const double*)q, plane, theta0, thf, dth, out);
  else
    indicator_kernel<float><<<grid, 32 * kIndWarps, 0, s>>>(E, n1, D, bg, (const float*)q, plane, theta0, thf, dth, out);
  return cudaGetLastError();
}

cudaError_t launch_tags(int prec, int32_t E, int n1, int D, const double* bg, const void* q, int64_t plane,
                        double theta0, double thr, uint8_t* tag, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  const int grid = (int)((E + kIndWarps - 1) / kIndWarps);
  const float thf = (float)theta0;
  const float dth = (float)(std::fabs((double)thf - theta0) * (1.0 + 0x1p-20));
  const double del = std::ldexp(std::fabs(theta0) + std::fabs(thr), -30);
  // FP32 bounds on the FP64 thresholds: fh >= thr + del, fl <= thr - del
  float fh = (float)(thr + del), fl = (float)(thr - del);
  if ((double)fh < thr + del) fh = std::nextafter(fh, INFINITY);
  if ((double)fl > thr - del) fl = std::nextafter(fl, -INFINITY);
  const int screen = std::isfinite(thr) && thr - del > 0.0 && std::isfinite(fh) ? 1 : 0;
  if (prec == 0)
    tag_kernel<double><<<grid, 32 * kIndWarps, 0, s>>>(E, n1, D, bg, (const double*)q, plane, theta0, thf, dth, thr,
                                                       fh, fl, screen, tag);
  else
    tag_kernel<float><<<grid, 32 * kIndWarps, 0, s>>>(E, n1, D, bg, (const float*)q, plane, theta0, thf, dth, thr,
                                                      fh, fl, screen, tag);
  return cudaGetLastError();
}

// State layout conversion: element-major s[e][v][n] <-> the planes d[v][plane][...] of the
// mesh (to_planes = 1: element-major in, planes out; 0: the reverse).  W: the element's word.
template <class W>
__global__ void state_layout_kernel(int to_planes, int64_t E, int NP, int NV, const W* src, W* dst,
                                    int64_t plane) {
  const int64_t total = E * NV * NP;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int64_t en = i / NP;               // (e, v) of element-major index i
  const int n = (int)(i - en * NP);
  const int64_t e = en / NV;
  const int v = (int)(en - e * NV);
  const int64_t p = (int64_t)v * plane + e * NP + n;
  if (to_planes) dst[p] = src[i];
  else dst[i] = src[p];
}

cudaError_t launch_state_layout(int tsize, int to_planes, int64_t E, int NP, int NV, const void* src,
                                void* dst, int64_t plane, cudaStream_t s) {
  const int64_t total = E * NV * NP;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (tsize == 8)
    state_layout_kernel<uint64_t><<<grid, 256, 0, s>>>(to_planes, E, NP, NV, (const uint64_t*)src, (uint64_t*)dst, plane);
  else
    state_layout_kernel<uint32_t><<<grid, 256, 0, s>>>(to_planes, E, NP, NV, (const uint32_t*)src, (uint32_t*)dst, plane);
  return cudaGetLastError();
}

cudaError_t launch_primitives(int prec, int32_t E, int n1, int D, const double* bg, const void* q,
                              int64_t plane, double theta0, double* out, cudaStream_t s) {
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int64_t total = (int64_t)E * NP;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (prec == 0) primitives_kernel<double><<<grid, 256, 0, s>>>(E, n1, D, bg, (const double*)q, plane, theta0, out);
  else primitives_kernel<float><<<grid, 256, 0, s>>>(E, n1, D, bg, (const float*)q, plane, theta0, out);
  return cudaGetLastError();
}

size_t integrals_scratch_doubles() { return (size_t)kIntBlocks * 3 * 2; }

cudaError_t launch_integrals_combine(const double* S, const double* B, const int* bad, double* res, cudaStream_t s) {
  integrals_combine<<<1, 32, 0, s>>>(S, B, bad, res);
  return cudaGetLastError();
}

cudaError_t launch_integrals(int prec, bool background, int32_t E, int n1, int D, const int32_t* elem,
                             const double* xi, const double* w, const double* root_h,
                             const double* bg, const void* q, int64_t plane, const PhysC& ph,
                             double* partial, int* bad, double* out, cudaStream_t s) {
  if (n1 * n1 * n1 > kMaxNP || n1 > 9) return cudaErrorInvalidValue;
  const double r0 = root_h[0], r1 = root_h[1], r2 = root_h[2];
  if (background)
    integrals_partial<double, true><<<kIntBlocks, kIntThreads, 0, s>>>(E, n1, D, elem, xi, w, r0, r1, r2, bg,
        (const double*)nullptr, plane, ph, partial, bad);
  else if (prec == 0)
    integrals_partial<double, false><<<kIntBlocks, kIntThreads, 0, s>>>(E, n1, D, elem, xi, w, r0, r1, r2, bg,
        (const double*)q, plane, ph, partial, bad);
  else
    integrals_partial<float, false><<<kIntBlocks, kIntThreads, 0, s>>>(E, n1, D, elem, xi, w, r0, r1, r2, bg,
        (const float*)q, plane, ph, partial, bad);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  integrals_final<<<1, kIntThreads, 0, s>>>(kIntBlocks, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_transfer(int prec, int32_t Enew, int n1, int D, int nv, const int32_t* tmap,
                            const double* ops, const void* qold, int64_t plane_old, void* qnew,
                            int64_t plane_new, cudaStream_t s) {
  if (Enew == 0) return cudaSuccess;
  const int NP = D == 3 ? n1 * n1 * n1 : n1 * n1;
  const int threads = ((NP + 31) / 32) * 32;
  const size_t smem = (size_t)(4 * n1 * n1 + 3 * NP) * sizeof(double);
  if (prec == 0)
    transfer_kernel<double><<<Enew, threads, smem, s>>>(Enew, n1, D, tmap, ops, (const double*)qold,
                                                        plane_old, (double*)qnew, plane_new, nv);
  else
    transfer_kernel<float><<<Enew, threads, smem, s>>>(Enew, n1, D, tmap, ops, (const float*)qold,
                                                       plane_old, (float*)qnew, plane_new, nv);
  return cudaGetLastError();
}

// ---- halo exchange of a sharded mesh: the face traces (NV state planes and the P' plane) of
// listed element faces, packed into or unpacked from a contiguous buffer.  Slot i holds face
// (rows[3i + 1], rows[3i + 2]) of element rows[3i] as [NV + 1][face nodes], the face nodes in
// the order of the kernels' face_node (axis a at 0 or N, the other axes lowest first).
__device__ __forceinline__ int halo_face_node(int n1, int D, int a, int side, int t) {
  int idx[3] = {0, 0, 0};
  idx[a] = side ? n1 - 1 : 0;
  int r = t;
  for (int b = 0; b < D; ++b)
    if (b != a) { idx[b] = r % n1; r /= n1; }
  return idx[0] + n1 * (idx[1] + n1 * idx[2]);
}

template <class T>
__global__ void halo_kernel(int unpack, int64_t slots, int n1, int D, int NV, const int32_t* rows,
                            T* q, T* pp, int64_t plane, T* buf) {
  const int NF = D == 3 ? n1 * n1 : n1, NP = NF * n1;
  const int64_t per = (int64_t)(NV + 1) * NF;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= slots * per) return;
  const int64_t sl = i / per;
  const int r = (int)(i - sl * per);
  const int v = r / NF, t = r - v * NF;
  const int64_t e = rows[sl * 3];
  const int n = halo_face_node(n1, D, rows[sl * 3 + 1], rows[sl * 3 + 2], t);
  T* dst = v < NV ? q + (size_t)v * plane + (size_t)e * NP + n : (pp ? pp + (size_t)e * NP + n : nullptr);
  if (unpack) {
    if (dst) *dst = buf[i];
  } else {
    buf[i] = dst ? *dst : (T)0;
  }
}

cudaError_t launch_halo(int prec, int unpack, int64_t slots, int n1, int D, int NV, const int32_t* rows,
                        void* q, void* pp, int64_t plane, void* buf, cudaStream_t s) {
  const int NF = D == 3 ? n1 * n1 : n1;
  const int64_t total = slots * (NV + 1) * NF;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  if (prec == 0)
    halo_kernel<double><<<blocks, threads, 0, s>>>(unpack, slots, n1, D, NV, rows, (double*)q, (double*)pp,
                                                   plane, (double*)buf);
  else
    halo_kernel<float><<<blocks, threads, 0, s>>>(unpack, slots, n1, D, NV, rows, (float*)q, (float*)pp,
                                                  plane, (float*)buf);
  return cudaGetLastError();
}

}  // namespace dgk
