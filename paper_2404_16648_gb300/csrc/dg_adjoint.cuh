// Hand-written discrete adjoint (vector-Jacobian products) of the FP64 dGSEM right-hand side.
//
// For a state q and a cotangent Lambda of L(q) = dq/dt, vjp_kernel computes J(q)^T Lambda where
// J is the Jacobian of the discrete operator of dg_device.cuh: the transpose of the volume term
// (D^T along each axis, then the flux Jacobian transpose at each node), of the buoyancy source,
// and of every face term.  Faces are handled by gather, like the forward: at each of its face
// nodes an element forms the cotangent of the shared numerical flux F* from its own and its
// neighbour's Lambda, mu* = sign c (Lambda_own - Lambda_nbr), and applies the transpose of the
// Rusanov flux with respect to its own state.  Hanging faces go through mortar_vjp_kernel, the
// transpose of mortar_kernel: C^T for the coarse side's back-projection, the Rusanov transpose on
// the mortar nodes, and P^T back to the coarse trace.
//
// The non-smooth parts follow the derivative of the active branch: lambda = max(s-, s+) gives
// its gradient to the low side on ties, and |u| has derivative sign(u) with sign(0) = 0 (what a
// central finite difference sees).  The epilogue combines the product with other cotangents,
// out = a1 A1 + a2 A2 + b (B + dt J^T Lambda), which is all the reverse SSP-RK3 step needs.
#pragma once
#include "dg_device.cuh"

namespace dgk {

struct AdjArgs {
  const double* q;       // state [NV][plane]
  const double* pp;      // P' of q, one plane (as the forward stage kernels read it)
  const double* lam;     // cotangent of L [NV][plane]
  const double* a1;      // optional [NV][plane]
  const double* a2;      // optional
  const double* b;       // optional
  double* out;           // [NV][plane]
  const double* abuf;    // mortar adjoint contributions [G][1 + 2^(d-1)][NV][NF]
  int64_t plane;
  int32_t E;
  const int32_t* elem;
  const int32_t* conn;
  const double* bg;      // [E][N+1][4]
  const double* ops;     // D, P0, P1, C0, C1, w, x
  double inv2h[kMaxLevels][3];
  double lift[kMaxLevels][3];   // (2/h_a) / w0 per level and axis
  double c1, c2, cb, dt;
  PhysC ph;
};

struct MortarAdjArgs {
  const double* q;
  const double* pp;      // P' plane of q
  const double* lam;
  double* abuf;
  int64_t plane;
  int32_t G;
  const int32_t* groups;
  const int32_t* elem;
  const double* bg;
  const double* ops;
  double inv2h[kMaxLevels][3];
  PhysC ph;
};

// Everything about one node's state that the Jacobians need (the sound speed c is formed only
// where a face needs it, see sound_speed).  Reciprocals and square roots are the forward
// kernels' Newton forms (recip, sqrt_fast: within one ulp of the rounded results), which take
// fewer FP64 operations than IEEE division and square root.
template <int D>
struct NodeLin {
  double rinv, u[D], Theta, iTheta, P, dPdT;
};

// pp = P' of the node: read from the state's P' plane (the value the forward pass used), or
// pressure_pert of Theta' where no plane exists.
template <int D>
__device__ __forceinline__ NodeLin<D> node_lin(const double* q, double rb, double Tb, double pb,
                                               double pp, const PhysC& ph) {
  NodeLin<D> L;
  L.rinv = recip(rb + q[0]);
#pragma unroll
  for (int b = 0; b < D; ++b) L.u[b] = q[1 + b] * L.rinv;
  L.Theta = Tb + q[D + 1];
  L.iTheta = recip(L.Theta);
  L.P = pb + pp;
  L.dPdT = ph.gamma * L.P * L.iTheta;                // dP/dTheta of the EOS of Sec. 2.1
  return L;
}

template <int D>
__device__ __forceinline__ double sound_speed(const NodeLin<D>& L, double gamma) {
  return sqrt_fast(gamma * L.P * L.rinv);
}

// out += J_a(q)^T mu with J_a = dF_a/dq (perturbation variables).
template <int D>
__device__ __forceinline__ void flux_jac_t(const NodeLin<D>& L, int a, const double* mu, double* out) {
  double mu_u = 0.0;
#pragma unroll
  for (int b = 0; b < D; ++b) mu_u += mu[1 + b] * L.u[b];
  const double ua = L.u[a];
  out[0] += -ua * mu_u - mu[D + 1] * L.Theta * ua * L.rinv;
#pragma unroll
  for (int c = 0; c < D; ++c) out[1 + c] += mu[1 + c] * ua;
  out[1 + a] += mu[0] + mu_u + mu[D + 1] * L.Theta * L.rinv;
  out[D + 1] += mu[1 + a] * L.dPdT + mu[D + 1] * ua;
}

template <int D>
__device__ __forceinline__ double speed_of(const NodeLin<D>& L, double c, int a) {
  return fabs(L.u[a]) + c;
}

// out += w * grad_q (|u_a| + c), c = sqrt(gamma P / rho).
template <int D>
__device__ __forceinline__ void speed_grad(const NodeLin<D>& L, double c, int a, double gamma,
                                           double w, double* out) {
  const double ua = L.u[a];
  const double sg = ua > 0.0 ? 1.0 : (ua < 0.0 ? -1.0 : 0.0);
  out[0] += w * (-sg * ua * L.rinv - 0.5 * c * L.rinv);
  out[1 + a] += w * sg * L.rinv;
  out[D + 1] += w * (0.5 * gamma * c * L.iTheta);
}

// Transpose of F* = (F(qm) + F(qp))/2 - lambda/2 (qp - qm), lambda = max(sm, sp) (low side on
// ties), for cotangent mu: adds d F*/d qm ^T mu to om and d F*/d qp ^T mu to op (either may be
// null when that side is not wanted).
template <int D>
__device__ __forceinline__ void rusanov_vjp(const double* qm, const NodeLin<D>& Lm, const double* qp,
                                            const NodeLin<D>& Lp, int a, double gamma,
                                            const double* mu, double* om, double* op) {
  constexpr int NV = D + 2;
  const double cm = sound_speed<D>(Lm, gamma), cp = sound_speed<D>(Lp, gamma);
  const double sm = speed_of<D>(Lm, cm, a), sp = speed_of<D>(Lp, cp, a);
  const bool low = sm >= sp;
  const double lam = low ? sm : sp;
  double mud = 0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) mud += mu[v] * (qp[v] - qm[v]);
  double hm[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) hm[v] = 0.5 * mu[v];
  if (om) {
    flux_jac_t<D>(Lm, a, hm, om);
#pragma unroll
    for (int v = 0; v < NV; ++v) om[v] += 0.5 * lam * mu[v];
    if (low) speed_grad<D>(Lm, cm, a, gamma, -0.5 * mud, om);
  }
  if (op) {
    flux_jac_t<D>(Lp, a, hm, op);
#pragma unroll
    for (int v = 0; v < NV; ++v) op[v] -= 0.5 * lam * mu[v];
    if (!low) speed_grad<D>(Lp, cp, a, gamma, -0.5 * mud, op);
  }
}

// Rusanov transpose seen from one side only (the element's own node on a conforming face): the
// flux-Jacobian part 0.5 mu is returned as a cotangent `cot` (applied later through the node's
// J_a^T together with its other cotangents along axis a); acc gets the dissipation and
// wave-speed parts.  The neighbour enters through its state qo and wave speed so alone.
template <int D>
__device__ __forceinline__ void rusanov_vjp_own(const double* q, const NodeLin<D>& L, double c_own,
                                                const double* qo, double so, int a, bool own_low,
                                                double gamma, const double* mu, double* cot, double* acc) {
  constexpr int NV = D + 2;
  const double s_own = speed_of<D>(L, c_own, a);
  const double sm = own_low ? s_own : so, sp = own_low ? so : s_own;
  const bool low = sm >= sp;
  const double lam = low ? sm : sp;
  double mud = 0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) mud += own_low ? mu[v] * (qo[v] - q[v]) : mu[v] * (q[v] - qo[v]);
#pragma unroll
  for (int v = 0; v < NV; ++v) cot[v] += 0.5 * mu[v];
  if (own_low) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += 0.5 * lam * mu[v];
    if (low) speed_grad<D>(L, c_own, a, gamma, -0.5 * mud, acc);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] -= 0.5 * lam * mu[v];
    if (!low) speed_grad<D>(L, c_own, a, gamma, -0.5 * mud, acc);
  }
}

// |u_a| + c of a neighbour node (all the transpose needs from it).
template <int D>
__device__ __forceinline__ double neighbour_speed(const double* q, double rb, double pb, double pp, int a,
                                                  double gamma) {
  const double rinv = recip(rb + q[0]);
  return fabs(q[1 + a] * rinv) + sqrt_fast(gamma * (pb + pp) * rinv);
}

// Shared memory of vjp_kernel (doubles): D, then per element of the block Lambda [NV][NP], the
// node reciprocals 1/rho and 1/Theta [2][NP], and the face contributions: the cotangent each face
// node adds to its node's J_a^T input [2D][NV][NF] and the part it adds to the node's result
// [2D][NV][NF].
template <int D, int N, int EPB>
struct VjpSmem {
  static constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  static constexpr int oL = n1 * n1;
  static constexpr int oR = oL + EPB * NV * NP;
  static constexpr int oC = oR + EPB * 2 * NP;
  static constexpr int oA = oC + EPB * 2 * D * NV * NF;
  static constexpr int total = oA + EPB * 2 * D * NV * NF;
  static constexpr size_t bytes = sizeof(double) * (size_t)total;
};

// Phase 2 of vjp_kernel at tangential node t of face (AX, s) of element e: the cotangent the
// face adds to the node's J_AX^T input (the lift's own-flux part and the Rusanov flux part) and
// the part it adds to the node's result (dissipation, wave-speed gradient, mirror state or
// mortar contribution), to sC and sA at [2 AX + s][v][t].
template <int D, int N, int AX>
__device__ __forceinline__ void vjp_face(const AdjArgs& A, int64_t e, int level, int s, int t,
                                         const double* sL, const double* sR, double* sC, double* sA) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  constexpr int a = AX;
  const int f = 2 * a + s;
  const size_t ebase = (size_t)e * NP;
  const int nn = face_node<D, N>(a, s, t);
  const int32_t* c = A.conn + ((size_t)e * 2 * D + f) * 5;
  const int kind = c[0];
  const double coef = A.lift[level][a];
  const double sign = s ? -1.0 : 1.0;
  double lo[NV], cotf[NV], accf[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    lo[v] = sL[v * NP + nn];
    cotf[v] = -sign * coef * lo[v];        // own flux in the lift: L += sign coef (F* - F(q))
    accf[v] = 0.0;
  }
  if (kind == FACE_CONF || kind == FACE_WALL) {
    double qn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) qn[v] = A.q[(size_t)v * A.plane + ebase + nn];
    const int kz = (D == 3) ? nn / (n1 * n1) : nn / n1;
    const double* bz = A.bg + ((size_t)e * n1 + kz) * 4;
    const double zrb = bz[0], zpb = bz[2];
    const double zpp = A.pp[ebase + nn];
    // the node's linearisation from its stored reciprocals (node_lin's values bit for bit)
    NodeLin<D> Ln;
    Ln.rinv = sR[nn];
    Ln.iTheta = sR[NP + nn];
#pragma unroll
    for (int b = 0; b < D; ++b) Ln.u[b] = qn[1 + b] * Ln.rinv;
    Ln.Theta = bz[1] + qn[D + 1];
    Ln.P = zpb + zpp;
    Ln.dPdT = A.ph.gamma * Ln.P * Ln.iTheta;
    if (kind == FACE_CONF) {
      constexpr int stride_a = (a == 0) ? 1 : (a == 1 ? n1 : n1 * n1);
      const size_t no = (size_t)c[1] * NP + nn + (s ? -N : N) * stride_a;
      double qo[NV], mu[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qo[v] = A.q[(size_t)v * A.plane + no];
        mu[v] = sign * coef * (lo[v] - A.lam[(size_t)v * A.plane + no]);
      }
      const double c_own = sound_speed<D>(Ln, A.ph.gamma);
      const double so = neighbour_speed<D>(qo, zrb, zpb, A.pp[no], a, A.ph.gamma);
      rusanov_vjp_own<D>(qn, Ln, c_own, qo, so, a, s == 1, A.ph.gamma, mu, cotf, accf);
    } else {
      // mirror state: momentum along a negated, so its linearisation differs from the node's
      // only in u_a (an exact negation)
      double gq[NV], mu[NV], gacc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) { gq[v] = qn[v]; mu[v] = sign * coef * lo[v]; gacc[v] = 0.0; }
      gq[1 + a] = -qn[1 + a];
      NodeLin<D> Lg = Ln;
      Lg.u[a] = -Ln.u[a];
      if (s) rusanov_vjp<D>(qn, Ln, gq, Lg, a, A.ph.gamma, mu, accf, gacc);
      else   rusanov_vjp<D>(gq, Lg, qn, Ln, a, A.ph.gamma, mu, gacc, accf);
      gacc[1 + a] = -gacc[1 + a];                        // mirror map is its own transpose
#pragma unroll
      for (int v = 0; v < NV; ++v) accf[v] += gacc[v];
    }
  } else {
    const int64_t g = (kind == FACE_FINE) ? c[2] : c[1];
    const int slot = (kind == FACE_FINE) ? 1 + c[3] : 0;
    const double* src = A.abuf + (((size_t)g * (1 + NSUB) + slot) * NV) * NF + t;
#pragma unroll
    for (int v = 0; v < NV; ++v) accf[v] = src[(size_t)v * NF];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    sC[(f * NV + v) * NF + t] = cotf[v];
    sA[(f * NV + v) * NF + t] = accf[v];
  }
}

// J(q)^T Lambda for EPB elements per block, in three phases.  (1) One thread per node: Lambda
// and the node's reciprocals to shared memory.  (2) One thread per face node (the element's
// 2D (N+1)^(D-1) face nodes spread over its threads): the face's contributions at that node,
// from its own and its neighbour's state and Lambda; then one thread per node again: the
// volume cotangents -(2/h_a) D_a^T Lambda.  (3) One thread per node: the contributions of the
// faces the node lies on, the flux-Jacobian transposes and the epilogue.  The face work of
// phase 2 runs with every lane of a warp on a face node; done by the node's own thread, only
// the lanes of face nodes would do it while the FP64 pipe is held for the whole warp.
template <int D, int N, int EPB>
__global__ void __launch_bounds__(EPB * ipow(N + 1, D))
vjp_kernel(const AdjArgs A) {
  using S = VjpSmem<D, N, EPB>;
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  extern __shared__ __align__(16) double vjp_smem[];
  double* sD = vjp_smem;
  const int tid = threadIdx.x;
  for (int i = tid; i < n1 * n1; i += blockDim.x) sD[i] = A.ops[i];
  const int le = tid / NP, n = tid - le * NP;
  double* sL = vjp_smem + S::oL + le * NV * NP;
  double* sR = vjp_smem + S::oR + le * 2 * NP;
  double* sC = vjp_smem + S::oC + le * 2 * D * NV * NF;
  double* sA = vjp_smem + S::oA + le * 2 * D * NV * NF;
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  const bool valid = e < A.E;
  int idx[3];
  idx[0] = n % n1;
  idx[1] = (n / n1) % n1;
  idx[2] = (D == 3) ? n / (n1 * n1) : 0;
  const size_t ebase = (size_t)(valid ? e : 0) * NP;
  const size_t base = ebase + n;
  double q[NV], lam[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    q[v] = valid ? A.q[(size_t)v * A.plane + base] : 0.0;
    lam[v] = valid ? A.lam[(size_t)v * A.plane + base] : 0.0;
    sL[v * NP + n] = lam[v];
  }
  const int level = valid ? A.elem[e * 4] : 0;
  const double* bgp = A.bg + ((size_t)(valid ? e : 0) * n1 + idx[D - 1]) * 4;
  const double rb = valid ? bgp[0] : 1.0, Tb = valid ? bgp[1] : 1.0;
  const double pb = valid ? bgp[2] : 1.0;
  const double ppn = valid ? A.pp[base] : 0.0;
  const NodeLin<D> L = node_lin<D>(q, rb, Tb, pb, ppn, A.ph);
  sR[n] = L.rinv;
  sR[NP + n] = L.iTheta;
  __syncthreads();
  // ---- phase 2: face contributions, one face node per thread
  if (valid) {
    for (int fi = n; fi < 2 * D * NF; fi += NP) {
      const int f = fi / NF, t = fi - f * NF;
      // the axis as a template argument keeps every per-axis index of the face arithmetic
      // constant, so its arrays stay in registers
      if (f < 2) vjp_face<D, N, 0>(A, e, level, f & 1, t, sL, sR, sC, sA);
      else if (D == 2 || f < 4) vjp_face<D, N, 1>(A, e, level, f & 1, t, sL, sR, sC, sA);
      else vjp_face<D, N, (D == 3 ? 2 : 1)>(A, e, level, f & 1, t, sL, sR, sC, sA);
    }
  }
  // ---- volume cotangents: every own-node term along axis a goes through J_a(q)^T, so the
  // volume cotangent mu_a = -(2/h_a) D_a^T Lambda, the face lift's own-flux part and the
  // Rusanov flux part are summed in cot[a] and transposed once per axis
  double acc[NV], cot[D][NV];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int stride = ipow(n1, a);
    const int ia = idx[a];
    const int b0 = n - ia * stride;
    const double s2h = A.inv2h[level][a];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < n1; ++i) s += sD[i * n1 + ia] * sL[v * NP + b0 + i * stride];
      cot[a][v] = -s2h * s;
    }
  }
  // buoyancy source -rho' g on the vertical momentum
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  acc[0] = -A.ph.g * lam[D];
  __syncthreads();
  if (!valid) return;
  // ---- phase 3: the contributions of the faces this node lies on
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (idx[a] != 0 && idx[a] != N) continue;
    const int f = 2 * a + (idx[a] == N ? 1 : 0);
    int t = 0, mul = 1;
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b != a) { t += idx[b] * mul; mul *= n1; }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cot[a][v] += sC[(f * NV + v) * NF + t];
      acc[v] += sA[(f * NV + v) * NF + t];
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) flux_jac_t<D>(L, a, cot[a], acc);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const size_t k = (size_t)v * A.plane + base;
    double r = A.cb * ((A.b ? A.b[k] : 0.0) + A.dt * acc[v]);
    if (A.a1) r += A.c1 * A.a1[k];
    if (A.a2) r += A.c2 * A.a2[k];
    A.out[k] = r;
  }
}

// Transpose of mortar_kernel for one mortar group.  Thread (m, t) owns mortar node t of mortar
// m.  Writes, per fine element, d/d q_fine of the mortar flux terms at its face nodes (slot 1+m)
// and, for the coarse element, d/d q_coarse through the projection (slot 0).
template <int D, int N>
__global__ void __launch_bounds__((1 << (D - 1)) * ipow(N + 1, D - 1))
mortar_vjp_kernel(const MortarAdjArgs A) {
  constexpr int n1 = N + 1, NP = ipow(n1, D), NF = ipow(n1, D - 1), NV = D + 2;
  constexpr int NSUB = 1 << (D - 1);
  __shared__ double sP[2][n1 * n1], sC[2][n1 * n1];
  __shared__ double sQc[NV][NF], sMc[NV][NF];
  __shared__ double sT[NSUB][NV][NF];
  __shared__ double sX[NSUB][NV][NF];
  const int tid = threadIdx.x;
  for (int i = tid; i < n1 * n1; i += blockDim.x) {
    sP[0][i] = A.ops[1 * n1 * n1 + i];
    sP[1][i] = A.ops[2 * n1 * n1 + i];
    sC[0][i] = A.ops[3 * n1 * n1 + i];
    sC[1][i] = A.ops[4 * n1 * n1 + i];
  }
  const double w0 = A.ops[5 * n1 * n1];
  const int g = blockIdx.x;
  const int32_t* row = A.groups + (size_t)g * 7;
  const int64_t ec = row[0];
  const int a = row[1], side = row[2];
  const int m = tid / NF, t = tid - m * NF;
  const int b0 = m & 1, b1 = (m >> 1) & 1;
  const int t0 = t % n1, t1 = t / n1;
  const int64_t ef = row[3 + m];
  const double cc = A.inv2h[A.elem[ec * 4]][a] / w0;        // coarse lift coefficient
  const double cf = A.inv2h[A.elem[ef * 4]][a] / w0;        // fine lift coefficient
  const double sign_c = side ? -1.0 : 1.0;                  // coarse outward normal
  const double sign_f = -sign_c;                            // fine outward normal
  for (int i = tid; i < NV * NF; i += blockDim.x) {
    const int v = i / NF, tt = i - v * NF;
    const size_t k = (size_t)v * A.plane + (size_t)ec * NP + face_node<D, N>(a, side, tt);
    sQc[v][tt] = A.q[k];
    sMc[v][tt] = sign_c * cc * A.lam[k];                    // cotangent of F~ at coarse nodes
  }
  __syncthreads();
  // projected coarse state on mortar m (forward), first and second tangential passes
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += sP[b0][t0 * n1 + j] * sQc[v][j + n1 * t1];
    sT[m][v][t] = s;
  }
  __syncthreads();
  double qc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (D == 3) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < n1; ++j) s += sP[b1][t1 * n1 + j] * sT[m][v][t0 + n1 * j];
      qc[v] = s;
    } else {
      qc[v] = sT[m][v][t];
    }
  }
  __syncthreads();
  // C^T of the back-projection: mu*_m = (C_b1 x C_b0)^T mu~ (first pass along t1 in 3D)
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (D == 3) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < n1; ++j) s += sC[b1][j * n1 + t1] * sMc[v][t0 + n1 * j];
      sT[m][v][t] = s;
    } else {
      sT[m][v][t] = sMc[v][t];
    }
  }
  __syncthreads();
  const int nf = face_node<D, N>(a, 1 - side, t);
  double qf[NV], mu[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += sC[b0][j * n1 + t0] * sT[m][v][j + n1 * t1];
    const size_t k = (size_t)v * A.plane + (size_t)ef * NP + nf;
    qf[v] = A.q[k];
    mu[v] = s + sign_f * cf * A.lam[k];                     // plus the fine lift's cotangent
  }
  const int kf = (D == 3) ? nf / (n1 * n1) : nf / n1;
  const double* bd = A.bg + ((size_t)ef * n1 + kf) * 4;
  const NodeLin<D> Lf = node_lin<D>(qf, bd[0], bd[1], bd[2], A.pp[(size_t)ef * NP + nf], A.ph);
  const NodeLin<D> Lc = node_lin<D>(qc, bd[0], bd[1], bd[2], pressure_pert<kSeries>(qc[D + 1], bd[3], bd[2], A.ph),
                                    A.ph);
  double gf[NV], gc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { gf[v] = 0.0; gc[v] = 0.0; }
  if (side) rusanov_vjp<D>(qc, Lc, qf, Lf, a, A.ph.gamma, mu, gc, gf);
  else      rusanov_vjp<D>(qf, Lf, qc, Lc, a, A.ph.gamma, mu, gf, gc);
  double* ab = A.abuf + ((size_t)g * (1 + NSUB) * NV) * NF;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ab[((size_t)(1 + m) * NV + v) * NF + t] = gf[v];
    sX[m][v][t] = gc[v];
  }
  __syncthreads();
  // P^T back to the coarse trace: first along t0 ...
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += sP[b0][j * n1 + t0] * sX[m][v][j + n1 * t1];
    sT[m][v][t] = s;
  }
  __syncthreads();
  // ... then along t1, summed over the mortars
  if (m == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double acc = 0.0;
      for (int mm = 0; mm < NSUB; ++mm) {
        if (D == 3) {
          const int c1 = (mm >> 1) & 1;
          double s = 0.0;
#pragma unroll
          for (int j = 0; j < n1; ++j) s += sP[c1][j * n1 + t1] * sT[mm][v][t0 + n1 * j];
          acc += s;
        } else {
          acc += sT[mm][v][t];
        }
      }
      ab[(size_t)v * NF + t] = acc;
    }
  }
}

}  // namespace dgk
