// C ABI of the GB300 dGSEM library (declared in include/dg.h).
//
// A dg_mesh owns: the host forest (tree.hpp), the 1D operators (basis.hpp), and device buffers
// for three state copies (q^n and two RK stage states), the per-element integer tables, the
// FP64 background, the mortar flux buffer, and the integral reduction scratch.  Regrids
// rebuild the tables and transfer q^n; the stage states are reallocated with it.
#include <atomic>
#include <initializer_list>
#include <utility>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "basis.hpp"
#include "dg_launch.hpp"
#include "host_pool.hpp"
#include "tree.hpp"

#include "dg_mesh.hpp"

namespace {

dg_status fail(dg_mesh* m, dg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (m) m->err = buf;
  return st;
}

// Returned by every call on a mesh whose regrid failed after it had committed the new tree.
constexpr const char* kBrokenMsg =
    "the mesh is unusable: a regrid failed after committing its new tree; destroy the mesh";

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(m, e_ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,     \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                   \
  } while (0)

void dfree(void* p) { if (p) cudaFree(p); }

// Grow-only device buffer: reallocates, with a quarter of headroom, only when `bytes` exceeds
// the capacity (the old contents are not kept).
template <class P>
cudaError_t reserve(P*& p, size_t& cap, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (p && cap >= bytes) return cudaSuccess;
  dfree(p);
  p = nullptr;
  cap = 0;
  const size_t want = bytes + bytes / 4;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, want);
  if (e != cudaSuccess) return e;
  p = (P*)v;
  cap = want;
  return cudaSuccess;
}

// Grow-only pinned host buffer `slot` of the mesh; the caller's stream work that reads the old
// buffer must be complete before it is replaced (the mesh stream is synchronised first).
cudaError_t pin_reserve(dg_mesh* m, int slot, size_t bytes) {
  if (m->h_pin[slot] && m->c_pin[slot] >= bytes) return cudaSuccess;
  if (m->h_pin[slot]) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return e;
    cudaFreeHost(m->h_pin[slot]);
  }
  m->h_pin[slot] = nullptr;
  m->c_pin[slot] = 0;
  const size_t want = bytes + bytes / 4 + 256;
  void* p = nullptr;
  cudaError_t e = cudaMallocHost(&p, want);
  if (e != cudaSuccess) return e;
  m->h_pin[slot] = (unsigned char*)p;
  m->c_pin[slot] = want;
  return cudaSuccess;
}

// Host arrays to device buffers through pinned staging buffer `slot`, asynchronously on the mesh
// stream; the staging buffer stays untouched until the mesh stream is next synchronised.
cudaError_t upload_pinned(dg_mesh* m, int slot, std::initializer_list<std::pair<void*, std::pair<const void*, size_t>>> items) {
  size_t total = 0;
  for (const auto& it : items) total += (it.second.second + 255) / 256 * 256;
  cudaError_t e = pin_reserve(m, slot, total);
  if (e != cudaSuccess) return e;
  size_t off = 0;
  for (const auto& it : items) {
    const size_t bytes = it.second.second;
    if (bytes == 0) continue;
    std::memcpy(m->h_pin[slot] + off, it.second.first, bytes);
    e = cudaMemcpyAsync(it.first, m->h_pin[slot] + off, bytes, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return e;
    off += (bytes + 255) / 256 * 256;
  }
  return cudaSuccess;
}

}  // namespace

namespace dgi {
int64_t plane(const dg_mesh* m) { return m->E * m->NP; }
}  // namespace dgi
using dgi::plane;

namespace {

dg_status upload_ops(dg_mesh* m) {
  const int nn = m->n1 * m->n1;
  std::vector<double> od;
  od.insert(od.end(), m->basis.D.begin(), m->basis.D.end());
  od.insert(od.end(), m->basis.P[0].begin(), m->basis.P[0].end());
  od.insert(od.end(), m->basis.P[1].begin(), m->basis.P[1].end());
  od.insert(od.end(), m->basis.C[0].begin(), m->basis.C[0].end());
  od.insert(od.end(), m->basis.C[1].begin(), m->basis.C[1].end());
  od.insert(od.end(), m->basis.w.begin(), m->basis.w.end());
  od.insert(od.end(), m->basis.x.begin(), m->basis.x.end());
  od.insert(od.end(), m->basis.G[0].begin(), m->basis.G[0].end());
  od.insert(od.end(), m->basis.G[1].begin(), m->basis.G[1].end());
  (void)nn;
  CU(cudaMalloc(&m->d_opsd, od.size() * sizeof(double)));
  CU(cudaMemcpy(m->d_opsd, od.data(), od.size() * sizeof(double), cudaMemcpyHostToDevice));
  CU(cudaMalloc(&m->d_ops, od.size() * m->tsize));
  if (m->prec == DG_FP64) {
    CU(cudaMemcpy(m->d_ops, od.data(), od.size() * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> of(od.begin(), od.end());
    CU(cudaMemcpy(m->d_ops, of.data(), of.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return DG_OK;
}

const double* d_w(const dg_mesh* m) { return m->d_opsd + 5 * m->n1 * m->n1; }
const double* d_x(const dg_mesh* m) { return m->d_opsd + 5 * m->n1 * m->n1 + m->n1; }

// Host tables of a forest, built and checked before anything of the mesh changes.
struct HostTables {
  int64_t E = 0, G = 0;
  std::vector<int32_t> conf, mort, bnd, conn, elem;
};

// Builds the face lists, the connectivity and the element table of forest f and checks every
// index a kernel will follow; the mesh is only read (its sizes and error string).
dg_status build_tables(dg_mesh* m, const dgl::Forest& f, HostTables* t) {
  t->E = f.size();
  if ((int64_t)(m->NV + 1) * t->E * m->NP >= ((int64_t)1 << 31))
    return fail(m, DG_ERR_UNSUPPORTED, "mesh too large for 32-bit state offsets (%lld elements)",
                (long long)t->E);
  f.face_lists(&t->conf, &t->mort, &t->bnd);
  t->G = (int64_t)(t->mort.size() / 7);
  f.connectivity(t->mort, &t->conn);
  const int nf = 2 * m->D;
  const int64_t E = t->E, G = t->G;
  // face-flux slots of stage layout 5 in the third field of the conforming and wall rows:
  // conforming faces 0 .. C-1 (list order), boundary faces C .. C+B-1
  const int64_t C = (int64_t)t->conf.size() / 3, Bn = (int64_t)t->bnd.size() / 3;
  for (int64_t c = 0; c < C; ++c) {
    const int32_t* r = t->conf.data() + c * 3;
    if (r[0] < 0 || r[0] >= E || r[1] < 0 || r[1] >= E || r[2] < 0 || r[2] >= m->D)
      return fail(m, DG_ERR_STATE, "inconsistent conforming face %lld", (long long)c);
    t->conn[((size_t)r[0] * nf + 2 * r[2] + 1) * 5 + 2] = (int32_t)c;
    t->conn[((size_t)r[1] * nf + 2 * r[2]) * 5 + 2] = (int32_t)c;
  }
  for (int64_t b = 0; b < Bn; ++b) {
    const int32_t* r = t->bnd.data() + b * 3;
    if (r[0] < 0 || r[0] >= E || r[1] < 0 || r[1] >= m->D || r[2] < 0 || r[2] > 1)
      return fail(m, DG_ERR_STATE, "inconsistent boundary face %lld", (long long)b);
    t->conn[((size_t)r[0] * nf + 2 * r[1] + r[2]) * 5 + 2] = (int32_t)(C + b);
  }
  // every index a kernel will follow must be in range before anything is uploaded; the error
  // names the first bad row
  const int NSUB = m->NSUB, D = m->D;
  const std::vector<int32_t>& conn = t->conn;
  const std::vector<int32_t>& mort = t->mort;
  std::atomic<int64_t> bad_face{INT64_MAX}, bad_group{INT64_MAX};
  auto note = [](std::atomic<int64_t>& first, int64_t r) {
    int64_t cur = first.load(std::memory_order_relaxed);
    while (r < cur && !first.compare_exchange_weak(cur, r, std::memory_order_relaxed)) {}
  };
  dgl::parallel_ranges(E * nf, 8192, [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      const int32_t* c = conn.data() + r * 5;
      bool ok = true;
      switch (c[0]) {
        case dgl::FACE_WALL: ok = c[2] >= C && c[2] < C + Bn; break;
        case dgl::FACE_CONF: ok = c[1] >= 0 && c[1] < E && c[2] >= 0 && c[2] < C; break;
        case dgl::FACE_FINE: ok = c[1] >= 0 && c[1] < E && c[2] >= 0 && c[2] < G && c[3] >= 0 && c[3] < NSUB; break;
        case dgl::FACE_COARSE: ok = c[1] >= 0 && c[1] < G; break;
        default: ok = false;
      }
      if (!ok) { note(bad_face, r); return; }
    }
  });
  if (bad_face.load() != INT64_MAX) {
    const int64_t r = bad_face.load();
    return fail(m, DG_ERR_STATE, "inconsistent connectivity at element %lld face %d", (long long)(r / nf), (int)(r % nf));
  }
  dgl::parallel_ranges(G, 4096, [&](int64_t g0, int64_t g1) {
    for (int64_t g = g0; g < g1; ++g)
      for (int k = 0; k < 3 + NSUB; ++k) {
        const int32_t v = mort[g * 7 + k];
        const bool ok = k == 0 || k >= 3 ? (v >= 0 && v < E) : (v >= 0 && v < (k == 1 ? D : 2));
        if (!ok) { note(bad_group, g); return; }
      }
  });
  if (bad_group.load() != INT64_MAX)
    return fail(m, DG_ERR_STATE, "inconsistent mortar group %lld", (long long)bad_group.load());
  t->elem.assign((size_t)E * 4, 0);
  const auto& L = f.leaves();
  for (int64_t e = 0; e < E; ++e) {
    t->elem[e * 4] = L[e].level;
    for (int a = 0; a < 3; ++a) t->elem[e * 4 + 1 + a] = L[e].c[a];
  }
  return DG_OK;
}

// Makes checked tables the mesh's own: sizes, host lists, device tables, background.
dg_status upload_tables(dg_mesh* m, HostTables&& t) {
  m->E = t.E;
  m->G = t.G;
  m->e_begin = 0;
  m->e_end = t.E;
  m->conf = std::move(t.conf);
  m->mort = std::move(t.mort);
  m->bnd = std::move(t.bnd);
  const std::vector<int32_t>& conn = t.conn;
  const std::vector<int32_t>& elem = t.elem;
  CU(reserve(m->d_elem, m->c_elem, elem.size() * sizeof(int32_t)));
  CU(reserve(m->d_conn, m->c_conn, conn.size() * sizeof(int32_t)));
  if (m->G > 0) {
    CU(reserve(m->d_groups, m->c_groups, m->mort.size() * sizeof(int32_t)));
    CU(reserve(m->d_mbuf, m->c_mbuf, (size_t)m->G * (1 + m->NSUB) * m->NV * m->NF * m->tsize));
  }
  CU(reserve(m->d_fconf, m->c_fconf, m->conf.size() * sizeof(int32_t)));
  CU(reserve(m->d_fbnd, m->c_fbnd, m->bnd.size() * sizeof(int32_t)));
  CU(upload_pinned(m, 1, {{m->d_elem, {elem.data(), elem.size() * sizeof(int32_t)}},
                          {m->d_conn, {conn.data(), conn.size() * sizeof(int32_t)}},
                          {m->d_groups, {m->mort.data(), m->G > 0 ? m->mort.size() * sizeof(int32_t) : 0}},
                          {m->d_fconf, {m->conf.data(), m->conf.size() * sizeof(int32_t)}},
                          {m->d_fbnd, {m->bnd.data(), m->bnd.size() * sizeof(int32_t)}}}));
  CU(reserve(m->d_bg, m->c_bg, (size_t)m->E * m->n1 * 4 * sizeof(double)));
  if (m->prec == DG_FP32_PERT) {
    CU(reserve(m->d_bgf, m->c_bgf, (size_t)m->E * m->n1 * 4 * sizeof(float)));
    CU(reserve(m->d_bgc, m->c_bgc, (size_t)m->E * m->n1 * sizeof(double)));
  }
  CU(reserve(m->d_ppscratch, m->c_pps, (size_t)(m->E > 0 ? plane(m) : 1) * m->tsize));
  if (m->desc.nu > 0.0) {
    const size_t pl = (size_t)(plane(m) > 0 ? plane(m) : 1);
    CU(reserve(m->d_sigma, m->c_sigma, (size_t)(m->D + 1) * m->D * pl * sizeof(double)));
    CU(reserve(m->d_V, m->c_V, (size_t)(m->D + 1) * pl * sizeof(double)));
    if (m->G > 0) CU(reserve(m->d_vbuf, m->c_vbuf, (size_t)m->G * (1 + m->NSUB) * (m->D + 1) * m->NF * sizeof(double)));
  }
  CU(dgk::launch_background((int32_t)m->E, m->n1, m->D, m->d_elem, d_x(m), m->root_h[m->D - 1],
                            m->ph, m->d_bg, m->d_bgf, m->d_bgc, m->stream));
  m->pp_valid = false;
  m->bgint_valid = false;
  return DG_OK;
}

// (Re)builds the device tables for the current forest (mesh creation).
dg_status rebuild_topology(dg_mesh* m) {
  HostTables t;
  dg_status st = build_tables(m, m->forest, &t);
  if (st != DG_OK) return st;
  return upload_tables(m, std::move(t));
}

// Each state buffer holds the NV variable planes followed by the P' plane of that state.
size_t state_bytes(const dg_mesh* m) { return (size_t)(m->NV + 1) * plane(m) * m->tsize; }

dg_status alloc_states(dg_mesh* m) {
  for (int i = 0; i < 3; ++i) CU(reserve(m->q[i], m->q_cap[i], state_bytes(m)));
  return DG_OK;
}

const void* bgt(const dg_mesh* m) {
  return m->prec == DG_FP64 ? (const void*)m->d_bg : (const void*)m->d_bgf;
}

}  // namespace

namespace dgi {

void* pp_plane(const dg_mesh* m, void* q) {
  return (char*)q + (size_t)m->NV * plane(m) * m->tsize;
}

void fill_stage_args(const dg_mesh* m, const void* qs, const void* pp_in, const void* qn, void* out,
                     void* pp_out, int mode, double dt, double ca, double cb, dgk::StageArgs* A) {
  A->qs = qs; A->pp_in = pp_in; A->qn = qn; A->out = out; A->pp_out = pp_out; A->mbuf = m->d_mbuf;
  A->plane = plane(m); A->E = (int32_t)m->e_end; A->e_begin = (int32_t)m->e_begin;
  A->fbuf = m->d_fbuf;
  A->elem = m->d_elem; A->conn = m->d_conn; A->bg = m->d_bg; A->bgt = bgt(m); A->bgc = m->d_bgc; A->ops = m->d_ops;
  for (int l = 0; l < dgk::kMaxLevels; ++l)
    for (int a = 0; a < 3; ++a) {
      // 2/h = (2/h_root) 2^level: power-of-two scaling is exact
      A->inv2hd[l][a] = std::ldexp(2.0 / m->root_h[a], l);
      A->inv2hf[l][a] = (float)A->inv2hd[l][a];
      // the same quotient the kernels formed per face: T(2/h) / T(w0), one IEEE division
      A->liftd[l][a] = A->inv2hd[l][a] / m->basis.w[0];
      A->liftf[l][a] = A->inv2hf[l][a] / (float)m->basis.w[0];
    }
  A->rw0d = 1.0 / m->basis.w[0];
  A->rw0f = (float)A->rw0d;
  A->dt = dt; A->ca = ca; A->cb = cb; A->mode = mode; A->variant = m->variant; A->ph = m->ph;
  A->dtf = (float)dt; A->caf = (float)ca; A->cbf = (float)cb; A->first = ca == 0.0 ? 1 : 0;
  A->plane32 = (int32_t)plane(m);
  A->gammaf = (float)m->ph.gamma; A->gf = (float)m->ph.g;
}

dg_status set_error(dg_mesh* m, dg_status st, const char* msg) {
  if (m) m->err = msg;
  return st;
}

void fill_face_args(const dg_mesh* m, const void* qs, const void* pp_in, dgk::FaceArgs* F) {
  const int64_t C = (int64_t)m->conf.size() / 3, Bn = (int64_t)m->bnd.size() / 3;
  *F = dgk::FaceArgs{qs, pp_in, m->d_fbuf, plane(m), (int32_t)C, (int32_t)Bn, m->d_fconf, m->d_fbnd, bgt(m),
                     (float)m->ph.gamma, m->ph};
}

dg_status ensure_face_buffer(dg_mesh* m) {
  const int64_t C = (int64_t)m->conf.size() / 3, Bn = (int64_t)m->bnd.size() / 3;
  CU(reserve(m->d_fbuf, m->c_fbuf, (size_t)(C + Bn > 0 ? C + Bn : 1) * m->NV * m->NF * m->tsize));
  return DG_OK;
}

void fill_mortar_args(const dg_mesh* m, const void* qs, const void* pp_in, dgk::MortarArgs* M) {
  const bool part = m->nparts > 1;
  *M = dgk::MortarArgs{qs, pp_in, m->d_mbuf, plane(m), (int32_t)(part ? m->G_part : m->G), m->d_groups,
                       m->d_bg, bgt(m), m->d_bgc, m->d_ops, (float)m->ph.gamma, m->ph,
                       part ? m->d_glist : nullptr};
}

dg_status launch_mortars(dg_mesh* m, const void* qs, const void* pp_in, cudaStream_t s) {
  if ((m->nparts > 1 ? m->G_part : m->G) == 0) return DG_OK;
  dgk::MortarArgs M;
  fill_mortar_args(m, qs, pp_in, &M);
  bool ok = m->prec == DG_FP64
                ? (m->D == 2 ? dgk::launch_mortar_f64_2d(m->N, M, s) : dgk::launch_mortar_f64_3d(m->N, M, s))
                : (m->D == 2 ? dgk::launch_mortar_f32_2d(m->N, M, s) : dgk::launch_mortar_f32_3d(m->N, M, s));
  if (!ok) return set_error(m, DG_ERR_UNSUPPORTED, "mortar kernel not compiled");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(m, DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

dg_status ensure_pp(dg_mesh* m, cudaStream_t s) {
  if (m->pp_valid || m->tracer) return DG_OK;           // a tracer state has no pressure
  const void* theta = (const char*)m->q[0] + (size_t)(m->NV - 1) * plane(m) * m->tsize;
  cudaError_t e = dgk::launch_pprime(m->prec, (int32_t)m->E, m->n1, m->D, theta, m->d_bg, m->d_bgc, m->ph,
                                     pp_plane(m, m->q[0]), s);
  if (e != cudaSuccess) return set_error(m, DG_ERR_CUDA, cudaGetErrorString(e));
  m->pp_valid = true;
  return DG_OK;
}

}  // namespace dgi
using dgi::pp_plane;

namespace {

// Tracer stage (or pure RHS) with the wind factor m->stage_g: hanging faces, then the stage.
dg_status tracer_pass(dg_mesh* m, const void* cs, const void* cn, void* out, int mode, double dt,
                      double ca, double cb, cudaStream_t s) {
  if (m->G > 0) {
    dgk::TracerMortarArgs M{};
    M.cs = (const double*)cs; M.mbuf = (double*)m->d_mbuf; M.plane = plane(m); M.G = (int32_t)m->G;
    M.groups = m->d_groups; M.elem = m->d_elem; M.ops = m->d_opsd;
    M.root_h[0] = m->root_h[0]; M.root_h[1] = m->root_h[1];
    M.g = m->stage_g; M.interp = m->desc.face_mode == DG_FACE_INTERP;
    if (!dgk::launch_tracer_mortar(m->N, M, s)) return fail(m, DG_ERR_UNSUPPORTED, "tracer N=%d not compiled", m->N);
    CU(cudaGetLastError());
  }
  dgk::TracerArgs A{};
  A.cs = (const double*)cs; A.cn = (const double*)cn; A.out = (double*)out; A.mbuf = (const double*)m->d_mbuf;
  A.plane = plane(m); A.E = (int32_t)m->E; A.elem = m->d_elem; A.conn = m->d_conn; A.ops = m->d_opsd;
  A.root_h[0] = m->root_h[0]; A.root_h[1] = m->root_h[1];
  for (int l = 0; l < dgk::kMaxLevels; ++l)
    for (int a = 0; a < 2; ++a) {
      A.inv2h[l][a] = std::ldexp(2.0 / m->root_h[a], l);
      A.lift[l][a] = A.inv2h[l][a] / m->basis.w[0];
    }
  A.g = m->stage_g; A.dt = dt; A.ca = ca; A.cb = cb; A.mode = mode;
  if (!dgk::launch_tracer_stage(m->N, A, s)) return fail(m, DG_ERR_UNSUPPORTED, "tracer N=%d not compiled", m->N);
  CU(cudaGetLastError());
  return DG_OK;
}

double wind_factor(const dg_mesh* m, double t) { return std::cos(M_PI * t / m->desc.wind_period); }

dg_status launch_rhs_pass(dg_mesh* m, const void* qs, const void* pp_in, const void* qn, void* out,
                          void* pp_out, int mode, double dt, double ca, double cb, cudaStream_t s) {
  if (m->tracer) return tracer_pass(m, qs, qn, out, mode, dt, ca, cb, s);
  const bool timed = m->timing && mode == 1;
  // layouts 4 and 2 directly after their mortar kernel: programmatic dependent launch, so the
  // stage kernel runs its elements without hanging faces while the mortar kernel finishes and
  // only the others wait for it.  A stage timed on its own (dg_enable_timing) needs an event
  // between the two launches, which rules this out.
  // layout 5 (face fluxes once per face, then the line-pass stage kernel) needs the whole mesh's
  // face lists; a partitioned mesh runs layout 2
  const int variant = (m->variant == 5 && m->nparts > 1) ? 2 : m->variant;
  const bool mortars = (m->nparts > 1 ? m->G_part : m->G) > 0;
  bool pdl = (variant == 4 || variant == 2) && mortars && !timed;
  dg_status st = dgi::launch_mortars(m, qs, pp_in, s);
  if (st != DG_OK) return st;
  // a timed stage spans the stage kernel and, in layout 5, the face kernel before it
  if (timed) {
    while (m->ev.size() < m->ev_used + 2) {
      cudaEvent_t e;
      CU(cudaEventCreate(&e));
      m->ev.push_back(e);
    }
    CU(cudaEventRecord(m->ev[m->ev_used], s));
  }
  if (variant == 5) {
    st = dgi::ensure_face_buffer(m);
    if (st != DG_OK) return st;
    dgk::FaceArgs F;
    dgi::fill_face_args(m, qs, pp_in, &F);
    const bool fpdl = mortars && !timed;   // the face kernel follows the mortar kernel directly
    CU(m->prec == DG_FP64
           ? (m->D == 2 ? dgk::launch_face_f64_2d(m->N, F, fpdl, s) : dgk::launch_face_f64_3d(m->N, F, fpdl, s))
           : (m->D == 2 ? dgk::launch_face_f32_2d(m->N, F, fpdl, s) : dgk::launch_face_f32_3d(m->N, F, fpdl, s)));
    pdl = !timed;                // the stage kernel follows the face kernel directly
  }
  dgk::StageArgs A{};
  dgi::fill_stage_args(m, qs, pp_in, qn, out, pp_out, mode, dt, ca, cb, &A);
  A.variant = variant;
  A.after_mortar = pdl ? 1 : 0;
  bool ok = m->prec == DG_FP64
                ? (m->D == 2 ? dgk::launch_stage_f64_2d(m->N, A, s) : dgk::launch_stage_f64_3d(m->N, A, s))
                : (m->D == 2 ? dgk::launch_stage_f32_2d(m->N, A, s) : dgk::launch_stage_f32_3d(m->N, A, s));
  if (!ok) return fail(m, DG_ERR_UNSUPPORTED, "stage kernel for N=%d not compiled", m->N);
  CU(cudaGetLastError());
  if (timed) {
    CU(cudaEventRecord(m->ev[m->ev_used + 1], s));
    m->ev_used += 2;
  }
  if (m->desc.nu > 0.0) {
    // BR1 viscous tendency of the stage input, added as cb dt V (the stage combination is linear
    // in the tendency); P' of the output is refreshed after the Theta' update
    dgk::ViscArgs V{};
    V.q = (const double*)qs; V.sigma = m->d_sigma; V.V = m->d_V; V.vbuf = m->d_vbuf;
    V.plane = plane(m); V.E = (int32_t)m->E; V.G = (int32_t)m->G; V.elem = m->d_elem;
    V.conn = m->d_conn; V.groups = m->d_groups; V.bg = m->d_bg; V.ops = m->d_opsd;
    for (int l = 0; l < dgk::kMaxLevels; ++l)
      for (int a = 0; a < 3; ++a) {
        V.inv2h[l][a] = std::ldexp(2.0 / m->root_h[a], l);
        V.lift[l][a] = V.inv2h[l][a] / m->basis.w[0];
      }
    V.nu = m->desc.nu; V.theta0 = m->ph.theta0;
    for (int pass = 1; pass <= 2; ++pass) {
      if (!dgk::launch_viscous_pass(m->D, m->N, V, pass, s))
        return fail(m, DG_ERR_UNSUPPORTED, "viscous kernels for N=%d not compiled", m->N);
      CU(cudaGetLastError());
    }
    CU(dgk::launch_visc_add((int32_t)m->E, m->n1, m->D, m->d_V, mode == 1 ? cb * dt : 1.0, (double*)out,
                            plane(m), m->d_bg, m->ph, mode == 1 ? (double*)pp_out : nullptr, s));
  }
  return DG_OK;
}

// Uploads the derivative matrices of every degree to the constant memory of each kernel unit,
// once per device.
dg_status init_device_tables(dg_mesh* m) {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(dev)) return DG_OK;
  std::vector<double> all;
  for (int N = 1; N <= DG_MAX_N; ++N) {
    dgl::Basis1D b = dgl::make_basis(N);
    all.insert(all.end(), b.D.begin(), b.D.end());
  }
  CU(dgk::init_stage_f64_2d(all.data()));
  CU(dgk::init_stage_f64_3d(all.data()));
  CU(dgk::init_stage_f32_2d(all.data()));
  CU(dgk::init_stage_f32_3d(all.data()));
  CU(dgk::init_stage_batch_w(all.data()));
  CU(dgk::init_stage_batch_d(all.data()));
  done.insert(dev);
  return DG_OK;
}

// Workspace of dg_step_state / dg_step_vjp for the current mesh size.
dg_status ensure_adjoint_ws(dg_mesh* m) {
  if (m->adj_E == m->E && m->adj_G == m->G) return DG_OK;
  for (int i = 0; i < 3; ++i) { dfree(m->adj_q[i]); m->adj_q[i] = nullptr; }
  for (int i = 0; i < 2; ++i) { dfree(m->adj_l[i]); m->adj_l[i] = nullptr; }
  dfree(m->d_abuf); m->d_abuf = nullptr;
  m->adj_E = m->adj_G = -1;
  const size_t pl = (size_t)(plane(m) > 0 ? plane(m) : 1);
  for (int i = 0; i < 3; ++i) CU(cudaMalloc(&m->adj_q[i], (m->NV + 1) * pl * m->tsize));
  for (int i = 0; i < 2; ++i) CU(cudaMalloc(&m->adj_l[i], m->NV * pl * sizeof(double)));
  if (m->G > 0) CU(cudaMalloc(&m->d_abuf, (size_t)m->G * (1 + m->NSUB) * m->NV * m->NF * sizeof(double)));
  m->adj_E = m->E;
  m->adj_G = m->G;
  return DG_OK;
}

// Copies a caller state (NV planes) into a workspace buffer and fills its P' plane.
dg_status stage_in(dg_mesh* m, const void* q, void* buf, cudaStream_t s) {
  const size_t bytes = (size_t)m->NV * plane(m) * m->tsize;
  CU(cudaMemcpyAsync(buf, q, bytes, cudaMemcpyDeviceToDevice, s));
  const void* theta = (const char*)buf + (size_t)(m->NV - 1) * plane(m) * m->tsize;
  CU(dgk::launch_pprime(m->prec, (int32_t)m->E, m->n1, m->D, theta, m->d_bg, m->d_bgc, m->ph, pp_plane(m, buf), s));
  return DG_OK;
}

// The three Shu-Osher stages of one step on workspace buffers: b0 -> b1 -> b2 -> b0.
dg_status rk3_on(dg_mesh* m, void* b0, void* b1, void* b2, double dt, cudaStream_t s) {
  dg_status st = launch_rhs_pass(m, b0, pp_plane(m, b0), b0, b1, pp_plane(m, b1), 1, dt, 0.0, 1.0, s);
  if (st == DG_OK) st = launch_rhs_pass(m, b1, pp_plane(m, b1), b0, b2, pp_plane(m, b2), 1, dt, 0.75, 0.25, s);
  if (st == DG_OK) st = launch_rhs_pass(m, b2, pp_plane(m, b2), b0, b0, pp_plane(m, b0), 1, dt, 1.0 / 3.0, 2.0 / 3.0, s);
  return st;
}

// out = c1 a1 + c2 a2 + cb (b + dt J(q)^T lam), with the mortar transposes first.
dg_status vjp_pass(dg_mesh* m, const double* q, const double* pp, const double* lam, const double* a1,
                   double c1, const double* a2, double c2, const double* b, double cb, double dt,
                   double* out, cudaStream_t s) {
  if (m->G > 0) {
    dgk::MortarAdjArgs M{};
    M.q = q; M.pp = pp; M.lam = lam; M.abuf = m->d_abuf; M.plane = plane(m); M.G = (int32_t)m->G;
    M.groups = m->d_groups; M.elem = m->d_elem; M.bg = m->d_bg; M.ops = m->d_opsd; M.ph = m->ph;
    for (int l = 0; l < dgk::kMaxLevels; ++l)
      for (int a = 0; a < 3; ++a) M.inv2h[l][a] = std::ldexp(2.0 / m->root_h[a], l);
    if (!dgk::launch_mortar_vjp(m->D, m->N, M, s)) return fail(m, DG_ERR_UNSUPPORTED, "mortar adjoint not compiled");
    CU(cudaGetLastError());
  }
  dgk::AdjArgs A{};
  A.q = q; A.pp = pp; A.lam = lam; A.a1 = a1; A.a2 = a2; A.b = b; A.out = out; A.abuf = m->d_abuf;
  A.plane = plane(m); A.E = (int32_t)m->E; A.elem = m->d_elem; A.conn = m->d_conn; A.bg = m->d_bg;
  A.ops = m->d_opsd; A.c1 = c1; A.c2 = c2; A.cb = cb; A.dt = dt; A.ph = m->ph;
  for (int l = 0; l < dgk::kMaxLevels; ++l)
    for (int a = 0; a < 3; ++a) {
      A.inv2h[l][a] = std::ldexp(2.0 / m->root_h[a], l);
      A.lift[l][a] = A.inv2h[l][a] / m->basis.w[0];
    }
  cudaError_t cfg = cudaSuccess;
  if (!dgk::launch_vjp(m->D, m->N, A, s, cfg)) return fail(m, DG_ERR_UNSUPPORTED, "adjoint kernel not compiled");
  CU(cfg);
  CU(cudaGetLastError());
  return DG_OK;
}

}  // namespace

namespace {

// The owned range, the halo slot lists and the part's mortar groups of an SFC partition of the
// mesh's (replicated) tree into nparts parts (Sec. 3.1 names SFC partitioning).  Every part
// derives the same lists from the same tree: part p sends, per destination part q, the traces
// of its halo rows toward q in row order; q receives them in that order, as the faces of the
// remote elements its own elements read.
dg_status apply_partition(dg_mesh* m) {
  const int P = m->nparts;
  m->send_off.assign(P + 1, 0);
  m->recv_off.assign(P + 1, 0);
  if (P <= 1) {
    m->e_begin = 0;
    m->e_end = m->E;
    m->G_part = m->G;
    return DG_OK;
  }
  std::vector<int64_t> starts;
  m->forest.partition(P, &starts);
  m->e_begin = starts[m->part];
  m->e_end = starts[m->part + 1];
  std::vector<int32_t> rows;
  m->forest.halo(starts, m->part, &rows);
  std::vector<std::vector<int32_t>> to(P);
  for (size_t r = 0; r < rows.size(); r += 5) {
    auto& v = to[rows[r + 4]];
    v.push_back(rows[r]); v.push_back(rows[r + 1]); v.push_back(rows[r + 2]);
  }
  std::vector<int32_t> send, recv;
  for (int q = 0; q < P; ++q) {
    m->send_off[q] = (int64_t)send.size() / 3;
    send.insert(send.end(), to[q].begin(), to[q].end());
  }
  m->send_off[P] = (int64_t)send.size() / 3;
  for (int q = 0; q < P; ++q) {
    m->recv_off[q] = (int64_t)recv.size() / 3;
    if (q == m->part) continue;
    std::vector<int32_t> rq;
    m->forest.halo(starts, q, &rq);
    for (size_t r = 0; r < rq.size(); r += 5)
      if (rq[r + 4] == m->part) { recv.push_back(rq[r]); recv.push_back(rq[r + 1]); recv.push_back(rq[r + 2]); }
  }
  m->recv_off[P] = (int64_t)recv.size() / 3;
  std::vector<int32_t> glist;
  const int nsub = m->NSUB;
  for (int64_t g = 0; g < m->G; ++g) {
    const int32_t* r = m->mort.data() + g * 7;
    bool mine = r[0] >= m->e_begin && r[0] < m->e_end;
    for (int k = 0; k < nsub && !mine; ++k) mine = r[3 + k] >= m->e_begin && r[3 + k] < m->e_end;
    if (mine) glist.push_back((int32_t)g);
  }
  m->G_part = (int64_t)glist.size();
  CU(reserve(m->d_send, m->c_send, send.size() * sizeof(int32_t)));
  CU(reserve(m->d_recv, m->c_recv, recv.size() * sizeof(int32_t)));
  CU(reserve(m->d_glist, m->c_glist, glist.size() * sizeof(int32_t)));
  if (!send.empty()) CU(cudaMemcpy(m->d_send, send.data(), send.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!recv.empty()) CU(cudaMemcpy(m->d_recv, recv.data(), recv.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!glist.empty()) CU(cudaMemcpy(m->d_glist, glist.data(), glist.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return DG_OK;
}

// Calls that need the whole mesh on one device refuse a partitioned mesh.
dg_status whole_mesh_only(dg_mesh* m, const char* what) {
  if (m->nparts > 1)
    return fail(m, DG_ERR_UNSUPPORTED, "%s needs the whole mesh: clear the partition first "
                "(dg_set_partition(mesh, 1, 0))", what);
  return DG_OK;
}

}  // namespace

extern "C" {

// Transpose of one SSP-RK3 step given its three stage inputs b0 = q, b1 = q1, b2 = q2 (each
// NV planes followed by its P' plane).
dg_status step_transpose(dg_mesh* m, const double* b0, const double* b1, const double* b2, double dt,
                         const double* lo, double* lam_in, cudaStream_t s) {
  double* l2 = m->adj_l[0];
  double* l1 = m->adj_l[1];
  const double* p0 = (const double*)pp_plane(m, (void*)b0);
  const double* p1 = (const double*)pp_plane(m, (void*)b1);
  const double* p2 = (const double*)pp_plane(m, (void*)b2);
  // q3 = 1/3 q + 2/3 (q2 + dt L(q2)):   lam_q2 = 2/3 (lam + dt J(q2)^T lam)
  dg_status st = vjp_pass(m, b2, p2, lo, nullptr, 0.0, nullptr, 0.0, lo, 2.0 / 3.0, dt, l2, s);
  // q2 = 3/4 q + 1/4 (q1 + dt L(q1)):   lam_q1 = 1/4 (lam_q2 + dt J(q1)^T lam_q2)
  if (st == DG_OK) st = vjp_pass(m, b1, p1, l2, nullptr, 0.0, nullptr, 0.0, l2, 0.25, dt, l1, s);
  // q1 = q + dt L(q):   lam_q = 1/3 lam + 3/4 lam_q2 + lam_q1 + dt J(q)^T lam_q1
  if (st == DG_OK) st = vjp_pass(m, b0, p0, l1, lo, 1.0 / 3.0, l2, 0.75, l1, 1.0, dt, lam_in, s);
  return st;
}

dg_status dg_rhs_vjp(dg_mesh* m, const void* q, const void* lam, void* out, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "the adjoint");
  if (!m || !q || !lam || !out) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  if (m->desc.nu > 0.0) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint has no viscous term");
  dg_status st = ensure_adjoint_ws(m);
  if (st != DG_OK) return st;
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  const void* theta = (const char*)q + (size_t)(m->NV - 1) * plane(m) * m->tsize;
  CU(dgk::launch_pprime(m->prec, (int32_t)m->E, m->n1, m->D, theta, m->d_bg, m->d_bgc, m->ph, m->d_ppscratch, s));
  return vjp_pass(m, (const double*)q, (const double*)m->d_ppscratch, (const double*)lam, nullptr, 0.0,
                  nullptr, 0.0, nullptr, 1.0, 1.0, (double*)out, s);
}

dg_status dg_step_state(dg_mesh* m, const void* q_in, void* q_out, double dt, int32_t nsteps,
                        void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "dg_step_state");
  if (!m || !q_in || !q_out || nsteps < 0 || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  dg_status st = ensure_adjoint_ws(m);
  if (st != DG_OK) return st;
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  st = stage_in(m, q_in, m->adj_q[0], s);
  for (int32_t i = 0; st == DG_OK && i < nsteps; ++i) st = rk3_on(m, m->adj_q[0], m->adj_q[1], m->adj_q[2], dt, s);
  if (st != DG_OK) return st;
  CU(cudaMemcpyAsync(q_out, m->adj_q[0], (size_t)m->NV * plane(m) * m->tsize, cudaMemcpyDeviceToDevice, s));
  return DG_OK;
}

dg_status dg_step_vjp(dg_mesh* m, const void* q_in, double dt, const void* lam_out, void* lam_in,
                      void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "the adjoint");
  if (!m || !q_in || !lam_out || !lam_in || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (lam_out == lam_in) return fail(m, DG_ERR_ARG, "lam_out and lam_in must not alias");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  if (m->desc.nu > 0.0) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint has no viscous term");
  dg_status st = ensure_adjoint_ws(m);
  if (st != DG_OK) return st;
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  // recompute the stage states q, q1, q2 of this step
  void* b0 = m->adj_q[0];
  void* b1 = m->adj_q[1];
  void* b2 = m->adj_q[2];
  st = stage_in(m, q_in, b0, s);
  if (st == DG_OK) st = launch_rhs_pass(m, b0, pp_plane(m, b0), b0, b1, pp_plane(m, b1), 1, dt, 0.0, 1.0, s);
  if (st == DG_OK) st = launch_rhs_pass(m, b1, pp_plane(m, b1), b0, b2, pp_plane(m, b2), 1, dt, 0.75, 0.25, s);
  if (st != DG_OK) return st;
  return step_transpose(m, (const double*)b0, (const double*)b1, (const double*)b2, dt,
                        (const double*)lam_out, (double*)lam_in, s);
}

dg_status dg_step_record(dg_mesh* m, const void* q_in, void* q_out, void* record, double dt, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "dg_step_record");
  if (!m || !q_in || !q_out || !record || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  if (m->desc.nu > 0.0) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint has no viscous term");
  dg_status st = ensure_adjoint_ws(m);
  if (st != DG_OK) return st;
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  const size_t sb = (size_t)(m->NV + 1) * plane(m);      // doubles per recorded state
  double* r0 = (double*)record;
  double* r1 = r0 + sb;
  double* r2 = r1 + sb;
  st = stage_in(m, q_in, r0, s);
  if (st == DG_OK) st = launch_rhs_pass(m, r0, pp_plane(m, r0), r0, r1, pp_plane(m, r1), 1, dt, 0.0, 1.0, s);
  if (st == DG_OK) st = launch_rhs_pass(m, r1, pp_plane(m, r1), r0, r2, pp_plane(m, r2), 1, dt, 0.75, 0.25, s);
  if (st == DG_OK)
    st = launch_rhs_pass(m, r2, pp_plane(m, r2), r0, q_out, pp_plane(m, m->adj_q[0]), 1, dt, 1.0 / 3.0, 2.0 / 3.0, s);
  return st;
}

dg_status dg_step_vjp_record(dg_mesh* m, const void* record, double dt, const void* lam_out, void* lam_in,
                             void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "the adjoint");
  if (!m || !record || !lam_out || !lam_in || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (lam_out == lam_in) return fail(m, DG_ERR_ARG, "lam_out and lam_in must not alias");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  if (m->desc.nu > 0.0) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint has no viscous term");
  dg_status st = ensure_adjoint_ws(m);
  if (st != DG_OK) return st;
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  const size_t sb = (size_t)(m->NV + 1) * plane(m);
  const double* r0 = (const double*)record;
  return step_transpose(m, r0, r0 + sb, r0 + 2 * sb, dt, (const double*)lam_out, (double*)lam_in, s);
}

dg_status dg_set_theta(dg_mesh* m, const double* theta, int where) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !theta || (where != DG_HOST && where != DG_DEVICE)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  const size_t bytes = (size_t)plane(m) * sizeof(double);
  const double* src = theta;
  double* tmp = nullptr;
  if (where == DG_HOST) {
    CU(cudaMalloc(&tmp, bytes > 0 ? bytes : 8));
    CU(cudaMemcpy(tmp, theta, bytes, cudaMemcpyHostToDevice));
    src = tmp;
  }
  cudaError_t e = dgk::launch_theta_state(m->prec, (int32_t)m->E, m->n1, m->D, m->d_bg, src,
                                          m->ph.theta0, m->q[0], plane(m), m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "theta state failed: %s", cudaGetErrorString(e));
  m->pp_valid = false;
  return DG_OK;
}

dg_status dg_theta_vjp(dg_mesh* m, const double* theta, const void* lam_q, double* lam_theta,
                       void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "the adjoint");
  if (!m || !theta || !lam_q || !lam_theta) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  CU(dgk::launch_theta_vjp((int32_t)m->E, m->n1, m->D, m->d_bg, theta, m->ph.theta0,
                           (const double*)lam_q, lam_theta, s));
  return DG_OK;
}

dg_status dg_ke_grad(dg_mesh* m, const void* q, void* out, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "dg_ke_grad");
  if (!m || !q || !out) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (m->prec != DG_FP64) return fail(m, DG_ERR_UNSUPPORTED, "the adjoint is FP64 only");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  CU(dgk::launch_ke_grad((int32_t)m->E, m->n1, m->D, m->d_elem, d_w(m), m->root_h, m->d_bg,
                         (const double*)q, plane(m), (double*)out, s));
  return DG_OK;
}

dg_status dg_set_option(dg_mesh* m, int32_t option, int64_t value) {
  if (!m) return DG_ERR_ARG;
  if (option == DG_OPT_STAGE_KERNEL) {
    if (value < 0 || value > 5) return fail(m, DG_ERR_ARG, "stage kernel layout must be 0 .. 5");
    m->variant = (int)value;
    return DG_OK;
  }
  if (option == DG_OPT_FAIL_NEXT_ADAPT) {
    if (value < 0 || value > 2) return fail(m, DG_ERR_ARG, "failure injection must be 0, 1 or 2");
    m->fail_next_adapt = (int)value;
    return DG_OK;
  }
  return fail(m, DG_ERR_ARG, "unknown option %d", option);
}

dg_status dg_set_time(dg_mesh* m, double t) {
  if (!m || !std::isfinite(t)) return fail(m, DG_ERR_ARG, "bad argument");
  m->time = t;
  return DG_OK;
}

double dg_get_time(const dg_mesh* m) { return m ? m->time : 0.0; }

const char* dg_version(void) { return "gb300-dgsem 0.1 (sm_103a)"; }

const char* dg_last_error(const dg_mesh* m) { return m ? m->err.c_str() : "null mesh"; }

dg_status dg_mesh_create(const dg_mesh_desc* desc, void* stream, dg_mesh** out) {
  dg_mesh* m = nullptr;
  if (!desc || !out) return DG_ERR_ARG;
  *out = nullptr;
  if (desc->dim != 2 && desc->dim != 3) return DG_ERR_ARG;
  if (desc->N < 1 || desc->N > DG_MAX_N) return DG_ERR_ARG;
  if (desc->max_level < 0 || desc->max_level > DG_MAX_LEVEL) return DG_ERR_ARG;
  if (desc->precision != DG_FP64 && desc->precision != DG_FP32_PERT) return DG_ERR_ARG;
  if (!(desc->nu >= 0.0)) return DG_ERR_ARG;
  if (desc->nu > 0.0 && desc->precision != DG_FP64) return DG_ERR_UNSUPPORTED;   // viscous: FP64
  for (int a = 0; a < desc->dim; ++a) {
    if (desc->base[a] < 1 || !(desc->length[a] > 0.0)) return DG_ERR_ARG;
    if (((int64_t)desc->base[a] << desc->max_level) >= (1 << 19)) return DG_ERR_ARG;
  }
  if (!(desc->p0 > 0.0) || !(desc->R > 0.0) || !(desc->cp > desc->R) || !(desc->theta0 > 0.0))
    return DG_ERR_ARG;
  if (desc->equations != DG_EQ_EULER && desc->equations != DG_EQ_TRACER) return DG_ERR_ARG;
  // the neutral background exists below z = cp theta0 / g, where the Exner function vanishes
  if (desc->g > 0.0 && !(desc->length[desc->dim - 1] < desc->cp * desc->theta0 / desc->g)) return DG_ERR_ARG;
  // a periodic vertical axis needs a uniform background (g = 0)
  if (desc->periodic[desc->dim - 1] && desc->g != 0.0) return DG_ERR_UNSUPPORTED;
  if (desc->face_mode != DG_FACE_MORTAR && desc->face_mode != DG_FACE_INTERP) return DG_ERR_ARG;
  if (desc->equations == DG_EQ_TRACER) {
    if (desc->dim != 2 || desc->precision != DG_FP64 || desc->nu != 0.0) return DG_ERR_UNSUPPORTED;
    if (!(desc->wind_period > 0.0)) return DG_ERR_ARG;
  } else if (desc->face_mode != DG_FACE_MORTAR) {
    return DG_ERR_UNSUPPORTED;
  }
  m = new (std::nothrow) dg_mesh();
  if (!m) return DG_ERR_OOM;
  m->desc = *desc;
  m->D = desc->dim; m->N = desc->N; m->n1 = m->N + 1;
  m->NP = m->D == 3 ? m->n1 * m->n1 * m->n1 : m->n1 * m->n1;
  m->NF = m->D == 3 ? m->n1 * m->n1 : m->n1;
  m->tracer = desc->equations == DG_EQ_TRACER;
  m->NV = m->tracer ? 1 : m->D + 2; m->NSUB = 1 << (m->D - 1);
  m->prec = desc->precision;
  m->tsize = m->prec == DG_FP64 ? sizeof(double) : sizeof(float);
  // fastest measured layouts: the line layout for FP32 in 3D, face fluxes once per face for FP64
  m->variant = (m->prec == DG_FP32_PERT && m->D == 3) ? 4 : (m->prec == DG_FP64 && !m->tracer ? 5 : 2);
  m->stream = (cudaStream_t)stream;
  m->ph.theta0 = desc->theta0; m->ph.p0 = desc->p0; m->ph.g = desc->g; m->ph.R = desc->R;
  m->ph.cp = desc->cp; m->ph.cv = desc->cp - desc->R; m->ph.gamma = desc->cp / (desc->cp - desc->R);
  {
    // binom(gamma, k) = prod_{j<k} (gamma - j) / k! for the P' series
    double c = 1.0;
    for (int k = 1; k <= dgk::kSeries; ++k) {
      c = c * (m->ph.gamma - (k - 1)) / k;
      m->ph.binom[k - 1] = c;
    }
    for (int k = 0; k < 3; ++k) m->ph.rel[k] = (float)(m->ph.binom[k + 1] / m->ph.gamma);
  }
  int base[3] = {desc->base[0], desc->base[1], desc->dim == 3 ? desc->base[2] : 1};
  for (int a = 0; a < 3; ++a) m->root_h[a] = a < m->D ? desc->length[a] / base[a] : 1.0;
  int per[3] = {0, 0, 0};
  for (int a = 0; a < m->D; ++a) per[a] = desc->periodic[a] ? 1 : 0;
  m->forest = dgl::Forest(m->D, base, desc->max_level, per);
  m->basis = dgl::make_basis(m->N);
  dg_status st = init_device_tables(m);
  if (st == DG_OK) st = upload_ops(m);
  if (st == DG_OK) st = rebuild_topology(m);
  if (st == DG_OK) st = alloc_states(m);
  if (st == DG_OK) {
    if (cudaMalloc(&m->d_partial, dgk::integrals_scratch_doubles() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_out, 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_bgint, 12 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m->d_bad, sizeof(int)) != cudaSuccess)
      st = fail(m, DG_ERR_OOM, "scratch allocation failed");
  }
  if (st == DG_OK) {
    if (cudaMemsetAsync(m->q[0], 0, (size_t)m->NV * plane(m) * m->tsize, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
      st = fail(m, DG_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (st != DG_OK) { dg_mesh_destroy(m); return st; }
  *out = m;
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream); else cudaDeviceSynchronize();
  for (int i = 0; i < 3; ++i) dfree(m->q[i]);
  dfree(m->q_spare); dfree(m->d_tm); dfree(m->d_ind);
  dfree(m->d_elem); dfree(m->d_conn); dfree(m->d_groups); dfree(m->d_bg); dfree(m->d_mbuf);
  dfree(m->d_bgf); dfree(m->d_bgc); dfree(m->d_ppscratch);
  dfree(m->d_sigma); dfree(m->d_V); dfree(m->d_vbuf);
  dfree(m->d_ops); dfree(m->d_opsd); dfree(m->d_partial); dfree(m->d_out); dfree(m->d_bad); dfree(m->d_bgint);
  for (int i = 0; i < 3; ++i) dfree(m->adj_q[i]);
  for (int i = 0; i < 2; ++i) dfree(m->adj_l[i]);
  dfree(m->d_abuf);
  dfree(m->d_send); dfree(m->d_recv); dfree(m->d_glist);
  dfree(m->d_fbuf); dfree(m->d_fconf); dfree(m->d_fbnd);
  for (int i = 0; i < 3; ++i) if (m->h_pin[i]) cudaFreeHost(m->h_pin[i]);
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  if (m->ev_order) cudaEventDestroy(m->ev_order);
  delete m;
}

int64_t dg_num_elements(const dg_mesh* m) { return m ? m->E : 0; }
int64_t dg_num_nodes(const dg_mesh* m) { return m ? m->E * m->NP : 0; }

dg_status dg_get_leaves(const dg_mesh* mc, int32_t* out, size_t cap) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !out) return DG_ERR_ARG;
  if (cap < (size_t)m->E * 5) return fail(m, DG_ERR_ARG, "leaf buffer too small");
  const auto& L = m->forest.leaves();
  for (int64_t e = 0; e < m->E; ++e) {
    out[e * 5] = m->forest.root_index(L[e]);
    out[e * 5 + 1] = L[e].level;
    for (int a = 0; a < 3; ++a) out[e * 5 + 2 + a] = L[e].c[a];
  }
  return DG_OK;
}

dg_status dg_get_faces(const dg_mesh* mc, int64_t counts[3], int32_t* conforming, size_t cap_c,
                       int32_t* mortars, size_t cap_m, int32_t* boundary, size_t cap_b) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !counts) return DG_ERR_ARG;
  counts[0] = (int64_t)m->conf.size() / 3;
  counts[1] = (int64_t)m->mort.size() / 7;
  counts[2] = (int64_t)m->bnd.size() / 3;
  if (conforming && cap_c >= (size_t)counts[0]) std::memcpy(conforming, m->conf.data(), m->conf.size() * 4);
  if (mortars && cap_m >= (size_t)counts[1]) std::memcpy(mortars, m->mort.data(), m->mort.size() * 4);
  if (boundary && cap_b >= (size_t)counts[2]) std::memcpy(boundary, m->bnd.data(), m->bnd.size() * 4);
  return DG_OK;
}

dg_status dg_set_state(dg_mesh* m, const void* q, int layout_flags, int where) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !q || (where != DG_HOST && where != DG_DEVICE) ||
      (layout_flags != DG_LAYOUT_PLANES && layout_flags != DG_LAYOUT_ELEMENTS))
    return fail(m, DG_ERR_ARG, "bad argument");
  const size_t bytes = (size_t)m->NV * plane(m) * m->tsize;
  m->pp_valid = false;
  const cudaMemcpyKind kind = where == DG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (layout_flags == DG_LAYOUT_PLANES) {
    CU(cudaMemcpyAsync(m->q[0], q, bytes, kind, m->stream));
  } else {
    // element-major in: host data through the stage buffer q[1] (it holds nothing between steps)
    const void* src = q;
    if (where == DG_HOST) {
      CU(cudaMemcpyAsync(m->q[1], q, bytes, kind, m->stream));
      src = m->q[1];
    }
    CU(dgk::launch_state_layout(m->tsize, 1, m->E, m->NP, m->NV, src, m->q[0], plane(m), m->stream));
  }
  CU(cudaStreamSynchronize(m->stream));
  return DG_OK;
}

dg_status dg_get_state(dg_mesh* m, void* q, int layout_flags, int where) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !q || (where != DG_HOST && where != DG_DEVICE) ||
      (layout_flags != DG_LAYOUT_PLANES && layout_flags != DG_LAYOUT_ELEMENTS))
    return fail(m, DG_ERR_ARG, "bad argument");
  const size_t bytes = (size_t)m->NV * plane(m) * m->tsize;
  if (layout_flags == DG_LAYOUT_PLANES) {
    CU(cudaMemcpyAsync(q, m->q[0], bytes, where == DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       m->stream));
  } else if (where == DG_DEVICE) {
    CU(dgk::launch_state_layout(m->tsize, 0, m->E, m->NP, m->NV, m->q[0], q, plane(m), m->stream));
  } else {
    CU(dgk::launch_state_layout(m->tsize, 0, m->E, m->NP, m->NV, m->q[0], m->q[1], plane(m), m->stream));
    CU(cudaMemcpyAsync(q, m->q[1], bytes, cudaMemcpyDeviceToHost, m->stream));
  }
  CU(cudaStreamSynchronize(m->stream));
  return DG_OK;
}

dg_status dg_get_pprime(dg_mesh* m, void* out, int where) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !out || (where != DG_HOST && where != DG_DEVICE)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  dg_status st = dgi::ensure_pp(m, m->stream);
  if (st != DG_OK) return st;
  CU(cudaMemcpyAsync(out, pp_plane(m, m->q[0]), (size_t)plane(m) * m->tsize,
                     where == DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, m->stream));
  CU(cudaStreamSynchronize(m->stream));
  return DG_OK;
}

// Evaluates the bubble at the nodes: into the state (theta_out == nullptr) or as theta' itself.
static dg_status bubble_eval(dg_mesh* m, const dg_bubble_desc* b, double* theta_out) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !b) return fail(m, DG_ERR_ARG, "bad argument");
  for (int a = 0; a < m->D; ++a)
    if (!(b->radius[a] > 0.0)) return fail(m, DG_ERR_ARG, "bubble radius must be positive");
  if (b->n_rff < 0 || (b->n_rff > 0 && (!b->rff_k || !b->rff_phase)))
    return fail(m, DG_ERR_ARG, "bad random-feature arguments");
  double* dk = nullptr;
  double* dp = nullptr;
  if (b->n_rff > 0) {
    CU(cudaMalloc(&dk, (size_t)b->n_rff * 3 * sizeof(double)));
    CU(cudaMalloc(&dp, (size_t)b->n_rff * sizeof(double)));
    CU(cudaMemcpy(dk, b->rff_k, (size_t)b->n_rff * 3 * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dp, b->rff_phase, (size_t)b->n_rff * sizeof(double), cudaMemcpyHostToDevice));
  }
  const double scale = b->n_rff > 0 ? b->rff_sigma * std::sqrt(2.0 / b->n_rff) : 0.0;
  m->pp_valid = false;
  cudaError_t e = dgk::launch_bubble(m->prec, (int32_t)m->E, m->n1, m->D, m->d_elem, d_x(m), m->root_h,
                                     m->d_bg, b->center, b->radius, b->amp, b->n_rff, scale, dk, dp,
                                     m->ph.theta0, m->q[0], plane(m), theta_out, m->stream);
  cudaError_t e2 = cudaStreamSynchronize(m->stream);
  dfree(dk); dfree(dp);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(m, DG_ERR_CUDA, "bubble kernel failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return DG_OK;
}

dg_status dg_set_bubble(dg_mesh* m, const dg_bubble_desc* b) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && b && m->tracer) {
    if (b->n_rff != 0) return fail(m, DG_ERR_ARG, "a tracer bell takes no random field");
    for (int a = 0; a < 2; ++a)
      if (!(b->radius[a] > 0.0)) return fail(m, DG_ERR_ARG, "radius must be positive");
    cudaError_t e = dgk::launch_tracer_bell((int32_t)m->E, m->n1, m->d_elem, d_x(m), m->root_h, b->center,
                                            b->radius, b->amp, (double*)m->q[0], m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "tracer bell failed: %s", cudaGetErrorString(e));
    return DG_OK;
  }
  return bubble_eval(m, b, nullptr);
}

dg_status dg_set_vortex(dg_mesh* m, const dg_vortex_desc* v) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !v) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer || m->D != 2) return fail(m, DG_ERR_ARG, "the vortex needs a 2D Euler mesh");
  if (m->desc.p0 != 1.0 || m->desc.R != 1.0 || m->desc.theta0 != 1.0 || m->desc.g != 0.0)
    return fail(m, DG_ERR_ARG, "the vortex is nondimensional: p0 = R = theta0 = 1, g = 0");
  if (!std::isfinite(v->beta) || !std::isfinite(v->t)) return fail(m, DG_ERR_ARG, "bad vortex");
  const int per[2] = {m->desc.periodic[0] ? 1 : 0, m->desc.periodic[1] ? 1 : 0};
  cudaError_t e = dgk::launch_vortex(m->prec, (int32_t)m->E, m->n1, m->d_elem, d_x(m), m->root_h,
                                     m->desc.length, per, v->center, v->beta, v->u_inf, v->t,
                                     m->ph.gamma, m->d_bg, m->q[0], plane(m), m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "vortex failed: %s", cudaGetErrorString(e));
  m->pp_valid = false;
  return DG_OK;
}

dg_status dg_bubble_theta(dg_mesh* m, const dg_bubble_desc* b, double* theta) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !theta) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "no theta' field on a tracer mesh");
  return bubble_eval(m, b, theta);
}

dg_status dg_rhs(dg_mesh* m, const void* q, void* dqdt, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !q || !dqdt) return fail(m, DG_ERR_ARG, "bad argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  if (m->tracer) {
    m->stage_g = wind_factor(m, m->time);
    return launch_rhs_pass(m, q, nullptr, nullptr, dqdt, nullptr, 0, 0.0, 0.0, 1.0, s);
  }
  const void* theta = (const char*)q + (size_t)(m->NV - 1) * plane(m) * m->tsize;
  CU(dgk::launch_pprime(m->prec, (int32_t)m->E, m->n1, m->D, theta, m->d_bg, m->d_bgc, m->ph, m->d_ppscratch, s));
  return launch_rhs_pass(m, q, m->d_ppscratch, nullptr, dqdt, nullptr, 0, 0.0, 0.0, 1.0, s);
}

dg_status dg_step(dg_mesh* m, double dt, int32_t nsteps, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1)
    return fail(m, DG_ERR_STATE, "a partitioned mesh steps stage by stage (dg_stage), with the halo "
                "traces of each stage input exchanged before the stage");
  if (!m || nsteps < 0 || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  void* p0 = pp_plane(m, m->q[0]);
  void* p1 = pp_plane(m, m->q[1]);
  void* p2 = pp_plane(m, m->q[2]);
  if (nsteps > 0) {
    dg_status st0 = dgi::ensure_pp(m, s);
    if (st0 != DG_OK) return st0;
  }
  for (int32_t it = 0; it < nsteps; ++it) {
    // Shu-Osher SSP-RK3: q1 = q + dt L(q); q2 = 3/4 q + 1/4 (q1 + dt L(q1));
    // q^{n+1} = 1/3 q + 2/3 (q2 + dt L(q2)), the last one written over q^n (each thread reads
    // q^n only at its own node, and the stage reads P' of q2, not of q^n).  The stages sit at
    // t, t + dt and t + dt/2 (the tracer's wind is evaluated there).
    const double t = m->time;
    m->stage_g = m->tracer ? wind_factor(m, t) : 1.0;
    dg_status st = launch_rhs_pass(m, m->q[0], p0, m->q[0], m->q[1], p1, 1, dt, 0.0, 1.0, s);
    m->stage_g = m->tracer ? wind_factor(m, t + dt) : 1.0;
    if (st == DG_OK) st = launch_rhs_pass(m, m->q[1], p1, m->q[0], m->q[2], p2, 1, dt, 0.75, 0.25, s);
    m->stage_g = m->tracer ? wind_factor(m, t + 0.5 * dt) : 1.0;
    if (st == DG_OK) st = launch_rhs_pass(m, m->q[2], p2, m->q[0], m->q[0], p0, 1, dt, 1.0 / 3.0, 2.0 / 3.0, s);
    if (st != DG_OK) return st;
    m->time = t + dt;
  }
  return DG_OK;
}

dg_status dg_indicator(dg_mesh* m, double* out, size_t cap) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !out || cap < (size_t)m->E) return fail(m, DG_ERR_ARG, "bad argument");
  CU(reserve(m->d_ind, m->c_ind, (size_t)(m->E > 0 ? m->E : 1) * sizeof(double)));
  double* d = m->d_ind;
  cudaError_t e = m->tracer
                      ? dgk::launch_tracer_indicator((int32_t)m->E, m->n1, (const double*)m->q[0], d, m->stream)
                      : dgk::launch_indicator(m->prec, (int32_t)m->E, m->n1, m->D, m->d_bg, m->q[0], plane(m),
                                              m->ph.theta0, d, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)m->E * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "indicator failed: %s", cudaGetErrorString(e));
  return DG_OK;
}

dg_status dg_primitives(dg_mesh* m, double* out, size_t cap, void* stream) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || (!out && m->E > 0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  const size_t need = (size_t)(m->D + 1) * (size_t)m->E * (size_t)m->NP;
  if (cap < need) return fail(m, DG_ERR_ARG, "output holds %zu doubles, %zu needed", cap, need);
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  cudaError_t e = dgk::launch_primitives(m->prec, (int32_t)m->E, m->n1, m->D, m->d_bg, m->q[0], plane(m),
                                         m->ph.theta0, out, s);
  if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "primitives failed: %s", cudaGetErrorString(e));
  return DG_OK;
}

dg_status dg_adapt(dg_mesh* m, const dg_adapt_params* p, dg_adapt_report* rep) {
  if (!m || !p) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->nparts > 1) return whole_mesh_only(m, "dg_adapt");
  if (p->buffer < 0) return fail(m, DG_ERR_ARG, "buffer must be >= 0");
  const int maxl = p->max_level < 0 ? m->desc.max_level : p->max_level;
  if (maxl > m->desc.max_level) return fail(m, DG_ERR_ARG, "max_level above the mesh limit");
  const int inject = m->fail_next_adapt;
  m->fail_next_adapt = 0;
  std::vector<uint8_t> tag((size_t)m->E, 0);
  if (p->criterion == DG_CRIT_FLAGS) {
    if (!p->flags) return fail(m, DG_ERR_ARG, "flags missing");
    for (int64_t e = 0; e < m->E; ++e) tag[e] = p->flags[e] ? 1 : 0;
  } else if (p->criterion == DG_CRIT_THETA && m->tracer) {
    CU(pin_reserve(m, 2, (size_t)(m->E > 0 ? m->E : 1) * sizeof(double)));
    double* ind = reinterpret_cast<double*>(m->h_pin[2]);
    dg_status st = dg_indicator(m, ind, (size_t)m->E);
    if (st != DG_OK) return st;
    for (int64_t e = 0; e < m->E; ++e) tag[e] = ind[e] > p->threshold ? 1 : 0;
  } else if (p->criterion == DG_CRIT_THETA) {
    // the comparison with the threshold decided on the device (launch_tags: the decisions of
    // dg_indicator > threshold, mostly without its divisions), one byte per element back
    CU(pin_reserve(m, 2, (size_t)(m->E > 0 ? m->E : 1)));
    CU(reserve(m->d_ind, m->c_ind, (size_t)(m->E > 0 ? m->E : 1) * sizeof(double)));
    uint8_t* d_tag = reinterpret_cast<uint8_t*>(m->d_ind);
    CU(dgk::launch_tags(m->prec, (int32_t)m->E, m->n1, m->D, m->d_bg, m->q[0], plane(m), m->ph.theta0,
                        p->threshold, d_tag, m->stream));
    if (m->E > 0) CU(cudaMemcpyAsync(m->h_pin[2], d_tag, (size_t)m->E, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    std::memcpy(tag.data(), m->h_pin[2], (size_t)m->E);
  } else {
    return fail(m, DG_ERR_ARG, "unknown criterion");
  }
  dgl::Forest nf;
  std::vector<dgl::TransferEntry> tmap;
  int64_t nref = 0, ncoarse = 0;
  std::string why;
  if (!m->forest.regrid(tag, p->buffer, maxl, &nf, &tmap, &nref, &ncoarse, &why, inject == 0))
    return fail(m, DG_ERR_STATE, "regrid failed: %s", why.c_str());
  const int64_t E_old = m->E;
  if (nref == 0 && ncoarse == 0 && inject == 0) {
    // nothing refined or coarsened: the new forest is the old one (the host pass skipped
    // building it), the transfer would copy every element and the tables would come out the
    // same, so the mesh is left as it is
    if (rep) {
      rep->elements_before = E_old;
      rep->elements_after = E_old;
      rep->refined = 0;
      rep->coarsened = 0;
    }
    return DG_OK;
  }
  const int64_t plane_old = plane(m);
  const int64_t E_new = nf.size();
  if ((int64_t)(m->NV + 1) * E_new * m->NP >= ((int64_t)1 << 31))
    return fail(m, DG_ERR_UNSUPPORTED, "mesh too large for 32-bit state offsets (%lld elements)",
                (long long)E_new);
  const int64_t plane_new = E_new * m->NP;
  // Until the new forest is committed below, every failure leaves the mesh as it was: the
  // transfer map and the spare state are scratch, and the stage buffers q[1], q[2] hold nothing
  // between steps (growing them keeps the old mesh valid).
  // the device reads the map as rows of 9 int32 {kind, src[8]}: the host entries as they lie
  static_assert(sizeof(dgl::TransferEntry) == 9 * sizeof(int32_t), "transfer rows are 9 int32");
  const size_t tm_bytes = tmap.size() * sizeof(dgl::TransferEntry);
  CU(reserve(m->d_tm, m->c_tm, tm_bytes + 4));
  CU(upload_pinned(m, 0, {{m->d_tm, {tmap.data(), tm_bytes}}}));
  CU(reserve(m->q_spare, m->q_spare_cap, (size_t)(m->NV + 1) * plane_new * m->tsize));
  const size_t sb_new = (size_t)(m->NV + 1) * plane_new * m->tsize;
  for (int i = 1; i < 3; ++i) CU(reserve(m->q[i], m->q_cap[i], sb_new));
  // the transfer reads q^n and writes the spare buffer, which then becomes q^n; it needs only
  // the map, so it runs while the host builds the new face tables
  {
    cudaError_t e = dgk::launch_transfer(m->prec, (int32_t)E_new, m->n1, m->D, m->NV, m->d_tm, m->d_opsd, m->q[0],
                                         plane_old, m->q_spare, plane_new, m->stream);
    if (e != cudaSuccess) return fail(m, DG_ERR_CUDA, "transfer failed: %s", cudaGetErrorString(e));
  }
  HostTables tables;
  dg_status st = inject == 1 ? fail(m, DG_ERR_STATE, "injected failure before the commit")
                             : build_tables(m, nf, &tables);
  if (st != DG_OK) {
    cudaStreamSynchronize(m->stream);   // the transfer wrote only the spare buffer
    return st;
  }
  // commit: from here a failure leaves device tables of mixed sizes, so the mesh is marked
  // unusable and every later call on it is refused
  m->forest = std::move(nf);
  ++m->generation;
  st = inject == 2 ? fail(m, DG_ERR_OOM, "injected failure after the commit")
                   : upload_tables(m, std::move(tables));
  if (st == DG_OK) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) st = fail(m, DG_ERR_CUDA, "transfer failed: %s", cudaGetErrorString(e));
  }
  if (st != DG_OK) {
    cudaStreamSynchronize(m->stream);
    m->broken = true;
    return st;
  }
  std::swap(m->q[0], m->q_spare);
  std::swap(m->q_cap[0], m->q_spare_cap);
  m->pp_valid = false;
  if (rep) {
    rep->elements_before = E_old;
    rep->elements_after = m->E;
    rep->refined = nref;
    rep->coarsened = ncoarse;
  }
  return DG_OK;
}

// a + b as an unevaluated pair: returns fl(a + b), *err the exact remainder (Knuth's TwoSum).
static double two_sum(double a, double b, double* err) {
  const double t = a + b;
  const double bb = t - a;
  *err = (a - (t - bb)) + (b - bb);
  return t;
}

// The background sums (int rho_bar, int (p_bar cv/R + rho_bar g z), volume) depend on the mesh
// alone and are taken once per topology; each call sums the parts that carry the state and
// adds the two compensated results with their rounding errors.
dg_status dg_integrals(dg_mesh* m, double out[DG_NUM_INTEGRALS]) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m && m->nparts > 1) return whole_mesh_only(m, "dg_integrals");
  if (!m || !out) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->tracer) {
    double r[2] = {0.0, 0.0};
    int bad = 0;
    CU(cudaMemsetAsync(m->d_bad, 0, sizeof(int), m->stream));
    CU(dgk::launch_tracer_total((int32_t)m->E, m->n1, m->d_elem, d_w(m), m->root_h, (const double*)m->q[0],
                                m->d_partial, m->d_bad, m->d_out, m->stream));
    CU(cudaMemcpyAsync(r, m->d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaMemcpyAsync(&bad, m->d_bad, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    out[0] = r[0]; out[1] = 0.0; out[2] = 0.0; out[3] = r[1]; out[4] = r[0];
    if (bad) return fail(m, DG_ERR_STATE, "non-finite value in the state");
    return DG_OK;
  }
  if (!m->bgint_valid) {
    CU(dgk::launch_integrals(m->prec, true, (int32_t)m->E, m->n1, m->D, m->d_elem, d_x(m), d_w(m), m->root_h,
                             m->d_bg, nullptr, plane(m), m->ph, m->d_partial, m->d_bad, m->d_out, m->stream));
    CU(cudaMemcpyAsync(m->bgint, m->d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaMemcpyAsync(m->d_bgint, m->d_out, 6 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    m->bgint_valid = true;
  }
  CU(cudaMemsetAsync(m->d_bad, 0, sizeof(int), m->stream));
  CU(dgk::launch_integrals(m->prec, false, (int32_t)m->E, m->n1, m->D, m->d_elem, d_x(m), d_w(m), m->root_h,
                           m->d_bg, m->q[0], plane(m), m->ph, m->d_partial, m->d_bad, m->d_out, m->stream));
  double S[6];
  int bad = 0;
  CU(cudaMemcpyAsync(S, m->d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CU(cudaMemcpyAsync(&bad, m->d_bad, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CU(cudaStreamSynchronize(m->stream));
  const double* B = m->bgint;
  double e0, e1;
  const double t0 = two_sum(B[0], S[0], &e0);
  const double t1 = two_sum(B[1], S[1], &e1);
  out[0] = t0 + (e0 + (B[3] + S[3]));          // mass
  out[1] = t1 + (e1 + (B[4] + S[4]));          // total energy
  out[2] = S[2];                               // kinetic energy
  out[3] = B[2];                               // volume
  out[4] = S[0];                               // perturbation mass
  if (bad) return fail(m, DG_ERR_STATE, "non-finite value in the state");
  return DG_OK;
}

dg_status dg_enable_timing(dg_mesh* m, int32_t enable) {
  if (!m) return DG_ERR_ARG;
  m->timing = enable != 0;
  return DG_OK;
}

dg_status dg_stage_timing(dg_mesh* m, double* total_ms, int64_t* launches, int32_t reset) {
  if (m && m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (!m || !total_ms || !launches) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->ev_used > 0) CU(cudaEventSynchronize(m->ev[m->ev_used - 1]));
  double sum = 0.0;
  for (size_t i = 0; i + 1 < m->ev_used; i += 2) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, m->ev[i], m->ev[i + 1]));
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)(m->ev_used / 2);
  if (reset) m->ev_used = 0;
  return DG_OK;
}

dg_status dg_set_partition(dg_mesh* m, int32_t nparts, int32_t part) {
  if (!m) return DG_ERR_ARG;
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (nparts < 1 || part < 0 || part >= nparts || nparts > m->E)
    return fail(m, DG_ERR_ARG, "need 1 <= nparts <= elements and 0 <= part < nparts");
  if (nparts > 1 && (m->tracer || m->desc.nu > 0.0))
    return fail(m, DG_ERR_UNSUPPORTED, "partitioned meshes: inviscid Euler equations only");
  m->nparts = nparts;
  m->part = part;
  dg_status st = apply_partition(m);
  if (st != DG_OK) {
    m->nparts = 1;
    m->part = 0;
    apply_partition(m);
  }
  return st;
}

dg_status dg_get_partition(const dg_mesh* mc, int64_t range[2], int64_t* send_slots, int64_t* recv_slots,
                           int64_t* slot_values) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  if (!m || !range) return DG_ERR_ARG;
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  range[0] = m->e_begin;
  range[1] = m->e_end;
  for (int q = 0; q < m->nparts; ++q) {
    if (send_slots) send_slots[q] = m->nparts > 1 ? m->send_off[q + 1] - m->send_off[q] : 0;
    if (recv_slots) recv_slots[q] = m->nparts > 1 ? m->recv_off[q + 1] - m->recv_off[q] : 0;
  }
  if (slot_values) *slot_values = (int64_t)(m->NV + 1) * m->NF;
  return DG_OK;
}

dg_status dg_halo_pack(dg_mesh* m, const void* q, const void* pp, void* sendbuf, void* stream) {
  if (!m || !q) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->nparts <= 1) return DG_OK;
  const int64_t n = m->send_off[m->nparts];
  if (n > 0 && !sendbuf) return fail(m, DG_ERR_ARG, "send buffer missing");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  CU(dgk::launch_halo(m->prec == DG_FP64 ? 0 : 1, 0, n, m->n1, m->D, m->NV, m->d_send, const_cast<void*>(q),
                      const_cast<void*>(pp), plane(m), sendbuf, s));
  return DG_OK;
}

dg_status dg_halo_unpack(dg_mesh* m, const void* recvbuf, void* q, void* pp, void* stream) {
  if (!m || !q) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->nparts <= 1) return DG_OK;
  const int64_t n = m->recv_off[m->nparts];
  if (n > 0 && !recvbuf) return fail(m, DG_ERR_ARG, "receive buffer missing");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  CU(dgk::launch_halo(m->prec == DG_FP64 ? 0 : 1, 1, n, m->n1, m->D, m->NV, m->d_recv, q, pp, plane(m),
                      const_cast<void*>(recvbuf), s));
  return DG_OK;
}

dg_status dg_stage_buffer(dg_mesh* m, int32_t index, void** q, void** pp) {
  if (!m || index < 0 || index > 2 || !q || !pp) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "not available for tracer meshes");
  if (index == 0) {
    dg_status st = dgi::ensure_pp(m, m->stream);
    if (st != DG_OK) return st;
  }
  *q = m->q[index];
  *pp = pp_plane(m, m->q[index]);
  return DG_OK;
}

dg_status dg_stage(dg_mesh* m, int32_t stage, double dt, void* stream) {
  if (!m || stage < 0 || stage > 2 || !(dt > 0.0)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->tracer || m->desc.nu > 0.0) return fail(m, DG_ERR_UNSUPPORTED, "dg_stage: inviscid Euler equations only");
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  void* p[3] = {pp_plane(m, m->q[0]), pp_plane(m, m->q[1]), pp_plane(m, m->q[2])};
  if (stage == 0) {
    dg_status st = dgi::ensure_pp(m, s);
    if (st != DG_OK) return st;
    return launch_rhs_pass(m, m->q[0], p[0], m->q[0], m->q[1], p[1], 1, dt, 0.0, 1.0, s);
  }
  if (stage == 1) return launch_rhs_pass(m, m->q[1], p[1], m->q[0], m->q[2], p[2], 1, dt, 0.75, 0.25, s);
  dg_status st = launch_rhs_pass(m, m->q[2], p[2], m->q[0], m->q[0], p[0], 1, dt, 1.0 / 3.0, 2.0 / 3.0, s);
  if (st == DG_OK) m->time += dt;
  return st;
}

// Work already queued on the mesh stream comes before later work on stream s.
static dg_status order_after_mesh(dg_mesh* m, cudaStream_t s) {
  if (s == m->stream) return DG_OK;
  if (!m->ev_order) CU(cudaEventCreateWithFlags(&m->ev_order, cudaEventDisableTiming));
  CU(cudaEventRecord(m->ev_order, m->stream));
  CU(cudaStreamWaitEvent(s, m->ev_order, 0));
  return DG_OK;
}

dg_status dg_set_state_async(dg_mesh* m, const void* q, int where, void* stream) {
  if (!m || !q || (where != DG_HOST && where != DG_DEVICE)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  dg_status st = order_after_mesh(m, s);
  if (st != DG_OK) return st;
  m->pp_valid = false;
  CU(cudaMemcpyAsync(m->q[0], q, (size_t)m->NV * plane(m) * m->tsize,
                     where == DG_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return DG_OK;
}

dg_status dg_get_state_async(dg_mesh* m, void* q, int where, void* stream) {
  if (!m || !q || (where != DG_HOST && where != DG_DEVICE)) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  dg_status st = order_after_mesh(m, s);
  if (st != DG_OK) return st;
  CU(cudaMemcpyAsync(q, m->q[0], (size_t)m->NV * plane(m) * m->tsize,
                     where == DG_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  return DG_OK;
}

dg_status dg_integrals_async(dg_mesh* m, double* out, void* stream) {
  if (!m || !out) return fail(m, DG_ERR_ARG, "bad argument");
  if (m->broken) return fail(m, DG_ERR_STATE, kBrokenMsg);
  if (m->nparts > 1) return whole_mesh_only(m, "dg_integrals_async");
  if (m->tracer) return fail(m, DG_ERR_UNSUPPORTED, "tracer meshes: use dg_integrals");
  if (!m->bgint_valid) {   // the background sums, once per topology (synchronous)
    double tmp[DG_NUM_INTEGRALS];
    dg_status st = dg_integrals(m, tmp);
    if (st != DG_OK && st != DG_ERR_STATE) return st;
  }
  cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
  dg_status st = order_after_mesh(m, s);
  if (st != DG_OK) return st;
  CU(cudaMemsetAsync(m->d_bad, 0, sizeof(int), s));
  CU(dgk::launch_integrals(m->prec, false, (int32_t)m->E, m->n1, m->D, m->d_elem, d_x(m), d_w(m), m->root_h,
                           m->d_bg, m->q[0], plane(m), m->ph, m->d_partial, m->d_bad, m->d_out, s));
  CU(dgk::launch_integrals_combine(m->d_out, m->d_bgint, m->d_bad, m->d_bgint + 6, s));
  CU(cudaMemcpyAsync(out, m->d_bgint + 6, 6 * sizeof(double), cudaMemcpyDefault, s));
  return DG_OK;
}

}  // extern "C"
