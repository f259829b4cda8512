// Batched time stepping of many independent meshes (dg_batch_* entry points of include/dg.h).
//
// 2D members run through one persistent launch per SSP-RK3 stage (dg_batch_persist.cuh): a
// device array of work items -- the mortar groups of every member, then tiles of elements of
// every member, whatever its N and precision -- taken in order by a grid sized to what stays
// resident.  3D members are grouped by (precision, N) and run one stage launch per group over
// all of its members' elements (per-block member map) after their members' mortar launches.
// A whole step is captured once into a CUDA graph and replayed.
//
// dg_batch_autotune chooses the persistent launch's shapes on the members themselves (timing
// stage 1, which reads q^n and writes only scratch): the register budget (2 or 4 resident CTAs
// of 128 threads per SM), per (precision, N) group the element tile (node layout: (N+1)^2
// threads per element, 128 / (N+1)^2 elements per CTA pass; column layout: N+1 threads per
// element, 128 / (N+1) elements per pass; for FP64 groups also the column layout that reads the
// conforming and wall fluxes from face items of the same launch, stage layout 5) and the tiles
// per work item; for 3D groups the faster of the two grouped layouts.
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dg_batch_persist.cuh"
#include "dg_mesh.hpp"

struct dg_batch {
  // 3D members: one grouped launch per (precision, N) group and stage
  struct Group {
    int prec = 0, D = 2, N = 1, layout = 2;
    std::vector<int> members;
    int nblocks[3] = {0, 0, 0};          // per layout (index 1 node, 2 async)
    int2* d_map[3] = {nullptr, nullptr, nullptr};
    dgk::StageArgs* d_tab[3] = {nullptr, nullptr, nullptr};   // per stage
  };
  // 2D members: the persistent launch; layout 0 node, 1 column-async, 2 column-async with the
  // face buffer (stage layout 5, FP64 only)
  struct PGroup {
    int prec32 = 0, N = 1, layout = 1;
    std::vector<int> members;
  };
  std::vector<dg_mesh*> meshes;
  std::vector<int64_t> elements;         // element counts when the batch was built
  std::vector<int64_t> generations;      // regrid generations when the batch was built
  std::vector<double> dt;
  std::vector<Group> groups;
  std::vector<PGroup> pgroups;
  int minb = 2;                          // register budget: 2 or 4 resident CTAs per SM
  int tiles_per_item = 2;                // element tiles per stage item
  int nitems = 0, grid = 0;
  size_t smem = 0;
  int4* d_items = nullptr;
  size_t items_cap = 0;
  dgk::StageArgs* d_ptab[3] = {nullptr, nullptr, nullptr};   // per stage, per member
  dgk::MortarArgs* d_mtab[3] = {nullptr, nullptr, nullptr};
  dgk::FaceArgs* d_ftab[3] = {nullptr, nullptr, nullptr};
  int32_t* d_need = nullptr;             // per member: mortar groups, plus face slots in layout 5
  int32_t* d_counters = nullptr;         // [3][1 + members]: item counter, mortar groups done
  int32_t* d_status = nullptr;           // 1 after a wait for mortar fluxes ran out
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool tables_dirty = true;
  bool items_dirty = true;
  std::string err;
};

namespace {

dg_status bfail(dg_batch* b, dg_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BCU(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return bfail(b, e_ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, \
                                        std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaError_t launch_group(const dg_batch::Group& g, int stage, int layout, cudaStream_t s) {
  const dgk::StageArgs* tab = g.d_tab[stage];
  const int2* map = g.d_map[layout];
  const int nb = g.nblocks[layout];
  if (g.prec == DG_FP64)
    return g.D == 2 ? dgk::launch_stage_batched_f64_2d(g.N, layout, tab, map, nb, s)
                    : dgk::launch_stage_batched_f64_3d(g.N, layout, tab, map, nb, s);
  return g.D == 2 ? dgk::launch_stage_batched_f32_2d(g.N, layout, tab, map, nb, s)
                  : dgk::launch_stage_batched_f32_3d(g.N, layout, tab, map, nb, s);
}

// Shu-Osher stage s of every member: inputs and outputs in the members' own state buffers.
void stage_buffers(dg_mesh* m, int s, const void** qs, void** pp_in, void** out, void** pp_out,
                   double* ca, double* cb) {
  void* q0 = m->q[0];
  void* q1 = m->q[1];
  void* q2 = m->q[2];
  if (s == 0) { *qs = q0; *out = q1; *ca = 0.0; *cb = 1.0; }
  else if (s == 1) { *qs = q1; *out = q2; *ca = 0.75; *cb = 0.25; }
  else { *qs = q2; *out = q0; *ca = 1.0 / 3.0; *cb = 2.0 / 3.0; }
  *pp_in = dgi::pp_plane(m, const_cast<void*>(*qs));
  *pp_out = dgi::pp_plane(m, *out);
}

// Elements of one tile of a 2D group's layout (one pass of its body in a 128-thread CTA).
int tile_elems(const dg_batch::PGroup& g) {
  return g.layout == 0 ? dgk::batch_epb_node(g.N) : dgk::batch_epb_col(g.N);
}

// Face slots (conforming, then boundary faces) of a layout-5 member.
int64_t face_slots(const dg_mesh* m) { return (int64_t)(m->conf.size() / 3 + m->bnd.size() / 3); }

// The single-mesh stage layout of a 2D group's layout.
int stage_layout(int glayout) { return glayout == 0 ? 1 : (glayout == 1 ? 2 : 5); }

// The work items of the persistent launch for the current shapes (the same list serves the
// three stages), the launch's shared memory and its grid.
dg_status build_items(dg_batch* b) {
  std::vector<int4> items;
  size_t smem = 0;
  // mortar items first: two passes of groups each
  for (const auto& g : b->pgroups) {
    const int per = 2 * dgk::batch_gpb(g.N);
    bool any = false;
    for (int idx : g.members) {
      const int64_t G = b->meshes[idx]->G;
      for (int64_t f = 0; f < G; f += per)
        items.push_back(make_int4(dgk::batch_code(0, 0, g.prec32, g.N), idx, (int)f, (int)std::min<int64_t>(per, G - f)));
      any = any || G > 0;
    }
    if (any) smem = std::max(smem, dgk::batch_body_smem_bytes(g.prec32, g.N, 2));
  }
  // then the face items of layout-5 members: four passes of slots each
  std::vector<int32_t> need(b->meshes.size(), 0);
  for (size_t i = 0; i < b->meshes.size(); ++i) need[i] = b->meshes[i]->D == 2 ? (int32_t)b->meshes[i]->G : 0;
  for (const auto& g : b->pgroups) {
    if (g.layout != 2) continue;
    const int per = 4 * dgk::batch_fpb(g.N);
    for (int idx : g.members) {
      const int64_t F = face_slots(b->meshes[idx]);
      for (int64_t f = 0; f < F; f += per)
        items.push_back(make_int4(dgk::batch_code(2, 2, 0, g.N), idx, (int)f, (int)std::min<int64_t>(per, F - f)));
      need[idx] += (int32_t)F;
    }
  }
  // stage items, the groups with the most work per element first
  std::vector<const dg_batch::PGroup*> order;
  for (const auto& g : b->pgroups) order.push_back(&g);
  std::stable_sort(order.begin(), order.end(), [](const dg_batch::PGroup* x, const dg_batch::PGroup* y) {
    const double cx = (x->prec32 ? 1.0 : 4.0) * (x->N + 1), cy = (y->prec32 ? 1.0 : 4.0) * (y->N + 1);
    return cx > cy;
  });
  for (const dg_batch::PGroup* g : order) {
    const int per = tile_elems(*g) * b->tiles_per_item;
    for (int idx : g->members) {
      const int64_t E = b->meshes[idx]->E;
      for (int64_t e = 0; e < E; e += per)
        items.push_back(make_int4(dgk::batch_code(1, g->layout, g->prec32, g->N), idx, (int)e,
                                  (int)std::min<int64_t>(per, E - e)));
    }
    smem = std::max(smem, dgk::batch_body_smem_bytes(g->prec32, g->N, g->layout == 2 ? 3 : g->layout));
  }
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    BCU(cudaMalloc(&b->d_items, items.size() * sizeof(int4)));
    b->items_cap = items.size();
  }
  if (!items.empty())
    BCU(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  b->nitems = (int)items.size();
  b->smem = smem;
  int per_sm = 0, dev = 0, sms = 0;
  BCU(b->minb == 2 ? dgk::occupancy_batch_w(smem, &per_sm) : dgk::occupancy_batch_d(smem, &per_sm));
  BCU(cudaGetDevice(&dev));
  BCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return bfail(b, DG_ERR_UNSUPPORTED, "persistent batch kernel does not fit an SM");
  b->grid = std::min(per_sm * sms, std::max(1, b->nitems));
  b->items_dirty = false;
  return DG_OK;
}

dg_status build_tables(dg_batch* b) {
  for (auto& g : b->groups) {
    for (int s = 0; s < 3; ++s) {
      std::vector<dgk::StageArgs> tab(g.members.size());
      for (size_t k = 0; k < g.members.size(); ++k) {
        dg_mesh* m = b->meshes[g.members[k]];
        const void* qs; void* pp_in; void* out; void* pp_out; double ca, cb;
        stage_buffers(m, s, &qs, &pp_in, &out, &pp_out, &ca, &cb);
        dgi::fill_stage_args(m, qs, pp_in, m->q[0], out, pp_out, 1, b->dt[g.members[k]], ca, cb, &tab[k]);
      }
      if (!g.d_tab[s]) BCU(cudaMalloc(&g.d_tab[s], tab.size() * sizeof(dgk::StageArgs)));
      BCU(cudaMemcpy(g.d_tab[s], tab.data(), tab.size() * sizeof(dgk::StageArgs), cudaMemcpyHostToDevice));
    }
  }
  if (!b->pgroups.empty()) {
    const size_t M = b->meshes.size();
    for (int s = 0; s < 3; ++s) {
      std::vector<dgk::StageArgs> tab(M);
      std::vector<dgk::MortarArgs> mt(M);
      std::vector<dgk::FaceArgs> ft(M);
      for (size_t i = 0; i < M; ++i) {
        dg_mesh* m = b->meshes[i];
        if (m->D != 2) continue;
        // every FP64 member gets its face buffer, so that the autotuner may pick layout 5
        if (m->prec == DG_FP64) {
          dg_status st = dgi::ensure_face_buffer(m);
          if (st != DG_OK) return bfail(b, st, m->err);
        }
        const void* qs; void* pp_in; void* out; void* pp_out; double ca, cb;
        stage_buffers(m, s, &qs, &pp_in, &out, &pp_out, &ca, &cb);
        dgi::fill_stage_args(m, qs, pp_in, m->q[0], out, pp_out, 1, b->dt[i], ca, cb, &tab[i]);
        dgi::fill_mortar_args(m, qs, pp_in, &mt[i]);
        dgi::fill_face_args(m, qs, pp_in, &ft[i]);
      }
      if (!b->d_ptab[s]) BCU(cudaMalloc(&b->d_ptab[s], M * sizeof(dgk::StageArgs)));
      if (!b->d_mtab[s]) BCU(cudaMalloc(&b->d_mtab[s], M * sizeof(dgk::MortarArgs)));
      if (!b->d_ftab[s]) BCU(cudaMalloc(&b->d_ftab[s], M * sizeof(dgk::FaceArgs)));
      BCU(cudaMemcpy(b->d_ptab[s], tab.data(), M * sizeof(dgk::StageArgs), cudaMemcpyHostToDevice));
      BCU(cudaMemcpy(b->d_mtab[s], mt.data(), M * sizeof(dgk::MortarArgs), cudaMemcpyHostToDevice));
      BCU(cudaMemcpy(b->d_ftab[s], ft.data(), M * sizeof(dgk::FaceArgs), cudaMemcpyHostToDevice));
    }
  }
  b->tables_dirty = false;
  return DG_OK;
}

// The persistent launch of stage `st` over the 2D members (the stage's counters must be zero).
dg_status launch_persistent(dg_batch* b, int st, cudaStream_t s) {
  if (b->pgroups.empty()) return DG_OK;
  const size_t M = b->meshes.size();
  dgk::BatchArgs B{};
  B.items = b->d_items;
  B.nitems = b->nitems;
  B.stage = b->d_ptab[st];
  B.mortar = b->d_mtab[st];
  B.face = b->d_ftab[st];
  B.need = b->d_need;
  B.fetch = b->d_counters + (size_t)st * (1 + M);
  B.done = B.fetch + 1;
  B.status = b->d_status;
  BCU(b->minb == 2 ? dgk::launch_batch_w(B, b->grid, b->smem, s) : dgk::launch_batch_d(B, b->grid, b->smem, s));
  return DG_OK;
}

dg_status zero_counters(dg_batch* b, cudaStream_t s) {
  if (b->pgroups.empty()) return DG_OK;
  BCU(cudaMemsetAsync(b->d_counters, 0, 3 * (1 + b->meshes.size()) * sizeof(int32_t), s));
  return DG_OK;
}

dg_status one_step(dg_batch* b, cudaStream_t s) {
  dg_status r = zero_counters(b, s);
  if (r != DG_OK) return r;
  for (int st = 0; st < 3; ++st) {
    r = launch_persistent(b, st, s);
    if (r != DG_OK) return r;
    for (auto& g : b->groups) {
      for (int idx : g.members) {
        dg_mesh* m = b->meshes[idx];
        const void* qs; void* pp_in; void* out; void* pp_out; double ca, cb;
        stage_buffers(m, st, &qs, &pp_in, &out, &pp_out, &ca, &cb);
        r = dgi::launch_mortars(m, qs, pp_in, s);
        if (r != DG_OK) return bfail(b, r, m->err);
      }
      BCU(launch_group(g, st, g.layout, s));
    }
  }
  return DG_OK;
}

void drop_graph(dg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

// DG_ERR_TIMEOUT (and a cleared flag) when a wait for mortar fluxes ran out; the stream must be
// idle.
dg_status check_status(dg_batch* b) {
  if (!b->d_status) return DG_OK;
  int32_t st = 0;
  BCU(cudaMemcpy(&st, b->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st == 0) return DG_OK;
  BCU(cudaMemset(b->d_status, 0, sizeof(int32_t)));
  return bfail(b, DG_ERR_TIMEOUT, "a wait for mortar fluxes in the persistent batch kernel ran out; "
                                  "the batch's states are not valid");
}

// Time of `reps` stage-1 persistent launches (the states are left alone: stage 1 writes the
// scratch stage buffer and the mortar buffers only).
dg_status time_persistent(dg_batch* b, int reps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  dg_status r = build_items(b);
  if (r != DG_OK) return r;
  const size_t M = b->meshes.size();
  auto one = [&]() -> dg_status {
    BCU(cudaMemsetAsync(b->d_counters, 0, (1 + M) * sizeof(int32_t), b->stream));
    return launch_persistent(b, 0, b->stream);
  };
  r = one();   // warm-up
  if (r != DG_OK) return r;
  BCU(cudaEventRecord(e0, b->stream));
  for (int i = 0; i < reps; ++i) {
    r = one();
    if (r != DG_OK) return r;
  }
  BCU(cudaEventRecord(e1, b->stream));
  BCU(cudaEventSynchronize(e1));
  BCU(cudaEventElapsedTime(ms, e0, e1));
  return check_status(b);
}

}  // namespace

extern "C" {

dg_status dg_batch_create(dg_mesh* const* meshes, int32_t count, dg_batch** out) {
  if (!meshes || count <= 0 || !out) return DG_ERR_ARG;
  *out = nullptr;
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ERR_OOM;
  std::map<std::tuple<int, int, int>, int> gid, pid;
  for (int32_t i = 0; i < count; ++i) {
    dg_mesh* m = meshes[i];
    if (!m) { delete b; return DG_ERR_ARG; }
    if (m->broken) { delete b; return DG_ERR_STATE; }   // a regrid of this mesh failed after its commit
    if (m->nparts > 1) { delete b; return DG_ERR_UNSUPPORTED; }   // a batch member is a whole mesh
    if (m->desc.nu > 0.0 || m->tracer) { delete b; return DG_ERR_UNSUPPORTED; }   // inviscid Euler only
    for (int32_t j = 0; j < i; ++j)
      if (meshes[j] == m) { delete b; return DG_ERR_ARG; }   // each mesh once
    b->meshes.push_back(m);
    b->elements.push_back(m->E);
    b->generations.push_back(m->generation);
    b->dt.push_back(0.0);
    auto key = std::make_tuple(m->prec, m->D, m->N);
    // the persistent launch has the face-buffer layout for FP64 members only: an FP32 member set
    // to it runs the column layout, in the batch and in its own launches alike
    if (m->D == 2 && m->prec != DG_FP64 && m->variant == 5) m->variant = 2;
    if (m->D == 2) {
      auto it = pid.find(key);
      if (it == pid.end()) {
        dg_batch::PGroup g;
        g.prec32 = m->prec == DG_FP32_PERT ? 1 : 0; g.N = m->N;
        g.layout = m->variant == 1 ? 0 : (m->variant == 5 && g.prec32 == 0 ? 2 : 1);
        pid[key] = (int)b->pgroups.size();
        b->pgroups.push_back(g);
        it = pid.find(key);
      }
      b->pgroups[it->second].members.push_back(i);
      continue;
    }
    auto it = gid.find(key);
    if (it == gid.end()) {
      dg_batch::Group g;
      g.prec = m->prec; g.D = m->D; g.N = m->N;
      g.layout = m->variant == 1 ? 1 : 2;
      gid[key] = (int)b->groups.size();
      b->groups.push_back(g);
      it = gid.find(key);
    }
    b->groups[it->second].members.push_back(i);
  }
  auto cleanup = [&](dg_status r) { dg_batch_destroy(b); return r; };
  if (cudaStreamCreate(&b->stream) != cudaSuccess || cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(DG_ERR_CUDA);
  for (auto& g : b->groups) {
    for (int layout = 1; layout <= 2; ++layout) {
      const int epb = layout == 1 ? dgk::epb_node(g.D, g.N) : dgk::epb_col(g.D, g.N);
      std::vector<int2> map;
      for (size_t k = 0; k < g.members.size(); ++k) {
        const int64_t E = b->meshes[g.members[k]]->E;
        for (int64_t e = 0; e < E; e += epb) map.push_back(make_int2((int)k, (int)e));
      }
      g.nblocks[layout] = (int)map.size();
      if (cudaMalloc(&g.d_map[layout], std::max<size_t>(1, map.size()) * sizeof(int2)) != cudaSuccess)
        return cleanup(DG_ERR_OOM);
      if (!map.empty() && cudaMemcpy(g.d_map[layout], map.data(), map.size() * sizeof(int2),
                                     cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(DG_ERR_CUDA);
    }
  }
  if (!b->pgroups.empty()) {
    const size_t M = b->meshes.size();
    if (cudaMalloc(&b->d_need, M * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&b->d_counters, 3 * (1 + M) * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&b->d_status, sizeof(int32_t)) != cudaSuccess)
      return cleanup(DG_ERR_OOM);
    if (cudaMemset(b->d_status, 0, sizeof(int32_t)) != cudaSuccess) return cleanup(DG_ERR_CUDA);
  }
  *out = b;
  return DG_OK;
}

void dg_batch_destroy(dg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& g : b->groups) {
    for (int i = 0; i < 3; ++i) { if (g.d_map[i]) cudaFree(g.d_map[i]); if (g.d_tab[i]) cudaFree(g.d_tab[i]); }
  }
  for (int s = 0; s < 3; ++s) {
    if (b->d_ptab[s]) cudaFree(b->d_ptab[s]);
    if (b->d_mtab[s]) cudaFree(b->d_mtab[s]);
    if (b->d_ftab[s]) cudaFree(b->d_ftab[s]);
  }
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_need) cudaFree(b->d_need);
  if (b->d_counters) cudaFree(b->d_counters);
  if (b->d_status) cudaFree(b->d_status);
  if (b->done) cudaEventDestroy(b->done);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

dg_status dg_batch_set_dt(dg_batch* b, const double* dt) {
  if (!b || !dt) return DG_ERR_ARG;
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    if (!(dt[i] > 0.0)) return bfail(b, DG_ERR_ARG, "every dt must be positive");
    b->dt[i] = dt[i];
  }
  b->tables_dirty = true;
  drop_graph(b);
  return DG_OK;
}

dg_status dg_batch_run(dg_batch* b, int32_t nsteps, int32_t use_graph) {
  if (!b || nsteps < 0) return DG_ERR_ARG;
  for (size_t i = 0; i < b->meshes.size(); ++i) {
    if (b->meshes[i]->broken || b->meshes[i]->E != b->elements[i] || b->meshes[i]->generation != b->generations[i])
      return bfail(b, DG_ERR_STATE, "a mesh was regridded after dg_batch_create");
    if (!(b->dt[i] > 0.0)) return bfail(b, DG_ERR_ARG, "dt not set (dg_batch_set_dt)");
  }
  if (b->tables_dirty) {
    drop_graph(b);
    dg_status st = build_tables(b);
    if (st != DG_OK) return st;
  }
  if (b->items_dirty && !b->pgroups.empty()) {
    drop_graph(b);
    dg_status st = build_items(b);
    if (st != DG_OK) return st;
  }
  // order after work queued on each member's stream, and bring P' of every state up to date
  for (dg_mesh* m : b->meshes) {
    BCU(cudaEventRecord(b->done, m->stream));
    BCU(cudaStreamWaitEvent(b->stream, b->done, 0));
    dg_status st = dgi::ensure_pp(m, b->stream);
    if (st != DG_OK) return bfail(b, st, m->err);
  }
  if (use_graph && nsteps > 0) {
    if (!b->exec) {
      // configure kernel attributes outside the capture
      for (auto& g : b->groups) {
        const int nb = g.nblocks[g.layout];
        g.nblocks[g.layout] = 0;
        cudaError_t e = launch_group(g, 0, g.layout, b->stream);
        g.nblocks[g.layout] = nb;
        BCU(e);
      }
      if (!b->pgroups.empty()) {
        int per_sm = 0;
        BCU(b->minb == 2 ? dgk::occupancy_batch_w(b->smem, &per_sm) : dgk::occupancy_batch_d(b->smem, &per_sm));
      }
      cudaGraph_t graph = nullptr;
      BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      dg_status st = one_step(b, b->stream);
      cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
      if (st != DG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
      BCU(e);
      e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      BCU(e);
    }
    for (int32_t i = 0; i < nsteps; ++i) BCU(cudaGraphLaunch(b->exec, b->stream));
  } else {
    for (int32_t i = 0; i < nsteps; ++i) {
      dg_status st = one_step(b, b->stream);
      if (st != DG_OK) return st;
    }
  }
  // later work on each member's stream waits for the batch
  BCU(cudaEventRecord(b->done, b->stream));
  for (dg_mesh* m : b->meshes) BCU(cudaStreamWaitEvent(m->stream, b->done, 0));
  return DG_OK;
}

dg_status dg_batch_sync(dg_batch* b) {
  if (!b) return DG_ERR_ARG;
  BCU(cudaStreamSynchronize(b->stream));
  return check_status(b);
}

dg_status dg_batch_autotune(dg_batch* b, int32_t reps, int32_t* layouts) {
  if (!b || reps <= 0) return DG_ERR_ARG;
  for (size_t i = 0; i < b->meshes.size(); ++i)
    if (!(b->dt[i] > 0.0)) return bfail(b, DG_ERR_ARG, "dt not set (dg_batch_set_dt)");
  if (b->tables_dirty) {
    dg_status st = build_tables(b);
    if (st != DG_OK) return st;
  }
  for (dg_mesh* m : b->meshes) {
    BCU(cudaEventRecord(b->done, m->stream));
    BCU(cudaStreamWaitEvent(b->stream, b->done, 0));
    dg_status st = dgi::ensure_pp(m, b->stream);
    if (st != DG_OK) return bfail(b, st, m->err);
  }
  cudaEvent_t e0, e1;
  BCU(cudaEventCreate(&e0));
  BCU(cudaEventCreate(&e1));
  auto finish = [&](dg_status r) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; };
  // 3D groups: the faster of the two grouped layouts on stage 1 (reads q^n, writes scratch)
  for (auto& g : b->groups) {
    for (int idx : g.members) {
      dg_mesh* m = b->meshes[idx];
      dg_status st = dgi::launch_mortars(m, m->q[0], dgi::pp_plane(m, m->q[0]), b->stream);
      if (st != DG_OK) return finish(bfail(b, st, m->err));
    }
    float best = 1e30f;
    int best_layout = g.layout;
    for (int layout = 1; layout <= 2; ++layout) {
      cudaError_t e = launch_group(g, 0, layout, b->stream);          // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_group(g, 0, layout, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) return finish(bfail(b, DG_ERR_CUDA, cudaGetErrorString(e)));
      if (ms < best) { best = ms; best_layout = layout; }
    }
    g.layout = best_layout;
    for (int idx : g.members) b->meshes[idx]->variant = best_layout;
  }
  // 2D members: the persistent launch's register budget, per group the element tile, and the
  // tiles per item -- greedy, groups with the most work first
  if (!b->pgroups.empty()) {
    std::vector<size_t> order(b->pgroups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    auto work = [&](const dg_batch::PGroup& g) {
      double w = 0.0;
      for (int idx : g.members) w += (double)b->meshes[idx]->E * (g.N + 1) * (g.N + 1);
      return w * (g.prec32 ? 1.0 : 4.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work(b->pgroups[x]) > work(b->pgroups[y]); });
    float best_all = 1e30f;
    int best_minb = b->minb, best_k = b->tiles_per_item;
    std::vector<int> best_layouts(b->pgroups.size());
    for (int minb : {2, 4}) {
      b->minb = minb;
      b->tiles_per_item = 2;
      for (auto& g : b->pgroups) g.layout = 1;
      float cur = 0.f;
      dg_status st = time_persistent(b, reps, e0, e1, &cur);
      if (st != DG_OK) return finish(st);
      for (size_t oi : order) {
        auto& g = b->pgroups[oi];
        const int keep = g.layout;
        int bestl = keep;
        for (int cand : {0, 1, 2}) {
          if (cand == keep || (cand == 2 && g.prec32)) continue;
          g.layout = cand;
          float t = 0.f;
          st = time_persistent(b, reps, e0, e1, &t);
          if (st != DG_OK) return finish(st);
          if (t < cur) { cur = t; bestl = cand; }
        }
        g.layout = bestl;
      }
      int kbest = b->tiles_per_item;
      for (int k : {1, 4, 8}) {
        b->tiles_per_item = k;
        float t = 0.f;
        st = time_persistent(b, reps, e0, e1, &t);
        if (st != DG_OK) return finish(st);
        if (t < cur) { cur = t; kbest = k; }
      }
      if (cur < best_all) {
        best_all = cur;
        best_minb = minb;
        best_k = kbest;
        for (size_t i = 0; i < b->pgroups.size(); ++i) best_layouts[i] = b->pgroups[i].layout;
      }
    }
    b->minb = best_minb;
    b->tiles_per_item = best_k;
    for (size_t i = 0; i < b->pgroups.size(); ++i) {
      b->pgroups[i].layout = best_layouts[i];
      for (int idx : b->pgroups[i].members) b->meshes[idx]->variant = stage_layout(best_layouts[i]);
    }
    b->items_dirty = true;
  }
  drop_graph(b);
  if (layouts) {
    for (auto& g : b->groups)
      for (int idx : g.members) layouts[idx] = g.layout;
    for (auto& g : b->pgroups)
      for (int idx : g.members) layouts[idx] = stage_layout(g.layout);
  }
  return finish(DG_OK);
}

// The persistent launch's shapes: out[0] register budget (resident CTAs per SM it is compiled
// for), out[1] tiles per stage item, out[2] grid, out[3] items per stage, out[4] dynamic shared
// memory in bytes.  Zeros when the batch has no 2D member.
dg_status dg_batch_shape(dg_batch* b, int64_t out[5]) {
  if (!b || !out) return DG_ERR_ARG;
  for (int i = 0; i < 5; ++i) out[i] = 0;
  if (b->pgroups.empty()) return DG_OK;
  if (b->items_dirty) {
    dg_status st = build_items(b);
    if (st != DG_OK) return st;
    drop_graph(b);
  }
  out[0] = b->minb; out[1] = b->tiles_per_item; out[2] = b->grid; out[3] = b->nitems; out[4] = (int64_t)b->smem;
  return DG_OK;
}

const char* dg_batch_last_error(const dg_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
