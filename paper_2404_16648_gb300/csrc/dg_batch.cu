// Batched time stepping of many independent meshes (dg_batch_* entry points of include/dg.h).
//
// Meshes are grouped by (precision, dimension, N).  Per SSP-RK3 stage the batch makes one stage
// launch per group that covers every element of every member: the per-member launch arguments
// live in a device table and each CTA reads its member index and first element from a block
// map.  Hanging faces keep their per-member mortar launches.  A whole step (three stages, all
// groups) is captured once into a CUDA graph and replayed; dg_batch_autotune times the two
// column and node layouts of each group on the members themselves and keeps the faster one.
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dg_mesh.hpp"

struct dg_batch {
  struct Group {
    int prec = 0, D = 2, N = 1, layout = 2;
    std::vector<int> members;
    int nblocks[3] = {0, 0, 0};          // per layout (index 1 node, 2 async)
    int2* d_map[3] = {nullptr, nullptr, nullptr};
    dgk::StageArgs* d_tab[3] = {nullptr, nullptr, nullptr};   // per stage
  };
  std::vector<dg_mesh*> meshes;
  std::vector<int64_t> elements;         // element counts when the batch was built
  std::vector<int64_t> generations;      // regrid generations when the batch was built
  std::vector<double> dt;
  std::vector<Group> groups;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool tables_dirty = true;
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
  b->tables_dirty = false;
  return DG_OK;
}

dg_status one_step(dg_batch* b, cudaStream_t s) {
  for (int st = 0; st < 3; ++st) {
    for (auto& g : b->groups) {
      for (int idx : g.members) {
        dg_mesh* m = b->meshes[idx];
        const void* qs; void* pp_in; void* out; void* pp_out; double ca, cb;
        stage_buffers(m, st, &qs, &pp_in, &out, &pp_out, &ca, &cb);
        dg_status r = dgi::launch_mortars(m, qs, pp_in, s);
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

}  // namespace

extern "C" {

dg_status dg_batch_create(dg_mesh* const* meshes, int32_t count, dg_batch** out) {
  if (!meshes || count <= 0 || !out) return DG_ERR_ARG;
  *out = nullptr;
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ERR_OOM;
  std::map<std::tuple<int, int, int>, int> gid;
  for (int32_t i = 0; i < count; ++i) {
    dg_mesh* m = meshes[i];
    if (!m) { delete b; return DG_ERR_ARG; }
    if (m->broken) { delete b; return DG_ERR_STATE; }   // a regrid of this mesh failed after its commit
    if (m->desc.nu > 0.0 || m->tracer) { delete b; return DG_ERR_UNSUPPORTED; }   // inviscid Euler only
    for (int32_t j = 0; j < i; ++j)
      if (meshes[j] == m) { delete b; return DG_ERR_ARG; }   // each mesh once
    b->meshes.push_back(m);
    b->elements.push_back(m->E);
    b->generations.push_back(m->generation);
    b->dt.push_back(0.0);
    auto key = std::make_tuple(m->prec, m->D, m->N);
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
  dg_status st = DG_OK;
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
  (void)st;
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
  return DG_OK;
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
    dg_status st = dgi::ensure_pp(m, b->stream);
    if (st != DG_OK) return bfail(b, st, m->err);
  }
  cudaEvent_t e0, e1;
  BCU(cudaEventCreate(&e0));
  BCU(cudaEventCreate(&e1));
  for (auto& g : b->groups) {
    // stage 0 reads q^n and writes the scratch stage buffer, so timing it leaves the states alone
    for (int idx : g.members) {
      dg_mesh* m = b->meshes[idx];
      dg_status st = dgi::launch_mortars(m, m->q[0], dgi::pp_plane(m, m->q[0]), b->stream);
      if (st != DG_OK) return bfail(b, st, m->err);
    }
    float best = 1e30f;
    int best_layout = g.layout;
    for (int layout = 1; layout <= 2; ++layout) {
      BCU(launch_group(g, 0, layout, b->stream));          // warm-up
      BCU(cudaEventRecord(e0, b->stream));
      for (int r = 0; r < reps; ++r) BCU(launch_group(g, 0, layout, b->stream));
      BCU(cudaEventRecord(e1, b->stream));
      BCU(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCU(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; best_layout = layout; }
    }
    g.layout = best_layout;
    for (int idx : g.members) b->meshes[idx]->variant = best_layout;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(b);
  if (layouts)
    for (auto& g : b->groups)
      for (int idx : g.members) layouts[idx] = g.layout;
  return DG_OK;
}

const char* dg_batch_last_error(const dg_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
