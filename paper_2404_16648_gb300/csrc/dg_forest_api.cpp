// Host-only forest entry points of the C ABI (no CUDA calls): the tree that dg_adapt uses.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "tree.hpp"

struct dg_forest {
  dgl::Forest f;
  std::vector<int32_t> conf, mort, bnd;
  void refresh() { f.face_lists(&conf, &mort, &bnd); }
};

extern "C" {

dg_status dg_forest_create_periodic(int32_t dim, const int32_t base[3], int32_t max_level,
                                    const int32_t periodic[3], dg_forest** out) {
  if (!out || !base || (dim != 2 && dim != 3) || max_level < 0 || max_level > DG_MAX_LEVEL)
    return DG_ERR_ARG;
  for (int a = 0; a < dim; ++a)
    if (base[a] < 1 || ((int64_t)base[a] << max_level) >= (1 << 19)) return DG_ERR_ARG;
  int b[3] = {base[0], base[1], dim == 3 ? base[2] : 1};
  int per[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) per[a] = periodic && periodic[a] ? 1 : 0;
  dg_forest* f = new (std::nothrow) dg_forest();
  if (!f) return DG_ERR_OOM;
  f->f = dgl::Forest(dim, b, max_level, per);
  f->refresh();
  *out = f;
  return DG_OK;
}

dg_status dg_forest_create(int32_t dim, const int32_t base[3], int32_t max_level, dg_forest** out) {
  return dg_forest_create_periodic(dim, base, max_level, nullptr, out);
}

void dg_forest_destroy(dg_forest* forest) { delete forest; }

int64_t dg_forest_size(const dg_forest* forest) { return forest ? forest->f.size() : 0; }

dg_status dg_forest_leaves(const dg_forest* forest, int32_t* out, size_t cap) {
  if (!forest || !out || cap < (size_t)forest->f.size() * 5) return DG_ERR_ARG;
  const auto& L = forest->f.leaves();
  for (size_t e = 0; e < L.size(); ++e) {
    out[e * 5] = forest->f.root_index(L[e]);
    out[e * 5 + 1] = L[e].level;
    for (int a = 0; a < 3; ++a) out[e * 5 + 2 + a] = L[e].c[a];
  }
  return DG_OK;
}

dg_status dg_forest_faces(const dg_forest* forest, int64_t counts[3], int32_t* conforming,
                          size_t cap_c, int32_t* mortars, size_t cap_m, int32_t* boundary,
                          size_t cap_b) {
  if (!forest || !counts) return DG_ERR_ARG;
  counts[0] = (int64_t)forest->conf.size() / 3;
  counts[1] = (int64_t)forest->mort.size() / 7;
  counts[2] = (int64_t)forest->bnd.size() / 3;
  if (conforming && cap_c >= (size_t)counts[0]) std::memcpy(conforming, forest->conf.data(), forest->conf.size() * 4);
  if (mortars && cap_m >= (size_t)counts[1]) std::memcpy(mortars, forest->mort.data(), forest->mort.size() * 4);
  if (boundary && cap_b >= (size_t)counts[2]) std::memcpy(boundary, forest->bnd.data(), forest->bnd.size() * 4);
  return DG_OK;
}

dg_status dg_forest_regrid(dg_forest* forest, const uint8_t* flags, int32_t buffer,
                           int32_t max_level, int32_t* transfer, size_t cap, int64_t* new_size) {
  if (!forest || !flags || buffer < 0) return DG_ERR_ARG;
  const int maxl = max_level < 0 ? forest->f.max_level() : max_level;
  if (maxl > forest->f.max_level()) return DG_ERR_ARG;
  std::vector<uint8_t> tag(flags, flags + forest->f.size());
  dgl::Forest nf;
  std::vector<dgl::TransferEntry> tmap;
  int64_t nr = 0, nc = 0;
  std::string err;
  if (!forest->f.regrid(tag, buffer, maxl, &nf, &tmap, &nr, &nc, &err)) return DG_ERR_STATE;
  forest->f = std::move(nf);
  forest->refresh();
  if (new_size) *new_size = forest->f.size();
  if (transfer && cap >= tmap.size() * 9) {
    for (size_t i = 0; i < tmap.size(); ++i) {
      transfer[i * 9] = tmap[i].kind;
      for (int k = 0; k < 8; ++k) transfer[i * 9 + 1 + k] = tmap[i].src[k];
    }
  }
  return DG_OK;
}

dg_status dg_forest_partition(const dg_forest* forest, int32_t nparts, int64_t* starts) {
  if (!forest || !starts || nparts < 1) return DG_ERR_ARG;
  std::vector<int64_t> st;
  forest->f.partition(nparts, &st);
  for (int p = 0; p <= nparts; ++p) starts[p] = st[p];
  return DG_OK;
}

dg_status dg_forest_halo(const dg_forest* forest, int32_t nparts, int32_t part, int32_t* rows,
                         size_t cap, int64_t* count) {
  if (!forest || !count || nparts < 1 || part < 0 || part >= nparts) return DG_ERR_ARG;
  std::vector<int64_t> st;
  forest->f.partition(nparts, &st);
  std::vector<int32_t> r;
  forest->f.halo(st, part, &r);
  *count = (int64_t)r.size() / 5;
  if (rows && cap >= r.size() / 5) std::memcpy(rows, r.data(), r.size() * sizeof(int32_t));
  return DG_OK;
}

}  // extern "C"
