// Host forest: leaf order, neighbour classification, regrid with buffer and 2:1 closure,
// canonical face lists and the per-element connectivity table used by the device kernels.
#include "tree.hpp"

#include <algorithm>
#include <atomic>

#include "host_pool.hpp"

namespace dgl {

uint64_t Forest::key(int level, const int32_t c[3]) {
  return (uint64_t)(uint32_t)level | ((uint64_t)(uint32_t)c[0] << 5) |
         ((uint64_t)(uint32_t)c[1] << 24) | ((uint64_t)(uint32_t)c[2] << 43);
}

Forest::Forest(int dim, const int base[3], int max_level, const int periodic[3])
    : dim_(dim), max_level_(max_level) {
  for (int a = 0; a < 3; ++a) base_[a] = (a < dim) ? base[a] : 1;
  for (int a = 0; a < 3; ++a) periodic_[a] = (periodic && a < dim && periodic[a]) ? 1 : 0;
  std::vector<Leaf> roots;
  for (int z = 0; z < base_[2]; ++z)
    for (int y = 0; y < base_[1]; ++y)
      for (int x = 0; x < base_[0]; ++x) roots.push_back(Leaf{0, {x, y, z}});
  set_leaves(std::move(roots));
}

static uint64_t mix64(uint64_t x) {   // splitmix64 finaliser
  x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ULL;
  x ^= x >> 27; x *= 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}
static constexpr uint64_t kEmpty = ~0ULL;   // never a key: levels < 32, coordinates < 2^19

void Forest::set_leaves(std::vector<Leaf> leaves) {
  leaves_ = std::move(leaves);
  uint64_t cap = 16;
  while (cap < 2 * (uint64_t)leaves_.size()) cap <<= 1;
  hkeys_.assign(cap, kEmpty);
  hvals_.assign(cap, -1);
  hmask_ = cap - 1;
  // leaves are distinct, so each key claims one slot; concurrent inserts claim slots with a
  // compare-and-swap, and where a key lands depends on the order of inserts but find() returns
  // the same leaf either way
  uint64_t* K = hkeys_.data();
  int32_t* V = hvals_.data();
  parallel_ranges((int64_t)leaves_.size(), 4096, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const uint64_t k = key(leaves_[i].level, leaves_[i].c);
      uint64_t h = mix64(k) & hmask_;
      for (;;) {
        uint64_t seen = kEmpty;
        if (__atomic_compare_exchange_n(&K[h], &seen, k, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED) ||
            seen == k) {
          V[h] = (int32_t)i;
          break;
        }
        h = (h + 1) & hmask_;
      }
    }
  });
  // face table; every entry depends on its own face only
  const int64_t n = (int64_t)leaves_.size();
  faces_.assign((size_t)n * dim_ * 2, FaceInfo{FACE_WALL, {-1, -1, -1, -1}});
  parallel_ranges(n, 512, [this](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      for (int a = 0; a < dim_; ++a)
        for (int s = 0; s < 2; ++s) faces_[((size_t)e * dim_ + a) * 2 + s] = classify((int32_t)e, a, s);
  });
}

int32_t Forest::root_index(const Leaf& l) const {
  int32_t r[3];
  for (int a = 0; a < 3; ++a) r[a] = l.c[a] >> l.level;
  return r[0] + base_[0] * (r[1] + base_[1] * r[2]);
}

int32_t Forest::find(int level, const int32_t c[3]) const {
  if (level < 0 || hkeys_.empty()) return -1;
  const uint64_t k = key(level, c);
  uint64_t h = mix64(k) & hmask_;
  while (hkeys_[h] != kEmpty) {
    if (hkeys_[h] == k) return hvals_[h];
    h = (h + 1) & hmask_;
  }
  return -1;
}

FaceInfo Forest::classify(int32_t e, int axis, int side) const {
  FaceInfo fi{FACE_WALL, {-1, -1, -1, -1}};
  const Leaf& L = leaves_[e];
  int32_t n[3] = {L.c[0], L.c[1], L.c[2]};
  n[axis] += side ? 1 : -1;
  const int32_t ext = extent(L.level, axis);
  if (n[axis] < 0 || n[axis] >= ext) {
    if (!periodic_[axis]) return fi;
    n[axis] = (n[axis] + ext) % ext;
  }
  int32_t idx = find(L.level, n);
  if (idx >= 0) { fi.kind = FACE_CONF; fi.nb[0] = idx; return fi; }
  if (L.level > 0) {
    int32_t p[3] = {n[0] >> 1, n[1] >> 1, n[2] >> 1};
    idx = find(L.level - 1, p);
    if (idx >= 0) { fi.kind = FACE_FINE; fi.nb[0] = idx; return fi; }
  }
  // refined neighbour: 2^(d-1) children touching this face, Morton over tangential axes
  fi.kind = FACE_COARSE;
  int tang[2], nt = 0;
  for (int a = 0; a < dim_; ++a) if (a != axis) tang[nt++] = a;
  for (int bits = 0; bits < (1 << (dim_ - 1)); ++bits) {
    int32_t cc[3] = {2 * n[0], 2 * n[1], 2 * n[2]};
    if (dim_ < 3) cc[2] = 0;
    cc[axis] += side ? 0 : 1;
    for (int t = 0; t < nt; ++t) cc[tang[t]] += (bits >> t) & 1;
    fi.nb[bits] = find(L.level + 1, cc);
    if (fi.nb[bits] < 0) { fi.kind = -1; return fi; }   // unbalanced
  }
  return fi;
}

bool Forest::regrid(const std::vector<uint8_t>& tag, int B, int max_level, Forest* out,
                    std::vector<TransferEntry>* tmap, int64_t* n_refined,
                    int64_t* n_coarsened, std::string* err, bool skip_unchanged) const {
  const int64_t n = size();
  const int nkids = 1 << dim_;
  const int nsub = 1 << (dim_ - 1);
  const int nf = 2 * dim_;
  // neighbour lists (CSR over the face table, faces in (axis, side) order)
  std::vector<int64_t> off(n + 1, 0);
  std::atomic<int> unbalanced{0};
  parallel_ranges(n, 1024, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int64_t c = 0;
      for (int f = 0; f < nf; ++f) {
        const int k = faces_[(size_t)e * nf + f].kind;
        if (k < 0) unbalanced.store(1, std::memory_order_relaxed);
        c += (k == FACE_CONF || k == FACE_FINE) ? 1 : (k == FACE_COARSE ? nsub : 0);
      }
      off[e] = c;
    }
  });
  if (unbalanced.load()) { *err = "forest is not 2:1 balanced"; return false; }
  off[n] = exclusive_scan(off.data(), n);
  std::vector<int32_t> adj((size_t)off[n]);
  parallel_ranges(n, 1024, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int64_t o = off[e];
      for (int f = 0; f < nf; ++f) {
        const FaceInfo& fi = faces_[(size_t)e * nf + f];
        const int c = (fi.kind == FACE_CONF || fi.kind == FACE_FINE) ? 1 : (fi.kind == FACE_COARSE ? nsub : 0);
        for (int k = 0; k < c; ++k) adj[o++] = fi.nb[k];
      }
    }
  });
  // buffer: dilate the tags B times over face neighbours
  std::vector<uint8_t> near(n), prev;
  for (int64_t e = 0; e < n; ++e) near[e] = tag[e] ? 1 : 0;
  for (int it = 0; it < B; ++it) {
    prev = near;
    parallel_ranges(n, 2048, [&](int64_t e0, int64_t e1) {
      for (int64_t e = e0; e < e1; ++e) {
        if (prev[e]) continue;
        for (int64_t k = off[e]; k < off[e + 1]; ++k)
          if (prev[adj[k]]) { near[e] = 1; break; }
      }
    });
  }
  // refinement and its 2:1 closure (least fixpoint, independent of visiting order)
  std::vector<uint8_t> ref(n, 0);
  std::vector<int32_t> work;
  for (int64_t e = 0; e < n; ++e)
    if (near[e] && leaves_[e].level < max_level) { ref[e] = 1; work.push_back((int32_t)e); }
  for (size_t head = 0; head < work.size(); ++head) {
    const int32_t e = work[head];
    for (int64_t k = off[e]; k < off[e + 1]; ++k) {
      const int32_t m = adj[k];
      if (!ref[m] && leaves_[m].level < leaves_[e].level) { ref[m] = 1; work.push_back(m); }
    }
  }
  // families: complete sibling groups are contiguous in Morton order, child index 0 first.  A
  // family head has even coordinates and its siblings odd ones, so families never overlap and
  // each head is tested on its own; coars = 2 at a coarsened family's head, 1 at its siblings.
  std::vector<uint8_t> coars(n, 0);
  parallel_ranges(n, 2048, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1 && e + nkids <= n; ++e) {
      const Leaf& L = leaves_[e];
      if (L.level == 0) continue;
      if ((L.c[0] & 1) || (L.c[1] & 1) || (L.c[2] & 1)) continue;
      bool complete = true;
      for (int k = 1; k < nkids && complete; ++k) {
        const Leaf& M = leaves_[e + k];
        int32_t want[3] = {L.c[0] + (k & 1), L.c[1] + ((k >> 1) & 1), L.c[2] + ((k >> 2) & 1)};
        if (dim_ == 2) want[2] = 0;
        complete = M.level == L.level && M.c[0] == want[0] && M.c[1] == want[1] && M.c[2] == want[2];
      }
      if (!complete) continue;
      bool ok = true;
      for (int k = 0; k < nkids && ok; ++k) if (near[e + k] || ref[e + k]) ok = false;
      for (int k = 0; k < nkids && ok; ++k) {
        const int64_t m = e + k;
        for (int64_t j = off[m]; j < off[m + 1]; ++j) {
          const int32_t o = adj[j];
          if (o >= e && o < e + nkids) continue;
          if (leaves_[o].level + ref[o] > L.level) { ok = false; break; }
        }
      }
      if (ok) {
        coars[e] = 2;
        for (int k = 1; k < nkids; ++k) coars[e + k] = 1;
      }
    }
  });
  // emit new leaves in order: a refined leaf gives its 2^d children, a coarsened family its
  // parent (at the head), every other leaf itself
  std::vector<int64_t> pos(n + 1);
  int64_t nref = 0, ncoarse = 0;
  for (int64_t e = 0; e < n; ++e) {
    nref += ref[e];
    ncoarse += coars[e] == 2;
    pos[e] = ref[e] ? nkids : (coars[e] == 1 ? 0 : 1);
  }
  if (skip_unchanged && nref == 0 && ncoarse == 0) {
    *n_refined = 0;
    *n_coarsened = 0;
    return true;
  }
  pos[n] = exclusive_scan(pos.data(), n);
  std::vector<Leaf> nl((size_t)pos[n]);
  tmap->assign((size_t)pos[n], TransferEntry{});
  TransferEntry* tm = tmap->data();
  parallel_ranges(n, 2048, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      const Leaf& L = leaves_[e];
      int64_t o = pos[e];
      if (ref[e]) {
        for (int ci = 0; ci < nkids; ++ci, ++o) {
          Leaf c{L.level + 1, {2 * L.c[0] + (ci & 1), 2 * L.c[1] + ((ci >> 1) & 1),
                               2 * L.c[2] + ((ci >> 2) & 1)}};
          if (dim_ == 2) c.c[2] = 0;
          nl[o] = c;
          tm[o] = TransferEntry{XFER_CHILD, {(int32_t)e, ci, -1, -1, -1, -1, -1, -1}};
        }
      } else if (coars[e] == 2) {
        nl[o] = Leaf{L.level - 1, {L.c[0] >> 1, L.c[1] >> 1, L.c[2] >> 1}};
        TransferEntry t{XFER_PARENT, {-1, -1, -1, -1, -1, -1, -1, -1}};
        for (int k = 0; k < nkids; ++k) t.src[k] = (int32_t)(e + k);
        tm[o] = t;
      } else if (coars[e] == 0) {
        nl[o] = L;
        tm[o] = TransferEntry{XFER_KEEP, {(int32_t)e, -1, -1, -1, -1, -1, -1, -1}};
      }
    }
  });
  out->dim_ = dim_;
  out->max_level_ = max_level_;
  for (int a = 0; a < 3; ++a) { out->base_[a] = base_[a]; out->periodic_[a] = periodic_[a]; }
  out->set_leaves(std::move(nl));
  *n_refined = nref;
  *n_coarsened = ncoarse;
  return true;
}

void Forest::face_lists(std::vector<int32_t>* conf, std::vector<int32_t>* mort,
                        std::vector<int32_t>* bnd) const {
  // per element: conforming faces on the + side, then every coarse face (mortar group) and
  // wall face in (axis, side) order; rows are placed by prefix sums of the per-element counts
  const int64_t n = size();
  const int nsub = 1 << (dim_ - 1);
  std::vector<int64_t> pc(n + 1), pm(n + 1), pb(n + 1);
  parallel_ranges(n, 2048, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int64_t c = 0, m = 0, b = 0;
      for (int a = 0; a < dim_; ++a) {
        c += face((int32_t)e, a, 1).kind == FACE_CONF;
        for (int s = 0; s < 2; ++s) {
          const int k = face((int32_t)e, a, s).kind;
          m += k == FACE_COARSE;
          b += k == FACE_WALL;
        }
      }
      pc[e] = c; pm[e] = m; pb[e] = b;
    }
  });
  pc[n] = exclusive_scan(pc.data(), n);
  pm[n] = exclusive_scan(pm.data(), n);
  pb[n] = exclusive_scan(pb.data(), n);
  conf->assign((size_t)pc[n] * 3, 0);
  mort->assign((size_t)pm[n] * 7, 0);
  bnd->assign((size_t)pb[n] * 3, 0);
  int32_t* C = conf->data();
  int32_t* M = mort->data();
  int32_t* W = bnd->data();
  parallel_ranges(n, 2048, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int32_t* c = C + pc[e] * 3;
      int32_t* m = M + pm[e] * 7;
      int32_t* w = W + pb[e] * 3;
      for (int a = 0; a < dim_; ++a) {
        const FaceInfo& fi = face((int32_t)e, a, 1);
        if (fi.kind == FACE_CONF) { c[0] = (int32_t)e; c[1] = fi.nb[0]; c[2] = a; c += 3; }
      }
      for (int a = 0; a < dim_; ++a)
        for (int s = 0; s < 2; ++s) {
          const FaceInfo& fi = face((int32_t)e, a, s);
          if (fi.kind == FACE_COARSE) {
            m[0] = (int32_t)e; m[1] = a; m[2] = s;
            for (int k = 0; k < 4; ++k) m[3 + k] = k < nsub ? fi.nb[k] : -1;
            m += 7;
          } else if (fi.kind == FACE_WALL) {
            w[0] = (int32_t)e; w[1] = a; w[2] = s;
            w += 3;
          }
        }
    }
  });
}

void Forest::partition(int nparts, std::vector<int64_t>* starts) const {
  starts->assign(nparts + 1, 0);
  for (int p = 0; p <= nparts; ++p) (*starts)[p] = (size() * p) / nparts;
}

void Forest::halo(const std::vector<int64_t>& starts, int part, std::vector<int32_t>* rows) const {
  rows->clear();
  const int nparts = (int)starts.size() - 1;
  auto owner = [&](int64_t e) {
    int p = (int)(std::upper_bound(starts.begin(), starts.end(), e) - starts.begin()) - 1;
    return std::min(std::max(p, 0), nparts - 1);
  };
  for (int64_t e = starts[part]; e < starts[part + 1]; ++e)
    for (int a = 0; a < dim_; ++a)
      for (int s = 0; s < 2; ++s) {
        const FaceInfo& fi = face((int32_t)e, a, s);
        int cnt = 0;
        if (fi.kind == FACE_CONF || fi.kind == FACE_FINE) cnt = 1;
        else if (fi.kind == FACE_COARSE) cnt = 1 << (dim_ - 1);
        for (int k = 0; k < cnt; ++k) {
          const int32_t nb = fi.nb[k];
          const int op = owner(nb);
          if (op == part) continue;
          rows->push_back((int32_t)e); rows->push_back(a); rows->push_back(s);
          rows->push_back(nb); rows->push_back(op);
        }
      }
}

void Forest::connectivity(const std::vector<int32_t>& mort, std::vector<int32_t>* conn) const {
  // Rows {kind, a, b, c, d} per element face f = 2*axis + side:
  //   WALL {0}; CONF {1, neighbour}; FINE {2, coarse element, mortar group, sub-face};
  //   COARSE {3, mortar group}.  Mortar groups are the rows of `mort` (face_lists order).
  // Every face belongs to at most one mortar group, so the groups fill disjoint rows.
  const int nf = 2 * dim_;
  const int nsub = 1 << (dim_ - 1);
  conn->resize((size_t)size() * nf * 5);
  int32_t* C = conn->data();
  parallel_ranges(size(), 2048, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      for (int f = 0; f < nf; ++f) {
        const FaceInfo& fi = faces_[(size_t)e * nf + f];
        int32_t* r = C + ((size_t)e * nf + f) * 5;
        r[0] = fi.kind;
        r[1] = fi.kind == FACE_CONF ? fi.nb[0] : -1;
        r[2] = r[3] = r[4] = -1;
      }
  });
  const int64_t ng = (int64_t)(mort.size() / 7);
  parallel_ranges(ng, 1024, [&](int64_t g0, int64_t g1) {
    for (int64_t g = g0; g < g1; ++g) {
      const int32_t* m = mort.data() + g * 7;
      const int32_t ec = m[0], a = m[1], s = m[2];
      C[((size_t)ec * nf + 2 * a + s) * 5 + 1] = (int32_t)g;
      for (int k = 0; k < nsub; ++k) {
        int32_t* rf = C + ((size_t)m[3 + k] * nf + 2 * a + (1 - s)) * 5;
        rf[1] = ec; rf[2] = (int32_t)g; rf[3] = k;
      }
    }
  });
}

}  // namespace dgl
