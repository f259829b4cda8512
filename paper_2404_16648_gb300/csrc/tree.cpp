// Host forest: leaf order, neighbour classification, regrid with buffer and 2:1 closure,
// canonical face lists and the per-element connectivity table used by the device kernels.
#include "tree.hpp"

#include <algorithm>
#include <deque>
#include <thread>

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

// fn(e0, e1) over [0, n) split into contiguous ranges on up to 16 threads (one below 8192).
template <class F>
static void parallel_ranges(int64_t n, F fn) {
  int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  if (n < 8192) nt = 1;
  if (nt == 1) { fn((int64_t)0, n); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(fn, n * t / nt, n * (t + 1) / nt);
  for (auto& x : th) x.join();
}

void Forest::set_leaves(std::vector<Leaf> leaves) {
  leaves_ = std::move(leaves);
  uint64_t cap = 16;
  while (cap < 2 * (uint64_t)leaves_.size()) cap <<= 1;
  hkeys_.assign(cap, kEmpty);
  hvals_.assign(cap, -1);
  hmask_ = cap - 1;
  for (size_t i = 0; i < leaves_.size(); ++i) {
    const uint64_t k = key(leaves_[i].level, leaves_[i].c);
    uint64_t h = mix64(k) & hmask_;
    while (hkeys_[h] != kEmpty && hkeys_[h] != k) h = (h + 1) & hmask_;
    hkeys_[h] = k;
    hvals_[h] = (int32_t)i;
  }
  // face table; every entry depends on its own face only, so the split over threads does not
  // change the result
  const int64_t n = (int64_t)leaves_.size();
  faces_.assign((size_t)n * dim_ * 2, FaceInfo{FACE_WALL, {-1, -1, -1, -1}});
  parallel_ranges(n, [this](int64_t e0, int64_t e1) {
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

void Forest::neighbours(int32_t e, std::vector<int32_t>* out) const {
  out->clear();
  for (int a = 0; a < dim_; ++a)
    for (int s = 0; s < 2; ++s) {
      const FaceInfo& fi = face(e, a, s);
      if (fi.kind == FACE_CONF || fi.kind == FACE_FINE) out->push_back(fi.nb[0]);
      else if (fi.kind == FACE_COARSE)
        for (int k = 0; k < (1 << (dim_ - 1)); ++k) out->push_back(fi.nb[k]);
    }
}

bool Forest::regrid(const std::vector<uint8_t>& tag, int B, int max_level, Forest* out,
                    std::vector<TransferEntry>* tmap, int64_t* n_refined,
                    int64_t* n_coarsened, std::string* err) const {
  const int64_t n = size();
  const int nkids = 1 << dim_;
  // neighbour lists (CSR)
  std::vector<int32_t> off(n + 1, 0), adj;
  std::vector<int32_t> tmp;
  for (int64_t e = 0; e < n; ++e) {
    for (int a = 0; a < dim_; ++a)
      for (int s = 0; s < 2; ++s)
        if (face((int32_t)e, a, s).kind < 0) { *err = "forest is not 2:1 balanced"; return false; }
    neighbours((int32_t)e, &tmp);
    adj.insert(adj.end(), tmp.begin(), tmp.end());
    off[e + 1] = (int32_t)adj.size();
  }
  // buffer: dilate the tags B times over face neighbours
  std::vector<uint8_t> near(n), prev(n);
  for (int64_t e = 0; e < n; ++e) near[e] = tag[e] ? 1 : 0;
  for (int it = 0; it < B; ++it) {
    prev = near;
    for (int64_t e = 0; e < n; ++e) {
      if (prev[e]) continue;
      for (int32_t k = off[e]; k < off[e + 1]; ++k)
        if (prev[adj[k]]) { near[e] = 1; break; }
    }
  }
  // refinement and its 2:1 closure (least fixpoint, independent of visiting order)
  std::vector<uint8_t> ref(n, 0);
  std::deque<int32_t> work;
  for (int64_t e = 0; e < n; ++e)
    if (near[e] && leaves_[e].level < max_level) { ref[e] = 1; work.push_back((int32_t)e); }
  while (!work.empty()) {
    int32_t e = work.front(); work.pop_front();
    for (int32_t k = off[e]; k < off[e + 1]; ++k) {
      int32_t m = adj[k];
      if (!ref[m] && leaves_[m].level < leaves_[e].level) { ref[m] = 1; work.push_back(m); }
    }
  }
  std::vector<int32_t> target(n);
  for (int64_t e = 0; e < n; ++e) target[e] = leaves_[e].level + ref[e];
  // families: complete sibling groups are contiguous in Morton order, child index 0 first
  std::vector<uint8_t> coars(n, 0);
  int64_t ncoarse = 0;
  for (int64_t e = 0; e + nkids <= n; ++e) {
    const Leaf& L = leaves_[e];
    if (L.level == 0) continue;
    if ((L.c[0] & 1) || (L.c[1] & 1) || (L.c[2] & 1)) continue;
    bool complete = true;
    for (int k = 1; k < nkids && complete; ++k) {
      const Leaf& M = leaves_[e + k];
      int32_t want[3] = {L.c[0] + (k & 1), L.c[1] + ((k >> 1) & 1), L.c[2] + ((k >> 2) & 1)};
      if (dim_ == 2) { want[1] = L.c[1] + ((k >> 1) & 1); want[2] = 0; }
      complete = M.level == L.level && M.c[0] == want[0] && M.c[1] == want[1] && M.c[2] == want[2];
    }
    if (!complete) continue;
    bool ok = true;
    for (int k = 0; k < nkids && ok; ++k) if (near[e + k] || ref[e + k]) ok = false;
    for (int k = 0; k < nkids && ok; ++k) {
      int64_t m = e + k;
      for (int32_t j = off[m]; j < off[m + 1]; ++j) {
        int32_t o = adj[j];
        if (o >= e && o < e + nkids) continue;
        if (target[o] > L.level) { ok = false; break; }
      }
    }
    if (ok) { for (int k = 0; k < nkids; ++k) coars[e + k] = 1; ++ncoarse; e += nkids - 1; }
  }
  // emit new leaves in order
  std::vector<Leaf> nl;
  tmap->clear();
  int64_t nref = 0;
  for (int64_t e = 0; e < n; ++e) {
    const Leaf& L = leaves_[e];
    if (ref[e]) {
      ++nref;
      for (int ci = 0; ci < nkids; ++ci) {
        Leaf c{L.level + 1, {2 * L.c[0] + (ci & 1), 2 * L.c[1] + ((ci >> 1) & 1),
                             2 * L.c[2] + ((ci >> 2) & 1)}};
        if (dim_ == 2) c.c[2] = 0;
        nl.push_back(c);
        TransferEntry t{XFER_CHILD, {(int32_t)e, ci, -1, -1, -1, -1, -1, -1}};
        tmap->push_back(t);
      }
    } else if (coars[e]) {
      Leaf p{L.level - 1, {L.c[0] >> 1, L.c[1] >> 1, L.c[2] >> 1}};
      nl.push_back(p);
      TransferEntry t{XFER_PARENT, {-1, -1, -1, -1, -1, -1, -1, -1}};
      for (int k = 0; k < nkids; ++k) t.src[k] = (int32_t)(e + k);
      tmap->push_back(t);
      e += nkids - 1;
    } else {
      nl.push_back(L);
      TransferEntry t{XFER_KEEP, {(int32_t)e, -1, -1, -1, -1, -1, -1, -1}};
      tmap->push_back(t);
    }
  }
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
  conf->clear(); mort->clear(); bnd->clear();
  for (int64_t e = 0; e < size(); ++e) {
    for (int a = 0; a < dim_; ++a) {
      const FaceInfo& fi = face((int32_t)e, a, 1);
      if (fi.kind == FACE_CONF) { conf->push_back((int32_t)e); conf->push_back(fi.nb[0]); conf->push_back(a); }
    }
    for (int a = 0; a < dim_; ++a)
      for (int s = 0; s < 2; ++s) {
        const FaceInfo& fi = face((int32_t)e, a, s);
        if (fi.kind == FACE_COARSE) {
          mort->push_back((int32_t)e); mort->push_back(a); mort->push_back(s);
          for (int k = 0; k < 4; ++k) mort->push_back(k < (1 << (dim_ - 1)) ? fi.nb[k] : -1);
        } else if (fi.kind == FACE_WALL) {
          bnd->push_back((int32_t)e); bnd->push_back(a); bnd->push_back(s);
        }
      }
  }
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
  const int nf = 2 * dim_;
  const int nsub = 1 << (dim_ - 1);
  conn->assign((size_t)size() * nf * 5, -1);
  for (int64_t e = 0; e < size(); ++e)
    for (int a = 0; a < dim_; ++a)
      for (int s = 0; s < 2; ++s) {
        const FaceInfo& fi = face((int32_t)e, a, s);
        int32_t* r = conn->data() + ((size_t)e * nf + 2 * a + s) * 5;
        r[0] = fi.kind;
        if (fi.kind == FACE_CONF) r[1] = fi.nb[0];
      }
  const size_t ng = mort.size() / 7;
  for (size_t g = 0; g < ng; ++g) {
    const int32_t* m = mort.data() + g * 7;
    const int32_t ec = m[0], a = m[1], s = m[2];
    int32_t* rc = conn->data() + ((size_t)ec * nf + 2 * a + s) * 5;
    rc[1] = (int32_t)g;
    for (int k = 0; k < nsub; ++k) {
      int32_t* rf = conn->data() + ((size_t)m[3 + k] * nf + 2 * a + (1 - s)) * 5;
      rf[1] = ec; rf[2] = (int32_t)g; rf[3] = k;
    }
  }
}

}  // namespace dgl
