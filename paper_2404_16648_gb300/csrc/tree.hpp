// Host forest of quad/oct-trees for the GB300 dGSEM library.
//
// Sec. 3.1 of arXiv 2404.16648: every base cell is the root of its own tree (a forest), and
// only active leaves are stored.  Sec. 3.2.1: regrid every T steps with a buffer of B cells.
// Sec. 4.3: 2:1 balance across all levels.  Sec. 3.3: conforming faces and hanging faces with
// 2^(d-1) mortars.  The integer work runs on the host; its outputs (leaf order, face kinds,
// neighbour indices, transfer map) are uploaded to the device as flat int32 arrays.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace dgl {

struct Leaf {
  int32_t level;
  int32_t c[3];   // integer coordinates at `level` (c[2] = 0 in 2D)
};

// Face kinds of an element face, as seen from that element.
enum FaceKind : int32_t {
  FACE_WALL = 0,     // domain boundary (no-flux wall)
  FACE_CONF = 1,     // same-level neighbour nb[0]
  FACE_FINE = 2,     // this element is the fine side; nb[0] is the coarse neighbour
  FACE_COARSE = 3    // this element is the coarse side; nb[0..2^(d-1)-1] are the fine ones
};

struct FaceInfo {
  int32_t kind;
  int32_t nb[4];
};

// Transfer map entry for one new leaf.
enum TransferKind : int32_t { XFER_KEEP = 0, XFER_CHILD = 1, XFER_PARENT = 2 };
struct TransferEntry {
  int32_t kind;
  int32_t src[8];   // KEEP: src[0]; CHILD: src[0] parent, src[1] child index; PARENT: 2^d kids
};

class Forest {
 public:
  Forest() = default;
  // uniform level-0 forest; periodic[a] != 0 joins the two boundaries of axis a (the neighbour
  // lookups wrap around, so balance, buffers and face lists see the periodic neighbours)
  Forest(int dim, const int base[3], int max_level, const int periodic[3] = nullptr);

  int dim() const { return dim_; }
  int max_level() const { return max_level_; }
  const int* base() const { return base_; }
  int64_t size() const { return (int64_t)leaves_.size(); }
  const std::vector<Leaf>& leaves() const { return leaves_; }
  int32_t root_index(const Leaf& l) const;

  // -1 if (level, c) is not a leaf.
  int32_t find(int level, const int32_t c[3]) const;
  FaceInfo classify(int32_t e, int axis, int side) const;
  // classify() of every face, tabulated once per leaf set: face(e, a, s).
  const FaceInfo& face(int32_t e, int axis, int side) const { return faces_[((size_t)e * dim_ + axis) * 2 + side]; }

  // One regrid pass.  Returns false (with `err`) if the forest is not 2:1 balanced.  With
  // skip_unchanged, a pass that refines and coarsens nothing returns with both counts zero and
  // leaves *out and *tmap untouched (the new forest would equal this one).
  bool regrid(const std::vector<uint8_t>& tag, int B, int max_level, Forest* out,
              std::vector<TransferEntry>* tmap, int64_t* n_refined, int64_t* n_coarsened,
              std::string* err, bool skip_unchanged = false) const;

  // Canonical face lists (see dg.h, dg_get_faces).
  void face_lists(std::vector<int32_t>* conf, std::vector<int32_t>* mort,
                  std::vector<int32_t>* bnd) const;

  // Space-filling-curve partition: nparts contiguous ranges of the leaf (Morton) order with
  // element counts that differ by at most one; starts has nparts + 1 entries.
  void partition(int nparts, std::vector<int64_t>* starts) const;
  // Faces of part `part` whose other side belongs to another part, as rows
  // {local element, axis, side, remote element, remote part}; one row per neighbour element
  // (a coarse face lists each fine neighbour).  These are the traces a rank would receive
  // before each right-hand-side evaluation.
  void halo(const std::vector<int64_t>& starts, int part, std::vector<int32_t>* rows) const;

  // Per element, per face f = 2*axis + side, 5 int32 (see tree.cpp); `mort` from face_lists.
  void connectivity(const std::vector<int32_t>& mort, std::vector<int32_t>* conn) const;

 private:
  void set_leaves(std::vector<Leaf> leaves);
  static uint64_t key(int level, const int32_t c[3]);
  int32_t extent(int level, int axis) const { return base_[axis] << level; }

  int dim_ = 0;
  int base_[3] = {1, 1, 1};
  int periodic_[3] = {0, 0, 0};
  int max_level_ = 0;
  std::vector<Leaf> leaves_;
  // open-addressing index key(level, c) -> leaf, linear probing, power-of-two capacity
  std::vector<uint64_t> hkeys_;
  std::vector<int32_t> hvals_;
  uint64_t hmask_ = 0;
  std::vector<FaceInfo> faces_;   // [leaf][axis][side]
};

}  // namespace dgl
