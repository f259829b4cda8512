"""Forest of quad/oct-trees with active-leaf storage (oracle; test infrastructure only).

Restates the tree-based AMR bookkeeping of arXiv 2404.16648:

* every base (coarse-mesh) cell is the root of its own tree, so the mesh is a forest (Sec. 3.1);
* only active leaves are stored; a parent is deleted once its children exist and the
  children are deleted when they are merged back (Sec. 3.1);
* regrid every T steps with a buffer of B cells between the tagged feature and the
  coarse/fine interface (Sec. 3.2.1, which says T and B are also used by the tree method);
* 2:1 balance kept across all levels (Sec. 4.3, rising thermal bubble);
* faces shared by two elements of one level are conforming; a face whose other side is
  refined once carries 2^(d-1) mortars (Sec. 3.3).

Readings (the paper does not fix these; the CUDA library's host tree follows the same rules,
written separately):
* a leaf is (level, integer coordinates at that level); axis d-1 is vertical;
* leaf order: roots lexicographic with x fastest, then Morton order inside a root with child
  index ix + 2 iy + 4 iz (2D: ix + 2 iz);
* B counts face-adjacency hops: "near" = tagged dilated B times over face neighbours;
* refine a leaf if near and level < max_level; then close refinement under the face 2:1 rule
  (a neighbour coarser than a refined leaf is refined too, to a fixpoint);
* coarsen a family only if its 2^d siblings are all leaves, none is near or refined, and every
  face neighbour outside the family ends at a level <= the siblings' level after refinement;
* conforming faces are listed from the low-side element in leaf order, axes x, y, z;
  mortars by coarse element in leaf order, then axis, then side (low, high), with the fine
  elements of one mortar group in Morton order over the tangential axes; boundary faces by
  element, axis, side.

Pinned by tests/test_oracle_forest.py (brute-force balance and coverage on small forests,
face-count identities, ordering, refine/coarsen round trips).
"""
import itertools

import numpy as np

MAXL = 20   # maximum supported level depth for Morton keys


class Forest:
    """Active leaves of a forest over a base grid of ``base`` root cells (length d)."""

    def __init__(self, base, max_level, leaves=None, periodic=None):
        self.base = tuple(int(b) for b in base)
        self.d = len(self.base)
        self.max_level = int(max_level)
        # periodic[a]: the two boundaries of axis a are joined (neighbour lookups wrap around)
        self.periodic = tuple(bool(p) for p in periodic) if periodic is not None else (False,) * self.d
        if leaves is None:
            leaves = [(0, c) for c in self._root_coords()]
        self.leaves = [(int(l), tuple(int(x) for x in c)) for l, c in leaves]
        self._index = {lf: i for i, lf in enumerate(self.leaves)}

    # ------------------------------------------------------------------ ordering
    def _root_coords(self):
        # lexicographic with x fastest
        ranges = [range(b) for b in reversed(self.base)]
        return [tuple(reversed(t)) for t in itertools.product(*ranges)]

    def root_index(self, level, c):
        r = [ci >> level for ci in c]
        idx = 0
        for a in reversed(range(self.d)):
            idx = idx * self.base[a] + r[a]
        return idx

    def morton(self, level, c):
        local = [(ci - ((ci >> level) << level)) << (MAXL - level) for ci in c]
        key = 0
        for b in range(MAXL):
            for a in range(self.d):
                key |= ((local[a] >> b) & 1) << (b * self.d + a)
        return key

    def sort_key(self, leaf):
        level, c = leaf
        return (self.root_index(level, c), self.morton(level, c))

    # ------------------------------------------------------------------ queries
    def __len__(self):
        return len(self.leaves)

    def is_leaf(self, level, c):
        return (level, tuple(c)) in self._index

    def index(self, level, c):
        return self._index[(level, tuple(c))]

    def extent(self, level, axis):
        return self.base[axis] << level

    def neighbor(self, e, axis, side):
        """Classify face (axis, side) of leaf e.

        Returns ('boundary', None) | ('same', n) | ('coarse', n) | ('fine', [n...]) where
        'coarse' means the neighbour is one level coarser (e is on the fine side) and 'fine'
        lists the 2^(d-1) finer neighbours in Morton order over the tangential axes.
        """
        level, c = self.leaves[e]
        cn = list(c)
        cn[axis] += 1 if side == 1 else -1
        if cn[axis] < 0 or cn[axis] >= self.extent(level, axis):
            if not self.periodic[axis]:
                return ("boundary", None)
            cn[axis] %= self.extent(level, axis)
        if self.is_leaf(level, cn):
            return ("same", self.index(level, cn))
        if level > 0:
            par = [x >> 1 for x in cn]
            if self.is_leaf(level - 1, par):
                return ("coarse", self.index(level - 1, par))
        tang = [a for a in range(self.d) if a != axis]
        fines = []
        for bits in range(1 << (self.d - 1)):
            cc = [2 * x for x in cn]
            cc[axis] += 0 if side == 1 else 1
            for t, a in enumerate(tang):
                cc[a] += (bits >> t) & 1
            if not self.is_leaf(level + 1, cc):
                raise RuntimeError("forest is not 2:1 balanced at leaf %d" % e)
            fines.append(self.index(level + 1, cc))
        return ("fine", fines)

    def face_neighbors(self, e):
        out = []
        for a in range(self.d):
            for s in (0, 1):
                kind, n = self.neighbor(e, a, s)
                if kind in ("same", "coarse"):
                    out.append(n)
                elif kind == "fine":
                    out.extend(n)
        return out

    # ------------------------------------------------------------------ regrid
    def regrid(self, tag, B):
        """One regrid pass (Sec. 3.1, 3.2.1); returns (new Forest, transfer map).

        ``tag``: per-leaf bool (refinement criterion met).  The transfer map lists, for every
        new leaf, ('keep', old) | ('child', old, child_index) | ('parent', [old x 2^d]).
        """
        n = len(self.leaves)
        d = self.d
        nbrs = [self.face_neighbors(e) for e in range(n)]
        near = [bool(t) for t in tag]
        for _ in range(B):
            prev = near[:]
            near = [prev[e] or any(prev[m] for m in nbrs[e]) for e in range(n)]
        level = [lf[0] for lf in self.leaves]
        refine = [near[e] and level[e] < self.max_level for e in range(n)]
        changed = True
        while changed:
            changed = False
            for e in range(n):
                if not refine[e]:
                    continue
                for m in nbrs[e]:
                    if level[m] < level[e] and not refine[m]:
                        refine[m] = True
                        changed = True
        target = [level[e] + (1 if refine[e] else 0) for e in range(n)]
        # families of complete siblings
        fam = {}
        for e, (l, c) in enumerate(self.leaves):
            if l > 0:
                fam.setdefault((l - 1, tuple(x >> 1 for x in c)), []).append(e)
        coarsen_first = {}
        coarsened = set()
        for (pl, pc), members in fam.items():
            if len(members) != (1 << d):
                continue
            l = pl + 1
            ok = all(not near[m] and not refine[m] for m in members)
            if ok:
                mset = set(members)
                for m in members:
                    for o in nbrs[m]:
                        if o not in mset and target[o] > l:
                            ok = False
                            break
                    if not ok:
                        break
            if ok:
                members = sorted(members)
                coarsen_first[members[0]] = (pl, pc, members)
                coarsened.update(members)
        new_leaves, tmap = [], []
        for e, (l, c) in enumerate(self.leaves):
            if refine[e]:
                for ci in range(1 << d):
                    cc = tuple(2 * c[a] + ((ci >> a) & 1) for a in range(d))
                    new_leaves.append((l + 1, cc))
                    tmap.append(("child", e, ci))
            elif e in coarsened:
                if e in coarsen_first:
                    pl, pc, members = coarsen_first[e]
                    new_leaves.append((pl, pc))
                    tmap.append(("parent", members))
            else:
                new_leaves.append((l, c))
                tmap.append(("keep", e))
        return Forest(self.base, self.max_level, new_leaves, self.periodic), tmap

    # ------------------------------------------------------------------ faces
    def face_lists(self):
        """Conforming faces, mortar groups and boundary faces in the canonical order."""
        conf, mort, bnd = [], [], []
        for e in range(len(self.leaves)):
            for a in range(self.d):
                kind, n = self.neighbor(e, a, 1)
                if kind == "same":
                    conf.append((e, n, a))
            for a in range(self.d):
                for s in (0, 1):
                    kind, n = self.neighbor(e, a, s)
                    if kind == "fine":
                        mort.append((e, a, s, list(n)))
                    elif kind == "boundary":
                        bnd.append((e, a, s))
        return conf, mort, bnd

    # ------------------------------------------------------------------ checks
    def is_balanced(self):
        """Brute force over all leaf pairs: face-adjacent leaves differ by <= 1 level (across a
        periodic boundary too, by comparing with the shifted copies of the other box)."""
        boxes = [self.box(e) for e in range(len(self.leaves))]
        for i in range(len(boxes)):
            for j in range(i + 1, len(boxes)):
                if any(_share_face(boxes[i], b, self.d) for b in self.periodic_images(boxes[j])):
                    if abs(self.leaves[i][0] - self.leaves[j][0]) > 1:
                        return False
        return True

    def periodic_images(self, box):
        """The box and its copies shifted by one domain length along each periodic axis."""
        out = [box]
        for a in range(self.d):
            if not self.periodic[a]:
                continue
            L = self.base[a] << MAXL
            out = out + [[(lo + sh, hi + sh) if k == a else (lo, hi) for k, (lo, hi) in enumerate(b)]
                         for b in out for sh in (-L, L)]
        return out

    def box(self, e):
        """Leaf extent in units of the finest supported level (integers)."""
        l, c = self.leaves[e]
        s = 1 << (MAXL - l)
        return [(ci * s, (ci + 1) * s) for ci in c]


def _share_face(b1, b2, d):
    touching = 0
    overlap = 0
    for a in range(d):
        lo = max(b1[a][0], b2[a][0])
        hi = min(b1[a][1], b2[a][1])
        if hi == lo:
            touching += 1
        elif hi > lo:
            overlap += 1
    return touching == 1 and overlap == d - 1


def leaf_array(forest):
    """Leaves as int32 rows (root, level, c_0, .., c_{d-1}) for comparison with other trees."""
    rows = []
    for l, c in forest.leaves:
        rows.append([forest.root_index(l, c), l] + list(c))
    return np.array(rows, dtype=np.int64).reshape(len(rows), 2 + forest.d)
