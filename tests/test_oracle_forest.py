"""Pins of the oracle's forest: brute force on small forests, ordering, face-list identities."""
import itertools

import numpy as np
import pytest

from oracle import forest as fo


def _random_forest(base, max_level, seed, rounds=3, B=1, p=0.2):
    rng = np.random.default_rng(seed)
    f = fo.Forest(base, max_level)
    maps = []
    for _ in range(rounds):
        tag = rng.random(len(f)) < p
        f, tmap = f.regrid(tag, B)
        maps.append(tmap)
    return f


def _brute_faces(f):
    """All (i, j) leaf pairs sharing a face, plus boundary faces, by geometry alone."""
    boxes = [f.box(e) for e in range(len(f))]
    pairs = set()
    for i in range(len(boxes)):
        for j in range(i + 1, len(boxes)):
            if fo._share_face(boxes[i], boxes[j], f.d):
                pairs.add((i, j))
    dom = [f.base[a] << fo.MAXL for a in range(f.d)]
    bnd = set()
    for e, b in enumerate(boxes):
        for a in range(f.d):
            if b[a][0] == 0:
                bnd.add((e, a, 0))
            if b[a][1] == dom[a]:
                bnd.add((e, a, 1))
    return pairs, bnd


CASES = [((1, 1), 3), ((2, 2), 3), ((3, 2), 3), ((4, 4), 2), ((2, 2, 2), 2), ((1, 2, 3), 2)]


@pytest.mark.parametrize("base,max_level", CASES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_balance_order_coverage(base, max_level, seed):
    f = _random_forest(base, max_level, seed, B=seed % 3)
    assert f.is_balanced()
    keys = [f.sort_key(lf) for lf in f.leaves]
    assert keys == sorted(keys)
    # coverage: leaf volumes (in units of the finest cell) sum to the domain exactly
    vol = sum(1 << (f.d * (fo.MAXL - l)) for l, _ in f.leaves)
    assert vol == int(np.prod(f.base)) << (f.d * fo.MAXL)
    # no overlaps: all boxes disjoint (volumes add up and anchors unique)
    assert len(set(f.leaves)) == len(f.leaves)
    assert max(l for l, _ in f.leaves) <= max_level


@pytest.mark.parametrize("base,max_level", CASES)
@pytest.mark.parametrize("seed", [3, 4])
def test_face_lists_match_geometry(base, max_level, seed):
    f = _random_forest(base, max_level, seed, B=1)
    conf, mort, bnd = f.face_lists()
    pairs, bnd_ref = _brute_faces(f)
    listed = set()
    for m, p, a in conf:
        assert f.leaves[m][0] == f.leaves[p][0]
        listed.add((min(m, p), max(m, p)))
    for ec, a, s, fines in mort:
        assert len(fines) == 1 << (f.d - 1)
        for fi in fines:
            assert f.leaves[fi][0] == f.leaves[ec][0] + 1
            listed.add((min(ec, fi), max(ec, fi)))
    assert listed == pairs
    assert len(listed) == len(conf) + sum(len(m[3]) for m in mort)
    assert set(bnd) == bnd_ref
    # every leaf face is accounted for exactly once
    nfaces = 2 * len(conf) + sum(1 + len(m[3]) for m in mort) + len(bnd)
    assert nfaces == 2 * f.d * len(f)
    # canonical order: conforming by low element, mortars by coarse element
    assert [c[0] for c in conf] == sorted(c[0] for c in conf)
    assert [m[0] for m in mort] == sorted(m[0] for m in mort)


def test_buffer_hops_refine_neighbourhood():
    f = fo.Forest((7, 7), 1)
    tag = np.zeros(len(f), dtype=bool)
    centre = f.index(0, (3, 3))
    tag[centre] = True
    for B, expect in [(0, 1), (1, 5), (2, 13)]:
        g, _ = f.regrid(tag, B)
        refined = {(c[0] >> 1, c[1] >> 1) for l, c in g.leaves if l == 1}
        assert len(refined) == expect
        # the refined set is the ball of radius B in the face-adjacency (L1) metric
        for (x, z) in refined:
            assert abs(x - 3) + abs(z - 3) <= B


def test_refine_then_coarsen_round_trip():
    for base in [(3, 3), (2, 2, 2)]:
        f = fo.Forest(base, 2)
        tag = np.zeros(len(f), dtype=bool)
        tag[0] = True
        g, _ = f.regrid(tag, 0)
        tag2 = np.zeros(len(g), dtype=bool)
        tag2[0] = True
        h, _ = g.regrid(tag2, 0)
        assert max(l for l, _ in h.leaves) == 2 and h.is_balanced()
        # no tags: level-2 families coarsen first, then level-1 families
        k, _ = h.regrid(np.zeros(len(h), dtype=bool), 0)
        m, _ = k.regrid(np.zeros(len(k), dtype=bool), 0)
        assert m.leaves == f.leaves


def test_ripple_balance_closure():
    # refining a leaf next to a coarser one forces the coarser one to refine
    f = fo.Forest((4, 1), 2)
    tag = np.zeros(4, dtype=bool)
    tag[1] = True
    g, _ = f.regrid(tag, 0)                       # leaf 1 -> 4 children at level 1
    tag2 = np.array([l == 1 and c == (3, 0) for l, c in g.leaves])
    h, _ = g.regrid(tag2, 0)                      # child at x=3 refines to level 2
    assert h.is_balanced()
    # its level-0 neighbour to the right (root 2) had to become level 1
    assert not h.is_leaf(0, (2, 0))
    assert h.is_leaf(1, (4, 0))


def test_transfer_map_covers_old_leaves():
    f = _random_forest((3, 3), 3, 9, rounds=2)
    rng = np.random.default_rng(5)
    g, tmap = f.regrid(rng.random(len(f)) < 0.3, 1)
    seen = []
    for entry, (l, c) in zip(tmap, g.leaves):
        if entry[0] == "keep":
            assert f.leaves[entry[1]] == (l, c)
            seen.append(entry[1])
        elif entry[0] == "child":
            pl, pc = f.leaves[entry[1]]
            assert pl + 1 == l and tuple(x >> 1 for x in c) == pc
            ci = sum(((c[a] & 1) << a) for a in range(f.d))
            assert ci == entry[2]
            seen.append(entry[1])
        else:
            for ci, e in enumerate(entry[1]):
                cl, cc = f.leaves[e]
                assert cl == l + 1 and tuple(x >> 1 for x in cc) == c
                assert sum(((cc[a] & 1) << a) for a in range(f.d)) == ci
                seen.append(e)
    assert sorted(set(seen)) == list(range(len(f)))
