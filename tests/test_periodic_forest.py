"""Periodic forests (joined boundaries): the oracle's neighbour search against brute-force
geometric adjacency with wrap-around, 2:1 balance across the joined boundaries, and the
library's host tree reproducing the oracle's leaves, face lists and transfer maps bit for bit."""
import numpy as np
import pytest

import workloads
from oracle import forest as fo


def _random_forest(base, L, periodic, seed, rounds=3, p=0.25):
    f = fo.Forest(base, L, periodic=periodic)
    for r in range(rounds):
        f, _ = f.regrid(workloads.random_flags(len(f), p, seed + r).astype(bool), 1)
    return f


@pytest.mark.parametrize("base,periodic", [((4, 3), (True, False)), ((3, 3), (True, True)),
                                           ((2, 2, 3), (True, False, True))])
def test_neighbours_match_geometry_with_wraparound(base, periodic):
    f = _random_forest(base, 2, periodic, seed=sum(base))
    assert f.is_balanced()
    boxes = [f.box(e) for e in range(len(f))]
    for e in range(len(f)):
        got = sorted(f.face_neighbors(e))
        want = sorted(j for j in range(len(f)) if j != e and
                      any(fo._share_face(boxes[e], b, f.d) for b in f.periodic_images(boxes[j])))
        assert got == want, e
        # a joined axis has no boundary faces
        for a in range(f.d):
            for s in (0, 1):
                kind, _ = f.neighbor(e, a, s)
                assert (kind == "boundary") <= (not periodic[a])


def test_balance_holds_across_the_joined_boundary():
    # refine only next to the x = 0 boundary: the ripple must reach across to x = max
    f = fo.Forest((6, 2), 3, periodic=(True, False))
    for _ in range(3):
        tag = np.array([f.box(e)[0][0] == 0 for e in range(len(f))])
        f, _ = f.regrid(tag, 0)
    assert f.is_balanced()
    top = [e for e in range(len(f)) if f.box(e)[0][1] == (6 << fo.MAXL)]
    assert max(f.leaves[e][0] for e in top) >= 2


def _oracle_rows(f):
    rows = [[f.root_index(l, c), l] + list(c) + [0] * (3 - len(c)) for l, c in f.leaves]
    return np.array(rows, dtype=np.int32).reshape(-1, 5)


def _oracle_tmap(tmap):
    rows = []
    for entry in tmap:
        if entry[0] == "keep":
            rows.append([0, entry[1]] + [-1] * 7)
        elif entry[0] == "child":
            rows.append([1, entry[1], entry[2]] + [-1] * 6)
        else:
            rows.append([2] + list(entry[1]) + [-1] * (8 - len(entry[1])))
    return np.array(rows, dtype=np.int32).reshape(-1, 9)


@pytest.mark.parametrize("base,periodic,L,B", [((4, 3), (True, False), 2, 1), ((3, 3), (True, True), 2, 2),
                                               ((2, 2, 2), (True, True, True), 1, 1)])
def test_library_forest_matches_oracle_periodic(base, periodic, L, B):
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as pkg
    d = len(base)
    lf = pkg.Forest(d, base, L, periodic=periodic)
    of = fo.Forest(base, L, periodic=periodic)
    for r in range(4):
        np.testing.assert_array_equal(lf.leaves(), _oracle_rows(of))
        conf, mort, bnd = lf.faces()
        oc, om, ob = of.face_lists()
        np.testing.assert_array_equal(conf, np.array(oc, dtype=np.int32).reshape(-1, 3))
        np.testing.assert_array_equal(bnd, np.array(ob, dtype=np.int32).reshape(-1, 3))
        want_m = np.array([[ec, a, s] + list(fs) + [-1] * (4 - len(fs)) for (ec, a, s, fs) in om],
                          dtype=np.int32).reshape(-1, 7)
        np.testing.assert_array_equal(mort, want_m)
        flags = workloads.random_flags(len(of), 0.2, seed=31 * r + d)
        tr = lf.regrid(flags, B)
        of, tmap = of.regrid(flags.astype(bool), B)
        np.testing.assert_array_equal(tr, _oracle_tmap(tmap))
    np.testing.assert_array_equal(lf.leaves(), _oracle_rows(of))
