"""CPU checks of the C ABI library: it loads, exports every declared symbol, and its host tree
reproduces the oracle's leaf order, face/mortar lists and transfer map bit for bit."""
import os
import re
import subprocess

import numpy as np
import pytest

import workloads
from oracle import forest as fo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as p
    return p


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree(pkg):
    assert _declared() == sorted(pkg.EXPORTED)


def test_library_exports_every_declared_symbol(pkg):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing
    lib = pkg.load_library()
    for s in _declared():
        assert hasattr(lib, s)
    assert b"sm_103a" in lib.dg_version()


def _oracle_leaves(f):
    rows = []
    for l, c in f.leaves:
        cc = list(c) + [0] * (3 - len(c))
        rows.append([f.root_index(l, c), l] + cc)
    return np.array(rows, dtype=np.int32).reshape(-1, 5)


def _oracle_faces(f):
    conf, mort, bnd = f.face_lists()
    c = np.array(conf, dtype=np.int32).reshape(-1, 3)
    m = np.array([[ec, a, s] + list(fs) + [-1] * (4 - len(fs)) for ec, a, s, fs in mort],
                 dtype=np.int32).reshape(-1, 7)
    b = np.array(bnd, dtype=np.int32).reshape(-1, 3)
    return c, m, b


def _oracle_tmap(tmap, d):
    rows = []
    for entry in tmap:
        if entry[0] == "keep":
            rows.append([0, entry[1]] + [-1] * 7)
        elif entry[0] == "child":
            rows.append([1, entry[1], entry[2]] + [-1] * 6)
        else:
            rows.append([2] + list(entry[1]) + [-1] * (8 - len(entry[1])))
    return np.array(rows, dtype=np.int32).reshape(-1, 9)


CASES = [((3, 3), 3, 1), ((4, 2), 2, 2), ((5, 5), 3, 0), ((2, 2, 2), 2, 1), ((3, 1, 2), 2, 2)]


@pytest.mark.parametrize("base,max_level,B", CASES)
def test_forest_matches_oracle_bit_exact(pkg, base, max_level, B):
    d = len(base)
    lf = pkg.Forest(d, base, max_level)
    of = fo.Forest(base, max_level)
    for rnd in range(5):
        np.testing.assert_array_equal(lf.leaves(), _oracle_leaves(of))
        for got, want in zip(lf.faces(), _oracle_faces(of)):
            np.testing.assert_array_equal(got, want)
        flags = workloads.random_flags(len(of), 0.15 if rnd < 3 else 0.0, seed=17 * rnd + d)
        tr = lf.regrid(flags, B)
        of, tmap = of.regrid(flags.astype(bool), B)
        np.testing.assert_array_equal(tr, _oracle_tmap(tmap, d))
    np.testing.assert_array_equal(lf.leaves(), _oracle_leaves(of))


def test_forest_rejects_bad_arguments(pkg):
    from paper_2404_16648_gb300.dg import DGError
    with pytest.raises(DGError):
        pkg.Forest(4, (2, 2), 1)
    with pytest.raises(DGError):
        pkg.Forest(2, (0, 2), 1)
    f = pkg.Forest(2, (2, 2), 1)
    with pytest.raises(ValueError):
        f.regrid(np.zeros(3, np.uint8), 1)


def test_null_mesh_handles_are_rejected_before_any_device_call(pkg):
    """Every mesh entry point checks its handle first, so these run without a GPU."""
    import ctypes
    from paper_2404_16648_gb300.dg import DG_ERR_ARG
    lib = pkg.load_library()
    buf = (ctypes.c_double * 8)()
    assert lib.dg_get_pprime(None, buf, 0) == DG_ERR_ARG
    assert lib.dg_get_state(None, buf, 0, 0) == DG_ERR_ARG
    assert lib.dg_set_state(None, buf, 0, 0) == DG_ERR_ARG
    assert lib.dg_step(None, 0.1, 1, None) == DG_ERR_ARG
    assert lib.dg_indicator(None, buf, 8) == DG_ERR_ARG
    assert lib.dg_integrals(None, buf) == DG_ERR_ARG
