"""The host tree's loops run on a pool of helper threads; results must not depend on it.  Four
Python threads regrid their own forests at the same time (the library is called with the GIL
released, so one call holds the pool and the others run their loops on their own thread); every
thread's leaves, face lists and transfer maps must equal those of the same sequence run alone."""
import threading

import numpy as np

import workloads


def _sequence(pkg, seed, rounds=4):
    f = pkg.Forest(3, (10, 10, 8), 3)
    out = []
    for r in range(rounds):
        flags = workloads.random_flags(len(f), 0.35, seed=1000 * seed + r)
        tr = f.regrid(flags, 1)
        out.append((f.leaves().copy(), [x.copy() for x in f.faces()], tr.copy()))
    return out


def test_concurrent_regrids_match_serial_runs():
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as pkg
    seeds = [1, 2, 3, 4]
    want = {s: _sequence(pkg, s) for s in seeds}
    assert len(want[1][-1][0]) > 20000          # large enough for the parallel loops
    got, errors = {}, []

    def run(s):
        try:
            got[s] = _sequence(pkg, s)
        except Exception as exc:                 # pragma: no cover - reported below
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(s,)) for s in seeds]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for s in seeds:
        for (lw, fw, tw), (lg, fg, tg) in zip(want[s], got[s]):
            np.testing.assert_array_equal(lg, lw)
            for a, b_ in zip(fg, fw):
                np.testing.assert_array_equal(a, b_)
            np.testing.assert_array_equal(tg, tw)
