"""The host tree's helper threads do not survive fork(): a child that inherits a started pool must
start its own instead of waiting on threads that do not exist.  The parent uses the pool, forks,
and the child repeats a regrid sequence on forests large enough for the parallel loops; it must
finish and give the parent's results."""
import hashlib
import multiprocessing as mp
import warnings

import numpy as np
import pytest

import workloads


def _sequence(pkg, seed, rounds=3):
    f = pkg.Forest(3, (10, 10, 8), 3)
    for r in range(rounds):
        f.regrid(workloads.random_flags(len(f), 0.35, seed=100 * seed + r), 1)
    c, m, b = f.faces()
    return f.leaves(), c, m, b


def _digests(arrays):
    return [hashlib.sha1(np.ascontiguousarray(x).tobytes()).hexdigest() for x in arrays]


def _child(q):
    import paper_2404_16648_gb300 as pkg
    q.put(_digests(_sequence(pkg, 7)))


@pytest.mark.timeout(300)
def test_forked_child_runs_its_own_pool():
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as pkg
    want = _sequence(pkg, 7)                   # the parent's pool is running now
    assert len(want[0]) > 20000
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", DeprecationWarning)   # fork of a threaded process
        p = ctx.Process(target=_child, args=(q,))
        p.start()
    try:
        got = q.get(timeout=120)               # read before join: the child exits after its put
    except Exception:
        got = None
    p.join(30)
    if p.is_alive():                           # a child stuck on the parent's pool
        p.kill()
        p.join()
        pytest.fail("forked child did not finish")
    assert p.exitcode == 0 and got is not None
    assert got == _digests(want)


def _regrid_loop(pkg, stop):
    k = 0
    while not stop.is_set():
        _sequence(pkg, 20 + (k % 5), rounds=2)
        k += 1


@pytest.mark.timeout(600)
def test_fork_while_another_thread_regrids():
    """Children forked while a parent thread is in the middle of regrids (inside the pool, its
    job loops or the pool's lookup) must still run their own pool to the end."""
    import threading
    from paper_2404_16648_gb300 import build as b
    b.build()
    import paper_2404_16648_gb300 as pkg
    want = _digests(_sequence(pkg, 7))
    stop = threading.Event()
    t = threading.Thread(target=_regrid_loop, args=(pkg, stop), daemon=True)
    t.start()
    ctx = mp.get_context("fork")
    try:
        for _ in range(6):
            q = ctx.Queue()
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", DeprecationWarning)
                p = ctx.Process(target=_child, args=(q,))
                p.start()
            try:
                got = q.get(timeout=120)
            except Exception:
                got = None
            p.join(30)
            if p.is_alive():
                p.kill()
                p.join()
                pytest.fail("child forked during a regrid did not finish")
            assert p.exitcode == 0 and got == want
    finally:
        stop.set()
        t.join(120)
