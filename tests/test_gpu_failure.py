"""Failure detection on the GPU without a fault: every spin-wait of the library is bounded,
and a wait that runs out latches GT_ETIMEOUT, returns, and leaves the context usable.

The check makes a real look-back wait run out (its predecessor never publishes), with a
short bound, then uses the same system for a full tree build and walk whose results
must still match the oracle.  A bound set on a system must not change its results.
"""
import time

import numpy as np
import pytest

from paper_1610_07279_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_07279_gb300 import build
    build.build()
    import oracle as O
    O.build()
    from paper_1610_07279_gb300 import gothic as g
    g.load()
    return torch, g, O


def _tree_matches_oracle(g, O, s, pos, mass, leaf):
    t = s.get_tree()
    p4 = np.zeros((len(mass), 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    tree = O.build_tree(skey, leaf)
    jpos, bj = O.pseudo_j(tree, p4[order])
    return (np.array_equal(t["keys"], skey) and np.array_equal(t["order"], order)
            and t["n_nodes"] == tree["n_nodes"] and np.array_equal(t["jpos"].view(np.uint32), jpos.view(np.uint32)))


@pytest.mark.parametrize("iterations", [1, 1000, 20000])
def test_bounded_wait_runs_out_and_the_context_stays_usable(env, iterations):
    torch, g, O = env
    n = 20000
    pos, vel, mass, eps = ics.plummer(n, seed=61)
    prm = g.gt_default_params()
    prm.eps = eps
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    t0 = time.perf_counter()
    assert s.probe_bounded_wait(iterations) == g.GT_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert s.status() == g.GT_OK  # the probe's status was read and cleared
    # the same system, and the GPU, still work
    s.build_tree()
    acc = torch.zeros((n, 4), device="cuda")
    s.accel_active(None, None, acc)
    assert s.status() == g.GT_OK
    assert _tree_matches_oracle(g, O, s, pos, mass, prm.leaf_max)
    assert torch.isfinite(acc).all()
    s.close()


def test_wait_bound_does_not_change_results(env):
    torch, g, O = env
    n = 1 << 16
    pos, vel, mass, eps = ics.nfw(n, seed=62)
    outs = []
    for limit in (0, 1 << 16):
        prm = g.gt_default_params()
        prm.eps = eps
        prm.rebuild_every = 2
        prm.group_mode = g.GT_GROUP_CELLS
        s = g.System(n, prm)
        s.set_wait_limit(limit)
        s.set_state(pos, vel, mass)
        s.start()
        for _ in range(6):
            s.block_step()
        assert s.status() == g.GT_OK
        outs.append(s.get_state())
        s.close()
    a, b = outs
    for f in ("pos", "vel", "level", "t0", "id"):
        assert np.array_equal(a[f], b[f]), f
