"""The debug build of the library (-DGT_DEBUG=1, built on demand into its own directory):
the walk checks every node index it takes from its queue and every child or particle
range it opens against the tree's node and particle counts, and the pseudo j-particle
pass checks every node of a chunk the same way; a failed check latches GT_EINVAL with
the kernel's tag and skips the access instead of reading outside the tree.  It stands in
for a memory checker, which this GPU pool does not run.

On small systems of every model it must give the release build's state bit for bit
(the checks change no arithmetic) after the start-up and block steps that reuse and
rebuild the tree, and latch no error.
"""
import numpy as np
import pytest

from paper_1610_07279_gb300 import ics

pytestmark = pytest.mark.gpu

MODELS = {"plummer": ics.plummer, "nfw": ics.nfw, "m31": ics.andromeda_like}


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_07279_gb300 import build
    from paper_1610_07279_gb300 import gothic as g
    build.build()
    g.load()
    dbg = g.open_library(build.build(variant="debug"))
    return g, dbg


def _steps(g, kind, n, steps):
    pos, vel, mass, eps = MODELS[kind](n, seed=21)
    prm = g.gt_default_params()
    prm.eps = eps
    prm.leaf_max = 8
    prm.rebuild_every = 3  # tree reuse and rebuilds
    prm.group_mode = g.GT_GROUP_CELLS
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    s.start()
    for _ in range(steps):
        s.block_step()
    st = s.get_state()
    stats = s.stats()
    s.close()
    return st, stats


@pytest.mark.parametrize("kind,n", [("plummer", 64), ("plummer", 1000), ("nfw", 4096), ("m31", 16384)])
def test_debug_build_matches_release(libs, kind, n):
    g, dbg = libs
    ref, ref_stats = _steps(g, kind, n, 7)
    with g.using(dbg):
        got, got_stats = _steps(g, kind, n, 7)
    assert got_stats["err"] == 0 and ref_stats["err"] == 0
    for k in ("T", "interactions", "mac_tests", "rebuilds", "block_steps", "n_nodes"):
        assert got_stats[k] == ref_stats[k], k
    for k in ("pos", "vel", "acc", "aold", "level", "t0", "id"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
