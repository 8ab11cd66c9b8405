"""gt_sort_pairs_noalloc: the sort for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they need a sort -- they run inside another
framework's memory budget, or in a loop that must not pay cudaMalloc's implicit
device synchronisation.  This entry point sorts their (key, value) pairs in place
with scratch that the library keeps in a static device array.  The test checks it
against the sort that gt_build_tree performs: the keys in the caller's order,
sorted with their indices as values, must give back exactly the tree's sorted keys
and sort order, on two calls in a row (the second call reuses the static scratch
the first one left behind).
"""
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
    from paper_1610_07279_gb300 import gothic as g
    g.load()
    return torch, g


def test_noalloc_sort_matches_tree_build_sort(env):
    torch, g = env
    n = (1 << 18) + 1234  # several sort tiles and a ragged last one
    pos, vel, mass, eps = ics.plummer(n, seed=31)
    prm = g.gt_default_params()
    prm.eps = eps
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    s.build_tree()
    tree = s.get_tree()
    s.sync()
    s.close()
    skey, order = tree["keys"], tree["order"]
    keys_in = np.empty_like(skey)
    keys_in[order] = skey  # every particle's key, in the caller's order
    for _ in range(2):
        d_keys = torch.from_numpy(keys_in.view(np.int64).copy()).cuda()
        d_vals = torch.arange(n, dtype=torch.int32, device="cuda")
        g.gt_sort_pairs_noalloc(d_keys, d_vals, n)
        torch.cuda.synchronize()
        assert np.array_equal(d_keys.cpu().numpy().view(np.uint64), skey)
        assert np.array_equal(d_vals.cpu().numpy().view(np.uint32), order)


def test_noalloc_sort_rejects_more_than_its_scratch(env):
    torch, g = env
    d_keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    d_vals = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GothicError) as e:
        g.gt_sort_pairs_noalloc(d_keys, d_vals, g.GT_NOALLOC_SORT_MAX + 1)
    assert e.value.status == g.GT_EINVAL
