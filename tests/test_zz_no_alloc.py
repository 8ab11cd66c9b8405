"""gt_sort_pairs_noalloc: the sort for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they need a sort -- they run inside another
framework's memory budget, or in a loop that must not pay cudaMalloc's implicit
device synchronisation.  This entry point sorts their (key, value) pairs in place
with scratch that the library keeps in a static device array.  The tests check it
against the sort that gt_build_tree performs (the keys in the caller's order, sorted
with their indices as values, must give back exactly the tree's sorted keys and sort
order) and against the oracle's stable sort and numpy's stable argsort on keys with
many ties, at the edges of the static array (0 and 1 pairs, an exact multiple of the
4096-key tile, the largest accepted size), each on two calls in a row (the second
call reuses the static scratch the first one left behind); after each, the sort's
device status (gt_sort_noalloc_status) must be clear.
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
    import oracle as O
    O.build()
    from paper_1610_07279_gb300 import gothic as g
    g.load()
    return torch, g, O


def test_noalloc_sort_matches_tree_build_sort(env):
    torch, g, O = env
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
        assert g.gt_sort_noalloc_status() == g.GT_OK
        assert np.array_equal(d_keys.cpu().numpy().view(np.uint64), skey)
        assert np.array_equal(d_vals.cpu().numpy().view(np.uint32), order)


def _tied_keys(rng, n):
    """63-bit keys, a third of them drawn from a small set (long runs of equal keys)."""
    k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    few = rng.integers(0, 1 << 63, 37, dtype=np.uint64)
    sel = rng.random(n) < 1 / 3
    k[sel] = few[rng.integers(0, 37, int(sel.sum()))]
    return k


@pytest.mark.parametrize("n", [0, 1, 2, 3 * 4096, (1 << 20) - 1, 1 << 20])
def test_noalloc_sort_edges_against_oracle(env, n):
    torch, g, O = env
    assert g.GT_NOALLOC_SORT_MAX == 1 << 20
    rng = np.random.default_rng(n + 17)
    keys = _tied_keys(rng, n)
    vals = rng.permutation(n).astype(np.uint32)
    perm = np.argsort(keys, kind="stable")
    if n:
        order, skey = O.sort(keys)  # the oracle's stable sort of (key, index)
        assert np.array_equal(order, perm.astype(np.uint32)) and np.array_equal(skey, keys[perm])
    for _ in range(2):
        d_keys = torch.from_numpy(keys.view(np.int64).copy()).to("cuda")
        d_vals = torch.from_numpy(vals.view(np.int32).copy()).to("cuda")
        g.gt_sort_pairs_noalloc(d_keys, d_vals, n)
        torch.cuda.synchronize()
        assert g.gt_sort_noalloc_status() == g.GT_OK
        assert np.array_equal(d_keys.cpu().numpy().view(np.uint64), keys[perm])
        assert np.array_equal(d_vals.cpu().numpy().view(np.uint32), vals[perm])


def test_noalloc_sort_rejects_more_than_its_scratch(env):
    torch, g, O = env
    d_keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    d_vals = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GothicError) as e:
        g.gt_sort_pairs_noalloc(d_keys, d_vals, g.GT_NOALLOC_SORT_MAX + 1)
    assert e.value.status == g.GT_EINVAL
