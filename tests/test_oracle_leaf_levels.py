"""The reading behind the one-sweep octree build (Sec. 2.1 tree, read on the sorted keys),
checked against the oracle's level-by-level tree on the CPU.

For sorted keys, let d(p) be the index of the first 3-bit digit in which keys p - 1 and p
differ (21 for equal keys; -1 at p = 0 and p = n).  A run of particles between two
positions with d < l shares its first l digits, so it is one level-l cell of the full
octree; the tree keeps a level-l run iff its parent run holds more than leaf_max
particles.  Hence particle i's leaf is at level
    L(i) = min(21, 1 + min over a in [0, M) of max(min d[i-a..i], min d[i+1..i+M-a]))
with M = leaf_max, i starts a node at every level l with d(i) < l <= L(i), and the nodes
of a level, in order of their first particle, are the tree's numbering of that level.
"""
import zlib

import numpy as np
import pytest

KEY_LEVELS = 21


def _digit_diff(skey):
    n = len(skey)
    d = np.full(n + 1, -1, np.int64)
    x = skey[1:] ^ skey[:-1]
    nz = x != 0
    bl = np.zeros(n - 1, np.int64)
    bl[nz] = np.floor(np.log2(x[nz].astype(np.float64))).astype(np.int64)  # highest set bit
    # exact highest set bit (log2 of a float can round up near powers of two)
    hi = bl.copy()
    over = nz & (np.left_shift(np.uint64(1), hi.astype(np.uint64)) > x)
    hi[over] -= 1
    d[1:n] = np.where(nz, (62 - hi) // 3, KEY_LEVELS)
    return d  # d[0] = d[n] = -1


def _leaf_levels(skey, M):
    n = len(skey)
    d = _digit_diff(skey)
    pad = np.concatenate([np.full(M, -1, np.int64), d, np.full(M + 1, -1, np.int64)])
    idx = np.arange(n) + M  # position i in pad
    mr = np.empty((M + 1, n), np.int64)  # mr[b] = min d[i+1 .. i+b]
    m = np.full(n, 127, np.int64)
    for b in range(1, M + 1):
        m = np.minimum(m, pad[idx + b])
        mr[b] = m
    ml = np.full(n, 127, np.int64)
    best = np.full(n, 127, np.int64)
    for a in range(M):
        ml = np.minimum(ml, pad[idx - a])
        best = np.minimum(best, np.maximum(ml, mr[M - a]))
    return np.minimum(best + 1, KEY_LEVELS), d


def _keys(rng, n, kind):
    if kind == "uniform":
        k = rng.integers(0, 1 << 63, n, dtype=np.uint64)
    elif kind == "clustered":  # a few coarse cells, many duplicates below them
        k = (rng.integers(0, 4, n, dtype=np.uint64) << np.uint64(60)) | rng.integers(0, 1 << 10, n, dtype=np.uint64)
    elif kind == "equal":  # runs of identical keys: chains down to level 21
        k = rng.integers(0, 3, n, dtype=np.uint64) << np.uint64(30)
    else:  # mixed scales
        shift = np.uint64(int(rng.integers(0, 62)))
        k = (rng.integers(0, 1 << 20, n, dtype=np.uint64) << np.uint64(40)) ^ (rng.integers(0, 1 << 62, n, dtype=np.uint64) >> shift)
    return np.sort(k)


@pytest.mark.parametrize("kind", ["uniform", "clustered", "equal", "mixed"])
@pytest.mark.parametrize("M", [1, 3, 16, 24, 64])
def test_leaf_levels_and_level_lists_match_the_tree(oracle_lib, kind, M):
    import oracle as O
    rng = np.random.default_rng(zlib.crc32(f"{kind}-{M}".encode()))  # fixed across runs
    for n in (1, 2, 37, 1500):
        skey = _keys(rng, n, kind)
        tree = O.build_tree(skey, M, cap=40 * n + 64)
        L, d = _leaf_levels(skey, M)
        # every particle's leaf in the oracle's tree, and its level
        leaf_level = np.full(n, -1, np.int64)
        for c in np.flatnonzero(tree["child"] < 0):
            f, k = int(tree["first"][c]), int(tree["count"][c])
            leaf_level[f:f + k] = tree["level"][c]
        assert np.array_equal(L, leaf_level), (kind, M, n)
        # the nodes of every level: particles with d(i) < l <= L(i), in particle order
        ls = tree["level_start"]
        for lvl in range(KEY_LEVELS + 1):
            starts = np.flatnonzero((d[:n] < lvl) & (lvl <= L))
            nodes = np.arange(ls[lvl], ls[lvl + 1])
            assert np.array_equal(tree["first"][nodes], starts), (kind, M, n, lvl)
