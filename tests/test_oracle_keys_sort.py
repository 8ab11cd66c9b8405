"""Pins of the oracle's Morton keys (Appendix A) and stable key sort (Sec. 2.1)."""
import os

import numpy as np
import pytest

from paper_1610_07279_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_morton_golden(oracle_lib):
    for qx, qy, qz, key in _rows("morton_keys.txt"):
        assert oracle_lib.morton3(int(qx), int(qy), int(qz)) == int(key, 16)


def _deinterleave(key):
    q = [0, 0, 0]
    for b in range(21):
        q[0] |= ((key >> (3 * b + 2)) & 1) << b
        q[1] |= ((key >> (3 * b + 1)) & 1) << b
        q[2] |= ((key >> (3 * b)) & 1) << b
    return q


def test_morton_roundtrip_random(oracle_lib):
    rng = np.random.default_rng(5)
    for _ in range(500):
        q = [int(v) for v in rng.integers(0, 1 << 21, 3)]
        key = oracle_lib.morton3(*q)
        assert key < (1 << 63)
        assert _deinterleave(key) == q


def _zorder_rank(q, bits):
    """Recursive octant order: at every level the octant index is 4 bx + 2 by + bz."""
    rank = 0
    for lvl in range(bits - 1, -1, -1):
        octant = (((q[0] >> lvl) & 1) << 2) | (((q[1] >> lvl) & 1) << 1) | ((q[2] >> lvl) & 1)
        rank = rank * 8 + octant
    return rank


def test_morton_brute_force_3bit_grid(oracle_lib):
    """All 512 cells of an 8^3 grid: key order equals the recursive octant order."""
    cells = [(x, y, z) for x in range(8) for y in range(8) for z in range(8)]
    # place points at cell corners of the unit cube so that q = cell << 18 exactly
    p4 = np.zeros((len(cells) + 1, 4), np.float32)
    for i, c in enumerate(cells):
        p4[i, :3] = np.array(c, np.float32) / 8.0
    p4[-1, :3] = 1.0  # extends the box to a side of exactly 1
    p4[:, 3] = 1.0
    key, box = oracle_lib.keys(p4)
    assert box[3] == 1.0 and box[4] == float(1 << 21)
    for i, c in enumerate(cells):
        q = [v << 18 for v in c]
        assert _deinterleave(int(key[i])) == q
        assert int(key[i]) >> 54 == _zorder_rank(list(c), 3)
    # the corner at the box maximum clamps to 2^21 - 1 on every axis
    assert int(key[-1]) == (1 << 63) - 1


def test_keys_quantisation_properties(oracle_lib):
    pos, vel, m, eps = ics.plummer(4096, seed=3)
    p4 = np.zeros((len(m), 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = m
    key, box = oracle_lib.keys(p4)
    q = np.array([_deinterleave(int(k)) for k in key])
    assert q.min() == 0 and q.max() <= (1 << 21) - 1
    # monotone in each coordinate: larger x never gets a smaller qx
    for a in range(3):
        o = np.argsort(p4[:, a], kind="stable")
        assert np.all(np.diff(q[o, a]) >= 0)
    # the axis of largest extent spans the full range
    ext = p4[:, :3].max(0).astype(np.float64) - p4[:, :3].min(0)
    a = int(np.argmax(ext))
    assert q[:, a].max() == (1 << 21) - 1


def test_keys_degenerate(oracle_lib):
    p4 = np.zeros((5, 4), np.float32)
    p4[:, :3] = 1.25
    key, box = oracle_lib.keys(p4)
    assert box[3] == 0.0 and np.all(key == 0)
    key, box = oracle_lib.keys(np.zeros((0, 4), np.float32))
    assert key.size == 0


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 65537])
def test_sort_is_stable_permutation(oracle_lib, n):
    rng = np.random.default_rng(n)
    key = rng.integers(0, 64, n).astype(np.uint64) << np.uint64(57)  # many ties
    key |= rng.integers(0, 4, n).astype(np.uint64)
    order, skey = oracle_lib.sort(key)
    ref = np.argsort(key, kind="stable")
    assert np.array_equal(order, ref.astype(np.uint32))
    assert np.array_equal(skey, key[ref])
    assert np.array_equal(np.sort(order), np.arange(n, dtype=np.uint32))


# ---------------------------------------------------------------- Peano-Hilbert keys (Sec. 2.1, App. A)
def _grid(o, side):
    r = np.arange(side)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    return g + np.asarray(o)


@pytest.mark.parametrize("origin", [(0, 0, 0), (8, 16, 24), (2**20, 2**19 + 8, 8)])
def test_hilbert_subcube_is_a_face_adjacent_run(oracle_lib, origin):
    """An aligned 8^3 block at full depth is one cell: its 512 keys are one contiguous
    range, and consecutive keys are face neighbours (a Morton order is not)."""
    O = oracle_lib
    pts = _grid(origin, 8)
    keys = np.array([O.hilbert3(int(x), int(y), int(z)) for x, y, z in pts], np.uint64)
    order = np.argsort(keys)
    ks = keys[order].astype(np.int64)
    assert ks[-1] - ks[0] == 511 and len(np.unique(ks)) == 512
    steps = np.abs(np.diff(pts[order], axis=0)).sum(1)
    assert np.all(steps == 1)
    mort = np.array([O.morton3(int(x), int(y), int(z)) for x, y, z in pts], np.uint64)
    assert np.any(np.abs(np.diff(pts[np.argsort(mort)], axis=0)).sum(1) != 1)


def test_hilbert_prefixes_name_the_cubes(oracle_lib):
    """The first 3l bits of a key identify the level-l cube, at every level."""
    O = oracle_lib
    rng = np.random.default_rng(3)
    pts = rng.integers(0, 2**21, (600, 3))
    keys = np.array([O.hilbert3(int(x), int(y), int(z)) for x, y, z in pts], np.uint64)
    for lvl in (1, 2, 4, 7, 12):
        cube = [tuple(p >> (21 - lvl)) for p in pts]
        pref = keys >> np.uint64(63 - 3 * lvl)
        by_cube = {}
        for c, k in zip(cube, pref):
            assert by_cube.setdefault(c, k) == k
        assert len(set(by_cube.values())) == len(by_cube)  # different cubes, different prefixes


def test_hilbert_coarse_cubes_are_face_adjacent_in_key_order(oracle_lib):
    O = oracle_lib
    cubes = _grid((0, 0, 0), 4)  # the 64 level-2 cubes, by their corner in units of 2^19
    keys = np.array([O.hilbert3(int(x) << 19, int(y) << 19, int(z) << 19) for x, y, z in cubes], np.uint64)
    pref = (keys >> np.uint64(57)).astype(np.int64)
    assert sorted(pref) == list(range(64))
    order = np.argsort(pref)
    assert np.all(np.abs(np.diff(cubes[order], axis=0)).sum(1) == 1)


def _hilbert_decode(h, bits=21):
    """Axes from a Hilbert index: de-interleave into the transposed form, then undo the
    Gray code and the rotations from the bottom bit up (the inverse of the encoder's
    steps, written independently here)."""
    x = [0, 0, 0]
    for b in range(bits):
        for a in range(3):
            x[a] |= ((h >> (3 * b + 2 - a)) & 1) << b
    n = 2 << (bits - 1)
    t = x[2] >> 1
    for i in (2, 1):
        x[i] ^= x[i - 1]
    x[0] ^= t
    q = 2
    while q != n:
        p = q - 1
        for i in (2, 1, 0):
            if x[i] & q:
                x[0] ^= p
            else:
                t = (x[0] ^ x[i]) & p
                x[0] ^= t
                x[i] ^= t
        q <<= 1
    return x


def test_hilbert_round_trip(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(8)
    for x, y, z in rng.integers(0, 2**21, (300, 3)):
        h = O.hilbert3(int(x), int(y), int(z))
        assert h < 2**63
        assert _hilbert_decode(h) == [int(x), int(y), int(z)]


def test_hilbert_tree_matches_morton_tree_as_sets(oracle_lib):
    """Both curves name the same cubes, so the trees hold the same cells (as particle
    sets per level); only the order of children and particles differs."""
    O = oracle_lib
    rng = np.random.default_rng(2)
    p4 = np.zeros((3000, 4), np.float32)
    p4[:, :3] = rng.normal(0, 1, (3000, 3))
    p4[:, 3] = 1.0 / 3000
    sets = []
    for curve in (0, 1):
        key, _ = O.keys(p4, curve)
        order, skey = O.sort(key)
        tree = O.build_tree(skey, 16)
        cells = set()
        for c in range(tree["n_nodes"]):
            f, k = int(tree["first"][c]), int(tree["count"][c])
            cells.add((int(tree["level"][c]), frozenset(order[f:f + k].tolist())))
        sets.append(cells)
    assert sets[0] == sets[1]
