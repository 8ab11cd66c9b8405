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
