"""Pins of the oracle's octree (Sec. 2.1) and pseudo j-particles (Sec. 2.1, Fig. 1)."""
import numpy as np
import pytest

from paper_1610_07279_gb300 import ics


def _sorted_system(n, seed=1, kind="plummer"):
    gen = ics.plummer if kind == "plummer" else ics.nfw
    pos, vel, m, eps = gen(n, seed=seed)
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = m
    return p4


def brute_tree(skey, leaf_max):
    """Depth-first recursive octree, renumbered afterwards by (level, first)."""
    nodes = []

    def rec(first, count, level, parent):
        me = len(nodes)
        nodes.append({"level": level, "first": first, "count": count, "parent": parent, "kids": []})
        if count > leaf_max and level < 21:
            shift = 3 * (20 - level)
            digits = [(int(k) >> shift) & 7 for k in skey[first:first + count]]
            s = 0
            for d in range(8):
                c = sum(1 for x in digits if x == d)
                if c:
                    nodes[me]["kids"].append(rec(first + s, c, level + 1, me))
                    s += c
            assert s == count
        return me

    if len(skey):
        rec(0, len(skey), 0, -1)
    perm = sorted(range(len(nodes)), key=lambda k: (nodes[k]["level"], nodes[k]["first"]))
    new = {old: i for i, old in enumerate(perm)}
    out = {"first": [], "count": [], "level": [], "parent": [], "child": [], "nchild": []}
    for old in perm:
        nd = nodes[old]
        kids = sorted(new[k] for k in nd["kids"])
        if kids:
            assert kids == list(range(kids[0], kids[0] + len(kids)))  # contiguous children
        out["first"].append(nd["first"])
        out["count"].append(nd["count"])
        out["level"].append(nd["level"])
        out["parent"].append(-1 if nd["parent"] < 0 else new[nd["parent"]])
        out["child"].append(kids[0] if kids else -1)
        out["nchild"].append(len(kids))
    return {k: np.array(v) for k, v in out.items()}


@pytest.mark.parametrize("n,leaf", [(1, 16), (2, 1), (17, 16), (1000, 16), (1024, 8), (777, 3)])
def test_build_matches_brute_force(oracle_lib, n, leaf):
    O = oracle_lib
    p4 = _sorted_system(n, seed=n)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    tree = O.build_tree(skey, leaf)
    ref = brute_tree(skey, leaf)
    assert tree["n_nodes"] == len(ref["first"])
    for k in ("first", "count", "level", "parent", "child", "nchild"):
        assert np.array_equal(tree[k].astype(np.int64), ref[k].astype(np.int64)), k


def test_build_coincident_particles_reach_level_21(oracle_lib):
    O = oracle_lib
    skey = np.zeros(40, np.uint64)
    tree = O.build_tree(skey, 16)
    assert tree["n_nodes"] == 22
    assert list(tree["level"]) == list(range(22))
    assert tree["child"][-1] == -1 and tree["count"][-1] == 40
    assert np.all(tree["nchild"][:-1] == 1)


def test_build_invariants(oracle_lib):
    O = oracle_lib
    p4 = _sorted_system(1 << 14, seed=2, kind="nfw")
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    leaf = 16
    t = O.build_tree(skey, leaf)
    nn = t["n_nodes"]
    leaves = t["child"] < 0
    # every particle sits in exactly one leaf
    cover = np.zeros(len(skey), np.int64)
    for f, c in zip(t["first"][leaves], t["count"][leaves]):
        cover[f:f + c] += 1
    assert np.all(cover == 1)
    # leaves are small unless at the deepest level; internal cells are large
    assert np.all((t["count"][leaves] <= leaf) | (t["level"][leaves] == 21))
    assert np.all(t["count"][~leaves] > leaf)
    # children partition their parent's range in order
    for c in np.nonzero(~leaves)[0]:
        k0, k1 = t["child"][c], t["child"][c] + t["nchild"][c]
        assert t["first"][k0] == t["first"][c]
        assert np.all(t["first"][k0 + 1:k1] == t["first"][k0:k1 - 1] + t["count"][k0:k1 - 1])
        assert t["count"][k0:k1].sum() == t["count"][c]
        assert np.all(t["parent"][k0:k1] == c) and np.all(t["level"][k0:k1] == t["level"][c] + 1)
    # level-major numbering, ordered by first within a level
    lv = t["level"].astype(np.int64)
    assert np.all(np.diff(lv) >= 0)
    same = np.diff(lv) == 0
    assert np.all(np.diff(t["first"].astype(np.int64))[same] > 0)
    ls = t["level_start"]
    for l in range(22):
        assert np.all(lv[ls[l]:ls[l + 1]] == l)
    assert ls[-1] == nn


def test_pseudo_j_invariants(oracle_lib):
    O = oracle_lib
    n = 1 << 13
    p4 = _sorted_system(n, seed=4)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = p4[order]
    t = O.build_tree(skey, 16)
    jpos, bj = O.pseudo_j(t, sp4)
    # equal power-of-two masses: the root mass is exact
    assert jpos[0, 3] == np.float32(sp4[:, 3].astype(np.float64).sum())
    # root COM = system COM (FP64), within the FP32 quotient's rounding (<= 1.5 ulp)
    com = (sp4[:, 3:4].astype(np.float64) * sp4[:, :3]).sum(0) / sp4[:, 3].astype(np.float64).sum()
    assert np.all(np.abs(jpos[0, :3] - com) <= 2 * np.spacing(np.abs(com).astype(np.float32)) + 1e-12)
    # every particle lies inside the b_J sphere of every cell that holds it
    for c in range(t["n_nodes"]):
        f, k = t["first"][c], t["count"][c]
        d = np.linalg.norm(sp4[f:f + k, :3].astype(np.float64) - jpos[c, :3].astype(np.float64), axis=1)
        assert d.max() <= bj[c]
    # single-particle cells: r_J is the particle, b_J = 0
    one = t["count"] == 1
    assert np.all(bj[one] == 0)
    assert np.array_equal(jpos[one, :3], sp4[t["first"][one], :3])
    # a leaf's b_J is its largest particle distance widened by ~2^-20 (tight)
    leaves = np.nonzero(t["child"] < 0)[0]
    for c in leaves[:500]:
        f, k = t["first"][c], t["count"][c]
        d = np.linalg.norm(sp4[f:f + k, :3].astype(np.float64) - jpos[c, :3].astype(np.float64), axis=1)
        assert d.max() <= bj[c] <= d.max() * (1 + 2.0 ** -18) + 1e-30


def test_pseudo_j_com_per_cell(oracle_lib):
    """Each cell's (m_J, r_J) equals its particles' FP64 mass and COM, to FP32 rounding."""
    O = oracle_lib
    p4 = _sorted_system(3000, seed=9, kind="nfw")
    p4[:, 3] *= np.random.default_rng(1).uniform(0.5, 1.5, 3000).astype(np.float32)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = p4[order]
    t = O.build_tree(skey, 8)
    jpos, bj = O.pseudo_j(t, sp4)
    for c in range(t["n_nodes"]):
        f, k = t["first"][c], t["count"][c]
        m = sp4[f:f + k, 3].astype(np.float64)
        M = m.sum()
        com = (m[:, None] * sp4[f:f + k, :3]).sum(0) / M
        assert abs(jpos[c, 3] - M) <= np.spacing(np.float32(M))
        assert np.all(np.abs(jpos[c, :3] - com) <= 2 * np.spacing(np.abs(com).astype(np.float32)) + 1e-15)


@pytest.mark.parametrize("kind,n,leaf", [("plummer", 4000, 1), ("nfw", 6000, 2), ("plummer", 1 << 13, 16)])
def test_pseudo_j_cell_radius_is_tight(oracle_lib, kind, n, leaf):
    """Sec. 2.1, Fig. 1: an upper bound on a cell's b_J from geometry alone.

    Let D_J be the largest distance of the cell's particles from r_J (brute force).  A
    child's centre of mass lies in the convex hull of its particles, so its distance
    from r_J is at most D_J; a sphere of radius b_c about it holds the child.  The child
    bound therefore satisfies D_J <= b_J <= D_J + max_c b_c: a radius summed over the
    children, taken about another centre, or built without the children's own radii
    breaks one side.  Where every child is a single particle (b_c = 0) the bound is
    exact.  Every child's sphere also lies inside its parent's.  Tolerances: FP32
    roundings (a few ulp per level) and the 2^-20 widening per level."""
    O = oracle_lib
    p4 = _sorted_system(n, seed=n + 5, kind=kind)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = p4[order].astype(np.float64)
    t = O.build_tree(skey, leaf)
    jpos, bj = O.pseudo_j(t, p4[order])
    jp = jpos.astype(np.float64)
    b = bj.astype(np.float64)
    scale = np.abs(sp4[:, :3]).max()
    slack = 64 * np.spacing(np.float32(scale))  # a few FP32 roundings of a coordinate
    internal = np.nonzero(t["child"] >= 0)[0]
    assert len(internal) > 10
    exact = 0
    for c in internal:
        f, k = t["first"][c], t["count"][c]
        D = np.linalg.norm(sp4[f:f + k, :3] - jp[c, :3], axis=1).max()
        kids = np.arange(t["child"][c], t["child"][c] + t["nchild"][c])
        bmax = b[kids].max()
        assert D <= b[c]
        assert b[c] <= (D + bmax) * (1 + 2.0 ** -17) + slack, (c, b[c], D, bmax)
        # nesting: |r_c - r_J| + b_c <= b_J
        dc = np.linalg.norm(jp[kids, :3] - jp[c, :3], axis=1)
        assert np.all(dc + b[kids] <= b[c] * (1 + 2.0 ** -20) + slack)
        if bmax == 0.0:
            exact += 1
            assert b[c] <= D * (1 + 2.0 ** -18) + slack
    if leaf <= 2:
        assert exact > 10  # the exact case is exercised


def test_pseudo_j_radius_bound_catches_a_summed_radius(oracle_lib):
    """The bound above rejects a plausible mistake: summing the children's reach instead
    of taking its maximum (checked on the oracle's own tree with a planted error)."""
    O = oracle_lib
    p4 = _sorted_system(3000, seed=11)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = p4[order].astype(np.float64)
    t = O.build_tree(skey, 2)
    jpos, bj = O.pseudo_j(t, p4[order])
    jp = jpos.astype(np.float64)
    bad = 0
    for c in np.nonzero(t["child"] >= 0)[0][-200:]:
        f, k = t["first"][c], t["count"][c]
        D = np.linalg.norm(sp4[f:f + k, :3] - jp[c, :3], axis=1).max()
        kids = np.arange(t["child"][c], t["child"][c] + t["nchild"][c])
        reach = np.linalg.norm(jp[kids, :3] - jp[c, :3], axis=1) + bj[kids]
        summed = reach.sum()
        if summed > (D + bj[kids].max()) * (1 + 2.0 ** -17) + 1e-6:
            bad += 1
    assert bad > 50
