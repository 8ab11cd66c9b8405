"""Pins of the oracle's MAC (Eqs. 2, 5-7), groups (Sec. 2.3) and tree walk."""
import numpy as np
import pytest

from paper_1610_07279_gb300 import ics


def _p4(n, seed=1, kind="plummer"):
    gen = ics.plummer if kind == "plummer" else ics.nfw
    pos, vel, m, eps = gen(n, seed=seed)
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = m
    return p4, eps


def _acc(oracle_lib, n=2048, seed=1, kind="plummer", **kw):
    O = oracle_lib
    p4, eps = _p4(n, seed, kind)
    prm = O.Params(eps=eps, **kw)
    return O, p4, prm


# ---------------------------------------------------------------- MAC by hand
def test_mac_opening_angle_boundary(oracle_lib):
    O = oracle_lib
    g = [0.0, 0.0, 0.0, 0.0]
    node = [2.0, 0.0, 0.0, 1.0]
    assert O.mac_accept(0, 0.5, 0, 0, 1, g, node, 1.0)             # b_J = theta d: accept
    assert not O.mac_accept(0, 0.5, 0, 0, 1, g, node, np.nextafter(np.float32(1), np.float32(2)))
    # pseudo i radius shortens the distance: d = lambda r = r - b_I (Eqs. 6-7)
    g2 = [0.0, 0.0, 0.0, 1.0]
    node3 = [3.0, 0.0, 0.0, 1.0]
    assert O.mac_accept(0, 0.5, 0, 0, 1, g2, node3, 1.0)            # d = 2
    assert not O.mac_accept(0, 0.5, 0, 0, 1, [0, 0, 0, 2.5], node3, 1.0)  # d = 0.5
    # b_I >= r: lambda = 0, only a point-like cell (b_J = 0) is accepted
    assert not O.mac_accept(0, 0.5, 0, 0, 1, [0, 0, 0, 3.0], node3, 1e-30)
    assert O.mac_accept(0, 0.5, 0, 0, 1, [0, 0, 0, 3.0], node3, 0.0)


def test_mac_acceleration_boundary(oracle_lib):
    O = oracle_lib
    # accept iff d^4 D_acc |a_old| >= G m_J b_J^2; with D_acc |a_old| = 1/16, m=b=G=1: d >= 2
    g = [0.0, 0.0, 0.0, 0.0]
    assert O.mac_accept(1, 0, 0.25, 0.25, 1.0, g, [2.0, 0, 0, 1.0], 1.0)
    below = float(np.nextafter(np.float32(2.0), np.float32(0)))
    assert not O.mac_accept(1, 0, 0.25, 0.25, 1.0, g, [below, 0, 0, 1.0], 1.0)
    # doubling G m_J b_J^2 needs d larger by 2^(1/4)
    assert not O.mac_accept(1, 0, 0.25, 0.25, 2.0, g, [2.0, 0, 0, 1.0], 1.0)
    assert O.mac_accept(1, 0, 0.25, 0.25, 2.0, g, [2.0 * 2 ** 0.25 * 1.000001, 0, 0, 1.0], 1.0)
    # |a_old| = 0 accepts only cells with b_J = 0 or m_J = 0
    assert not O.mac_accept(1, 0, 0.25, 0.0, 1.0, g, [100.0, 0, 0, 1.0], 1.0)
    assert O.mac_accept(1, 0, 0.25, 0.0, 1.0, g, [100.0, 0, 0, 1.0], 0.0)


# ---------------------------------------------------------------- groups
def _sorted_tree(O, n, seed, kind="nfw", leaf=16):
    p4, eps = _p4(n, seed=seed, kind=kind)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    return p4[order], O.build_tree(skey, leaf)


def _brute_group_starts(tree, n, active, gmax, bj=None, r_crit=0.0):
    """Recursive descent from the root: a cell is a group cell when it holds at most
    gmax actives and is a leaf or has b_J <= r_crit (no radius test when r_crit <= 0),
    or when it is a leaf; its actives are cut into runs of gmax."""
    pos = {int(a): k for k, a in enumerate(active)}
    act = np.zeros(n + 1, bool)
    act[active] = True
    out = []

    def rec(c):
        f, k = int(tree["first"][c]), int(tree["count"][c])
        mine = [pos[i] for i in range(f, f + k) if act[i]]
        if not mine:
            return
        small = len(mine) <= gmax and (r_crit <= 0 or bj[c] <= np.float32(r_crit))
        if small or tree["child"][c] < 0:
            out.extend(mine[::gmax])
            return
        for ch in range(tree["child"][c], tree["child"][c] + tree["nchild"][c]):
            rec(ch)

    if tree["n_nodes"]:
        rec(0)
    return np.array(sorted(out) + [len(active)], np.uint32)


@pytest.mark.parametrize("frac,gmax", [(1.0, 32), (0.3, 32), (0.05, 8), (1.0, 1)])
def test_group_starts_match_recursive_definition(oracle_lib, frac, gmax):
    O = oracle_lib
    n = 3000
    sp4, tree = _sorted_tree(O, n, 11)
    rng = np.random.default_rng(2)
    active = np.sort(rng.choice(n, max(1, int(frac * n)), replace=False)).astype(np.uint32)
    starts = O.group_starts(tree, n, active, gmax)
    assert np.array_equal(starts, _brute_group_starts(tree, n, active, gmax))
    assert starts[0] == 0 and starts[-1] == active.size and np.all(np.diff(starts.astype(int)) >= 1)
    assert np.all(np.diff(starts.astype(int)) <= gmax)


@pytest.mark.parametrize("frac,gmax", [(1.0, 32), (0.2, 64), (0.02, 16)])
def test_group_starts_with_rcrit_match_recursive_definition(oracle_lib, frac, gmax):
    """Sec. 2.4: a cell wider than r_crit is not one group even when it holds few actives."""
    O = oracle_lib
    n = 4000
    sp4, tree = _sorted_tree(O, n, 12)
    jpos, bj = O.pseudo_j(tree, sp4)
    rng = np.random.default_rng(3)
    active = np.sort(rng.choice(n, max(1, int(frac * n)), replace=False)).astype(np.uint32)
    base = O.group_starts(tree, n, active, gmax)
    inner = bj[tree["child"][:tree["n_nodes"]] >= 0]
    prev = len(base)
    for q in (1.0, 0.9, 0.6, 0.3, 0.0):
        r_crit = float(np.float32(np.quantile(inner, q))) if q > 0 else 1e-30
        starts = O.group_starts(tree, n, active, gmax, 1, bj, r_crit)
        assert np.array_equal(starts, _brute_group_starts(tree, n, active, gmax, bj, r_crit)), q
        assert len(starts) >= prev  # a tighter limit only splits groups
        prev = len(starts)
        assert starts[0] == 0 and starts[-1] == active.size and np.all(np.diff(starts.astype(int)) <= gmax)
    # no limit, and a limit above every radius, leave the groups of the cell rule unchanged
    assert np.array_equal(O.group_starts(tree, n, active, gmax, 1, bj, 0.0), base)
    assert np.array_equal(O.group_starts(tree, n, active, gmax, 1, bj, float(bj.max()) * 2), base)


def test_groups_enclose_members(oracle_lib):
    O = oracle_lib
    n = 4096
    sp4, tree = _sorted_tree(O, n, 3)
    rng = np.random.default_rng(0)
    active = np.sort(rng.choice(n, 1000, replace=False)).astype(np.uint32)
    aold = rng.uniform(0.1, 2.0, n).astype(np.float32)
    for mode, gmax in ((1, 32), (0, 7), (0, 64), (1, 5)):
        starts = O.group_starts(tree, n, active, gmax, mode)
        gI, gamin = O.groups(starts, active, sp4, aold)
        assert len(gI) == len(starts) - 1
        for g in range(len(gI)):
            mem = active[starts[g]:starts[g + 1]]
            pts = sp4[mem, :3]
            np.testing.assert_array_equal(gI[g, :3], np.float32(0.5) * (pts.min(0) + pts.max(0)))
            d = np.linalg.norm(pts.astype(np.float64) - gI[g, :3].astype(np.float64), axis=1)
            assert d.max() <= gI[g, 3] <= d.max() * (1 + 2.0 ** -18) + 1e-30
            assert gamin[g] == aold[mem].min()


def test_cell_groups_are_compact(oracle_lib):
    """Grouping by cells keeps every group inside one small cell (Sec. 2.4)."""
    O = oracle_lib
    n = 1 << 14
    sp4, tree = _sorted_tree(O, n, 5)
    active = np.arange(n, dtype=np.uint32)
    cells = O.group_starts(tree, n, active, 32, 1)
    runs = O.group_starts(tree, n, active, 32, 0)
    bc = O.groups(cells, active, sp4)[0][:, 3]
    br = O.groups(runs, active, sp4)[0][:, 3]
    assert bc.max() < 0.5 * br.max() and bc.mean() < br.mean()


# ---------------------------------------------------------------- walk
def _rel(a, b):
    return np.linalg.norm(a[:, :3] - b[:, :3], axis=1) / np.linalg.norm(b[:, :3], axis=1)


def test_theta_zero_equals_direct(oracle_lib):
    O, p4, prm = _acc(oracle_lib, 2048, seed=2)
    r = O.tree_force(p4, prm, mac=0, theta=0.0)
    d = O.direct(p4, prm.eps)[r["order"]]
    assert np.all(r["inter"] == 2048)
    np.testing.assert_allclose(r["acc"], d, rtol=1e-12, atol=1e-12)


def test_delta_acc_to_zero_equals_direct(oracle_lib):
    O, p4, prm = _acc(oracle_lib, 2048, seed=5, kind="nfw", delta_acc=1e-30)
    aold = np.ones(2048, np.float32)
    r = O.tree_force(p4, prm, aold=aold)
    d = O.direct(p4, prm.eps)[r["order"]]
    np.testing.assert_allclose(r["acc"], d, rtol=1e-12, atol=1e-12)


def test_error_decreases_with_theta(oracle_lib):
    O, p4, prm = _acc(oracle_lib, 4096, seed=1)
    d = O.direct(p4, prm.eps)
    meds, inters = [], []
    for th in (0.9, 0.7, 0.5, 0.3, 0.1):
        r = O.tree_force(p4, prm, mac=0, theta=th)
        meds.append(np.median(_rel(r["acc"], d[r["order"]])))
        inters.append(r["inter"].mean())
    assert all(a > b for a, b in zip(meds, meds[1:]))
    assert all(a < b for a, b in zip(inters, inters[1:]))
    # the paper's typical accuracy, ~1e-3 for theta 0.5-0.7 (an order-of-magnitude band:
    # the groups here are tighter cells, so a given theta accepts a little more)
    assert 1e-4 < meds[2] < 5e-3 and 1e-4 < meds[1] < 5e-3


def test_acceleration_mac_accuracy_band(oracle_lib):
    O, p4, prm = _acc(oracle_lib, 4096, seed=1)
    d = O.direct(p4, prm.eps)
    aold = O.bootstrap_aold(p4, prm)
    errs = []
    for k in (5, 7, 9, 11):
        prm.delta_acc = 2.0 ** -k
        r = O.tree_force(p4, prm, aold=aold)
        errs.append(np.median(_rel(r["acc"], d[r["order"]])))
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert 1e-4 < errs[1] < 3e-3   # Delta_acc = 2^-7, the paper's fiducial value


def test_walk_sampled_groups_equal_full(oracle_lib):
    O, p4, prm = _acc(oracle_lib, 3000, seed=8, kind="nfw")
    aold = O.bootstrap_aold(p4, prm)
    full = O.tree_force(p4, prm, aold=aold)
    gids = np.array([0, 5, 17, len(full["gI"]) - 1])
    part = O.tree_force(p4, prm, aold=aold, group_ids=gids)
    st = full["starts"]
    for g in gids:
        sl = slice(st[g], st[g + 1])
        np.testing.assert_array_equal(part["acc"][sl], full["acc"][sl])
        np.testing.assert_array_equal(part["inter"][sl], full["inter"][sl])


def test_walk_single_and_empty(oracle_lib):
    O = oracle_lib
    prm = O.Params(eps=0.1)
    p4 = np.array([[1.0, 2.0, 3.0, 0.5]], np.float32)
    r = O.tree_force(p4, prm, aold=np.ones(1, np.float32))
    assert np.all(r["acc"] == 0.0) and r["inter"][0] == 1
    r = O.tree_force(np.zeros((0, 4), np.float32), prm)
    assert r["acc"].shape == (0, 4)


def _seb_radius(pts, iters=4000):
    """Smallest enclosing ball by Badoiu-Clarkson: step towards the farthest point by
    1/(k+1); the radius converges to the optimum (error ~ 1/sqrt(iters))."""
    c = pts.mean(0)
    for k in range(iters):
        far = pts[np.argmax(((pts - c) ** 2).sum(1))]
        c = c + (far - c) / (k + 1.0)
    return np.sqrt(((pts - c) ** 2).sum(1).max())


def _one_group_sphere(O, pts, sphere):
    n = len(pts)
    sp4 = np.zeros((n, 4), np.float32)
    sp4[:, :3] = pts
    active = np.arange(n, dtype=np.uint32)
    gI, _ = O.groups(np.array([0, n], np.uint32), active, sp4, None, sphere)
    return gI[0]


def test_ebs_sphere_special_cases(oracle_lib):
    """Appendix B, Ritter's efficient bounding sphere: exact on a segment (two points,
    collinear points), near the circumscribed sphere for points on a sphere, always
    enclosing, and no worse than the box-centred (GEO) sphere there."""
    O = oracle_lib
    two = np.array([[0.25, -1.0, 2.0], [1.25, 0.5, -1.0]], np.float32)
    s = _one_group_sphere(O, two, 1)
    half = 0.5 * np.linalg.norm(two[1].astype(np.float64) - two[0])
    np.testing.assert_allclose(s[:3], 0.5 * (two[0] + two[1]), rtol=0, atol=1e-6)
    assert half <= s[3] <= half * (1 + 2e-6)
    t = np.linspace(0, 1, 23)[:, None]
    line = (np.array([1.0, 2.0, -0.5]) + t * np.array([2.0, -1.0, 0.25])).astype(np.float32)
    s = _one_group_sphere(O, line, 1)
    half = 0.5 * np.linalg.norm(line[-1].astype(np.float64) - line[0])
    assert half <= s[3] <= half * (1 + 1e-5)
    rng = np.random.default_rng(4)
    worse = []
    for _ in range(20):
        v = rng.normal(size=(48, 3))
        pts = (3.0 + 2.0 * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
        se, sg = _one_group_sphere(O, pts, 1), _one_group_sphere(O, pts, 0)
        d = np.linalg.norm(pts.astype(np.float64) - se[:3].astype(np.float64), axis=1)
        assert d.max() <= se[3]
        assert se[3] <= 2.0 * 1.15  # within 15 % of the circumscribed radius
        worse.append(se[3] / sg[3])
    assert np.median(worse) <= 1.02


def _seb_radius(pts, iters=4000):
    """Smallest enclosing ball by Badoiu-Clarkson: step towards the farthest point by
    1/(k+1); the radius converges to the optimum (error ~ 1/sqrt(iters))."""
    c = pts.mean(0)
    for k in range(iters):
        far = pts[np.argmax(((pts - c) ** 2).sum(1))]
        c = c + (far - c) / (k + 1.0)
    return np.sqrt(((pts - c) ** 2).sum(1).max())


def test_ebs_and_geo_spheres_against_the_smallest_ball(oracle_lib):
    """Both pseudo i-particle spheres enclose their group and stay within ~1.5x of the
    smallest enclosing ball on tree-cell groups (the paper reports ~1.1-1.15 on its
    groups; cell-bounded groups are compact)."""
    O = oracle_lib
    n = 8192
    sp4, tree = _sorted_tree(O, n, 21)
    active = np.arange(n, dtype=np.uint32)
    starts = O.group_starts(tree, n, active, 64, 1)
    rng = np.random.default_rng(1)
    for sphere in (0, 1):
        gI, _ = O.groups(starts, active, sp4, None, sphere)
        ratios = []
        for g in rng.choice(len(starts) - 1, 40, replace=False):
            mem = active[starts[g]:starts[g + 1]]
            if len(mem) < 4:
                continue
            pts = sp4[mem, :3].astype(np.float64)
            d = np.linalg.norm(pts - gI[g, :3].astype(np.float64), axis=1)
            assert d.max() <= gI[g, 3]
            ratios.append(gI[g, 3] / _seb_radius(pts))
        assert min(ratios) >= 0.999 and np.median(ratios) < 1.2 and max(ratios) < 1.6, (sphere, ratios)


# ---------------------------------------------------------------- multipole MAC (Sec. 2.2)
def test_b2_moments_match_their_definition(oracle_lib):
    """B_2 of every cell equals sum over its particles of m |r - r_J|^2 (FP64 reference);
    the cell value is built from its children by parallel axes."""
    O = oracle_lib
    n = 4096
    sp4, tree = _sorted_tree(O, n, 9)
    jpos, bj, b2 = O.pseudo_j(tree, sp4, with_b2=True)
    assert np.all(b2 >= 0)
    pts = sp4[:, :3].astype(np.float64)
    m = sp4[:, 3].astype(np.float64)
    for c in range(tree["n_nodes"]):
        f, k = int(tree["first"][c]), int(tree["count"][c])
        ref = (m[f:f + k] * ((pts[f:f + k] - jpos[c, :3].astype(np.float64)) ** 2).sum(1)).sum()
        if k == 1:
            assert b2[c] == 0.0
        else:
            assert abs(b2[c] - ref) <= 1e-4 * ref + 1e-30, (c, b2[c], ref)


def test_multipole_mac_boundary_cases(oracle_lib):
    O = oracle_lib
    gI = np.array([0.0, 0.0, 0.0, 0.0], np.float32)
    # b_J = 2, B_2 = 1, Delta_mul = 3: threshold 1 + sqrt(1 + 1) = 2.41421356...
    thr = 1.0 + np.sqrt(1.0 + np.sqrt(3.0 * 1.0 / 3.0))
    far = np.array([np.float32(thr) * 1.001, 0, 0, 1.0], np.float32)
    near = np.array([np.float32(thr) * 0.999, 0, 0, 1.0], np.float32)
    assert O.mac_accept(2, 0.5, 3.0, 1.0, 1.0, gI, far, 2.0, 1.0)
    assert not O.mac_accept(2, 0.5, 3.0, 1.0, 1.0, gI, near, 2.0, 1.0)
    # a point mass (b_J = 0, B_2 = 0) is accepted at any distance, even inside b_I = 0
    assert O.mac_accept(2, 0.5, 1e-6, 1.0, 1.0, gI, np.array([1e-3, 0, 0, 1.0], np.float32), 0.0, 0.0)


def test_multipole_mac_limits(oracle_lib):
    """Delta_mul -> 0 opens every cell with B_2 > 0: direct summation; the error falls
    monotonically as Delta_mul decreases."""
    O, p4, prm = _acc(oracle_lib, 2048, seed=6, kind="nfw", delta_acc=1e-30)
    r = O.tree_force(p4, prm, mac=2)
    d = O.direct(p4, prm.eps)[r["order"]]
    np.testing.assert_allclose(r["acc"], d, rtol=1e-12, atol=1e-12)
    O, p4, prm = _acc(oracle_lib, 4096, seed=3, kind="nfw")
    d = O.direct(p4, prm.eps)
    meds = []
    for k in (2, 6, 10, 14):
        prm.delta_acc = 2.0 ** -k
        r = O.tree_force(p4, prm, mac=2)
        meds.append(np.median(_rel(r["acc"], d[r["order"]])))
    assert all(meds[i + 1] < meds[i] for i in range(len(meds) - 1)), meds
