"""Pins of the oracle's block time step (Sec. 1; Sec. 2.7, Eqs. 15-19)."""
import math

import numpy as np
import pytest

from paper_1610_07279_gb300 import ics


def test_level_from_a2_brute_force(oracle_lib):
    """Smallest k with dt_max 2^-k <= dt_i = sqrt(c/|a|), c = 2 eta eps, decided exactly
    (rational arithmetic on the FP64 inputs: dt_k^4 |a|^2 <= c^2, c^2 rounded once)."""
    from fractions import Fraction as Fr
    O = oracle_lib
    eta, eps, M, L = 0.025, 0.01, 2, 8
    c = (2.0 * eta) * eps
    c2 = Fr(c * c)
    rng = np.random.default_rng(3)
    a2s = list(10.0 ** rng.uniform(-12, 6, 3000)) + [0.0, 1e300]
    # values sitting exactly on level boundaries: |a|^2 = c2 / dt_k^4
    a2s += [float(c2 / Fr(2) ** (4 * (M - k))) for k in range(L)]
    for a2 in a2s:
        want = 0
        if a2 > 0:
            want = next((k for k in range(L) if Fr(2) ** (4 * (M - k)) * Fr(a2) <= c2), L - 1)
        assert O.level_from_a2(a2, eta, eps, M, L) == want, a2


def test_dtmax_exponent_brute_force(oracle_lib):
    from fractions import Fraction as Fr
    O = oracle_lib
    eta, eps = 0.025, 1.0 / 64
    c2 = Fr(((2.0 * eta) * eps) ** 2)
    rng = np.random.default_rng(4)
    for _ in range(300):
        acc = np.zeros((5, 4), np.float32)
        acc[:, :3] = (rng.standard_normal((5, 3)) * 10.0 ** rng.uniform(-6, 3)).astype(np.float32)
        a2 = O.a2(acc)
        a2min = Fr(float(a2[a2 > 0].min()))
        # largest M with 2^M <= dt_i of the particle with the smallest |a|
        M = max(m for m in range(-80, 80) if Fr(2) ** (4 * m) * a2min <= c2)
        assert O.dtmax_exponent(acc, eta, eps) == M


def _one(O, kold, kc_amag, T, t0, L=6, M=0, eta=0.025, eps=0.01):
    r0 = np.zeros((1, 3))
    vh = np.zeros((1, 3))
    t0a = np.array([t0], np.int64)
    lv = np.array([kold], np.uint8)
    ao = np.zeros(1, np.float32)
    acc = np.array([[kc_amag, 0, 0, 0]], np.float32)
    O.correct(np.array([0], np.uint32), acc, T, math.ldexp(1.0, M), M, L, eta, eps, r0, vh, t0a, lv, ao)
    return int(lv[0]), int(t0a[0])


def _amag_for_level(k, M=0, eta=0.025, eps=0.01):  # |a| whose dt_i is 1.5 dt_k
    dti = 1.5 * math.ldexp(1.0, int(M) - int(k))  # level k holds dt in [dt_k, 2 dt_k)
    return float(np.float32((2.0 * eta) * eps / (dti * dti)))


def test_level_change_rules(oracle_lib):
    O = oracle_lib
    L = 6  # ticks(k) = 2^(5-k)
    # a shorter step is always taken, whatever T
    assert _one(O, 2, _amag_for_level(4), T=8 + 8, t0=8) == (4, 16)
    # a longer step only by one level, and only when T is a multiple of the longer step
    assert _one(O, 3, _amag_for_level(1), T=8, t0=4) == (2, 8)      # 8 % ticks(2)=8 == 0
    assert _one(O, 3, _amag_for_level(1), T=12, t0=8) == (3, 12)    # 12 % 8 != 0: stay
    assert _one(O, 0, _amag_for_level(0), T=32, t0=0) == (0, 32)
    assert _one(O, 5, _amag_for_level(5), T=33, t0=32) == (5, 33)


def test_active_counts_closed_form(oracle_lib):
    """Fixed levels: the active count at tick T is sum_k n_k [T mod 2^(L-1-k) == 0]."""
    O = oracle_lib
    L, M = 5, 0
    n_k = [3, 5, 7, 11, 13]
    level = np.repeat(np.arange(L), n_k).astype(np.uint8)
    n = level.size
    amg = np.array([_amag_for_level(k, M) for k in level], np.float32)
    acc = np.zeros((n, 4), np.float32)
    acc[:, 0] = amg
    r0 = np.zeros((n, 3))
    vh = np.zeros((n, 3))
    t0 = np.zeros(n, np.int64)
    aold = np.zeros(n, np.float32)
    ticks = lambda lv: np.left_shift(1, (L - 1 - lv.astype(np.int64)))
    seen = []
    for _ in range(40):
        T = int((t0 + ticks(level)).min())
        active = np.nonzero(t0 + ticks(level) == T)[0].astype(np.uint32)
        want = sum(nk for k, nk in enumerate(n_k) if T % (1 << (L - 1 - k)) == 0)
        assert active.size == want
        O.correct(active, acc[active], T, 1.0, M, L, 0.025, 0.01, r0, vh, t0, level, aold)
        seen.append(T)
    assert seen == list(range(1, 41))
    assert np.array_equal(level, np.repeat(np.arange(L), n_k))


def test_shared_step_reduces_to_leapfrog(oracle_lib):
    """L = 1 (one shared, fixed step): the block-step scheme is the KDK leap-frog (Sec. 2.7);
    the reference here uses separate multiplies and adds, the scheme fused ones, so the two
    agree to rounding."""
    O = oracle_lib
    n = 512
    pos, vel, m, eps = ics.plummer(n, seed=21)
    prm = O.Params(eps=eps, mac=0, theta=0.5, levels=1, dt_max=2.0 ** -6)
    sim = O.BlockStepSim(pos, vel, m, prm)
    sim.start()

    def force(r):
        p4 = np.zeros((n, 4), np.float32)
        p4[:, :3] = r
        p4[:, 3] = m
        res = O.tree_force(p4, prm, mac=0)
        a = np.empty((n, 4), np.float32)
        a[res["order"]] = res["acc"].astype(np.float32)
        return a[:, :3].astype(np.float64)

    dt = 2.0 ** -6
    r = pos.copy()
    a = force(r)
    vh = vel + (0.5 * dt) * a
    for step in range(6):
        sim.step()
        r = r + dt * vh
        a = force(r)
        v = vh + (0.5 * dt) * a
        vh = v + (0.5 * dt) * a
        back = np.empty_like(sim.r0)
        back[sim.id] = sim.r0
        np.testing.assert_allclose(back, r, rtol=1e-13, atol=1e-15)
        bv = np.empty_like(sim.vh)
        bv[sim.id] = sim.vh
        np.testing.assert_allclose(bv, vh, rtol=1e-11, atol=1e-14)
        assert sim.T == step + 1


def test_kepler_orbit(oracle_lib):
    """Two equal bodies on a circular orbit: one period 2 pi returns them, energy kept."""
    O = oracle_lib
    pos = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    vel = np.array([[0.0, 0.5, 0.0], [0.0, -0.5, 0.0]])
    m = np.array([0.5, 0.5], np.float32)
    dt = 2.0 ** -8
    prm = O.Params(eps=2.0 ** -20, mac=0, theta=0.5, levels=1, dt_max=dt)
    sim = O.BlockStepSim(pos, vel, m, prm)
    sim.start()

    def energy():
        v = sim.vh - (0.5 * dt) * sim.acc[:, :3].astype(np.float64)
        r = np.linalg.norm(sim.r0[0] - sim.r0[1])
        return 0.5 * float((m.astype(np.float64) * (v * v).sum(1)).sum()) - 0.25 / r

    e0 = energy()
    nsteps = int(round(2.0 * math.pi / dt))
    emax = 0.0
    for _ in range(nsteps):
        sim.step()
        emax = max(emax, abs(energy() - e0))
    assert emax < 1e-4 * abs(e0)
    back = np.empty_like(sim.r0)
    back[sim.id] = sim.r0
    # after one period the bodies are back where they started (to O(dt))
    assert np.linalg.norm(back - pos) < 2e-2


def test_block_step_runs_and_levels_spread(oracle_lib):
    O = oracle_lib
    pos, vel, m, eps = ics.nfw(4096, seed=2)
    prm = O.Params(eps=eps, levels=6)
    sim = O.BlockStepSim(pos, vel, m, prm)
    sim.start()
    assert len(np.unique(sim.level)) >= 3
    Ts = [sim.step()["T"] for _ in range(8)]
    assert all(b > a for a, b in zip(Ts, Ts[1:]))
    assert np.all(sim.t0 <= sim.T)
    assert np.all((sim.t0 % np.left_shift(1, (prm.levels - 1 - sim.level.astype(np.int64)))) == 0)


def test_tree_reused_between_rebuilds(oracle_lib):
    """Sec. 2.6: between builds the order and topology are kept; the pseudo j-particles
    follow the predicted particles, so every particle stays inside its ancestors'
    spheres and the forces keep the tree accuracy against direct summation."""
    O = oracle_lib
    n = 3000
    pos, vel, mass, eps = ics.plummer(n, seed=41)
    prm = O.Params(eps=O.f32(eps), levels=4, rebuild_every=4)
    sim = O.BlockStepSim(pos, vel, mass, prm)
    sim.start()
    prev = None
    for k in range(9):
        r = sim.step()
        if k % 4 != 0:
            assert r["tree"] is prev["tree"] and np.array_equal(r["order"], np.arange(n))
            assert np.array_equal(r["skey"], prev["skey"])
        prev = r
        p4 = O.predict(sim.r0, sim.vh, sim.t0, sim.mass, sim.T, float(np.ldexp(sim.dt_max, -(sim.L - 1))))
        tree = r["tree"]
        jpos, bj = O.pseudo_j(tree, p4)
        for c in range(0, tree["n_nodes"], 7):  # enclosure by the refreshed spheres
            f, cnt = int(tree["first"][c]), int(tree["count"][c])
            d = np.linalg.norm(p4[f:f + cnt, :3].astype(np.float64) - jpos[c, :3].astype(np.float64), axis=1)
            assert d.max() <= bj[c] * (1 + 1e-6) + 1e-12
        act = r["active"]
        ref = O.direct(p4, prm.eps, prm.G, idx=act.astype(np.int64))
        rel = np.linalg.norm(r["acc"][:, :3] - ref[:, :3], axis=1) / np.linalg.norm(ref[:, :3], axis=1)
        assert np.median(rel) < 5e-3, (k, np.median(rel))
