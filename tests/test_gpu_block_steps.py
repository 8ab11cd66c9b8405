"""Block time steps on the GPU against the oracle's block-step driver (Sec. 1; Sec. 2.6;
Sec. 2.7, Eqs. 15-17), at the sizes of the paper-like workloads.

Two ways of running the same steps:

* Teacher-forced.  Before every block step both sides hold the oracle's state (the GPU
  is loaded with gt_set_state + gt_set_integrator_state).  Then keys, sort order, tree,
  pseudo j-particles, block time T, active set and interaction count must agree bit for
  bit, the accelerations within 1e-5 (median) / 1e-4 (99th percentile) of the oracle's
  FP64 sums over the same lists, and the correction driven by the oracle's own forces
  (gt_correct) must give the oracle's state bit for bit.  The GPU's own correction (FP32
  forces) may put a few particles on another level; that fraction is reported.
* Free-running.  Both sides integrate on their own from the same start; the fractions of
  active particles and of levels that differ are reported and bounded.

The oracle's start-up (an opening-angle pass whose |a| seeds a_old, then the
acceleration pass) gives both sides the same a_old.
"""
import numpy as np
import pytest

from paper_1610_07279_gb300 import ics

pytestmark = pytest.mark.gpu

MED_TOL, P99_TOL = 1e-5, 1e-4


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


def _p4(pos, mass):
    p4 = np.zeros((len(mass), 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    return p4


def _params(g, eps, **kw):
    prm = g.gt_default_params()
    prm.eps = eps
    prm.group_mode = g.GT_GROUP_CELLS  # a fixed group size on both sides
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def _oparams(O, prm):
    return O.Params(mac=prm.mac, theta=prm.theta, delta_acc=prm.delta_acc, eps=prm.eps, G=prm.G,
                    leaf_max=prm.leaf_max, group_max=prm.group_max, levels=prm.levels, eta=prm.eta,
                    dt_max=prm.dt_max, group_mode=prm.group_mode & 0xff, r_crit=max(prm.r_crit, 0.0),
                    rebuild_every=max(prm.rebuild_every, 1), key_curve=prm.key_curve)


def _rel(a, r):
    a = np.asarray(a, np.float64)
    num = np.linalg.norm(a[:, :3] - r[:, :3], axis=1)
    den = np.linalg.norm(r[:, :3], axis=1)
    out = np.full(num.shape, np.inf)
    ok = den > 0
    out[ok] = num[ok] / den[ok]
    out[(den == 0) & (num == 0)] = 0.0
    return out


def _load(s, sim, pre):
    s.set_state(pre["r0"], pre["vh"], pre["mass"])
    s.set_integrator_state(pre["level"], pre["t0"], pre["aold"], pre["acc"], sim.dt_max, pre["T"])


def _snapshot(sim):
    return {"r0": sim.r0.copy(), "vh": sim.vh.copy(), "mass": sim.mass.copy(), "level": sim.level.copy(),
            "t0": sim.t0.copy(), "aold": sim.aold.copy(), "acc": sim.acc.copy(), "T": int(sim.T)}


def teacher_forced(env, pos, vel, mass, prm, nsteps, tag, full_tree=True):
    """Runs nsteps teacher-forced block steps; returns per-step reports."""
    torch, g, O = env
    n = len(mass)
    oprm = _oparams(O, prm)
    sim = O.BlockStepSim(pos, vel, mass, oprm)
    boot = O.bootstrap_aold(_p4(pos, mass), oprm)
    sim.start(aold_boot=boot)
    s = g.System(n, prm)
    reports = []
    for k in range(nsteps):
        pre = _snapshot(sim)
        _load(s, sim, pre)
        i0 = s.stats()["interactions"]
        s.block_step()
        r = sim.step()
        st = s.stats()
        assert st["T"] == r["T"], (tag, k, st["T"], r["T"])
        # A1-A5 on the predicted positions
        t = s.get_tree()
        assert np.array_equal(t["keys"], r["skey"]), (tag, k, "keys")
        assert np.array_equal(t["order"], r["order"]), (tag, k, "order")
        tr = r["tree"]
        assert t["n_nodes"] == tr["n_nodes"], (tag, k, "nodes")
        if full_tree:
            for f in ("first", "count", "child"):
                assert np.array_equal(t[f], tr[f]), (tag, k, f)
        assert np.array_equal(t["jpos"].view(np.uint32), r["jpos"].view(np.uint32)), (tag, k, "jpos")
        assert np.array_equal(t["bj"].view(np.uint32), r["bj"].view(np.uint32)), (tag, k, "bj")
        # A6: the active set; A7: the same interaction lists, forces within tolerance
        act = s.get_active()
        assert np.array_equal(act, r["active"]), (tag, k, "active")
        assert st["interactions"] - i0 == int(r["inter"].sum()), (tag, k, "interactions")
        gs = s.get_state()
        assert np.array_equal(gs["id"], r["order"])
        rel = _rel(gs["acc"][act], r["acc"])
        prel = np.abs(gs["acc"][act, 3] - r["acc"][:, 3]) / np.abs(r["acc"][:, 3])
        assert np.median(rel) <= MED_TOL and np.percentile(rel, 99) <= P99_TOL, (tag, k, np.median(rel),
                                                                                 np.percentile(rel, 99))
        assert np.median(prel) <= MED_TOL and np.percentile(prel, 99) <= P99_TOL
        # A8-A9 with the GPU's forces: drifted positions and t0 exact, levels nearly all equal
        assert np.array_equal(gs["pos"][act].view(np.uint64), sim.r0[act].view(np.uint64)), (tag, k, "r0")
        assert np.all(gs["t0"][act] == sim.t0[act])
        lvl_diff = float(np.mean(gs["level"][act] != sim.level[act])) if act.size else 0.0
        assert lvl_diff <= 1e-3, (tag, k, lvl_diff)
        # A9 driven by the oracle's forces: the oracle's state bit for bit
        _load(s, sim, pre)
        act_pre = r["order"][r["active"]].astype(np.int32)
        acc32 = np.ascontiguousarray(r["acc"].astype(np.float32))
        if act.size:
            s.correct(torch.from_numpy(act_pre).cuda(), torch.from_numpy(acc32).cuda(), r["T"])
        gd = s.get_state()
        o = r["order"]
        for f, ref in (("pos", sim.r0), ("vel", sim.vh)):
            assert np.array_equal(gd[f][o].view(np.uint64), ref.view(np.uint64)), (tag, k, f)
        assert np.array_equal(gd["level"][o], sim.level), (tag, k, "level")
        assert np.array_equal(gd["t0"][o], sim.t0), (tag, k, "t0")
        assert np.array_equal(gd["aold"][o].view(np.uint32), sim.aold.view(np.uint32)), (tag, k, "aold")
        reports.append({"T": r["T"], "n_active": int(act.size), "interactions": int(r["inter"].sum()),
                        "acc_median": float(np.median(rel)) if act.size else 0.0,
                        "acc_p99": float(np.percentile(rel, 99)) if act.size else 0.0,
                        "level_disagreement": lvl_diff})
    assert s.status() == g.GT_OK
    s.close()
    print(f"\n[{tag}] teacher-forced block steps: " + "; ".join(
        f"T={q['T']} actives={q['n_active']} inter={q['interactions']} med={q['acc_median']:.2e} "
        f"p99={q['acc_p99']:.2e} level-diff={q['level_disagreement']:.1e}" for q in reports))
    return reports


def free_running(env, pos, vel, mass, prm, nsteps, tag):
    """Both sides integrate on their own; returns the disagreement report."""
    torch, g, O = env
    n = len(mass)
    oprm = _oparams(O, prm)
    sim = O.BlockStepSim(pos, vel, mass, oprm)
    boot = O.bootstrap_aold(_p4(pos, mass), oprm)
    sim.start(aold_boot=boot)
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    s.start(boot)
    rows = []
    for k in range(nsteps):
        i0 = s.stats()["interactions"]
        r = sim.step()
        s.block_step()
        st = s.stats()
        assert st["T"] == r["T"], (tag, k, st["T"], r["T"])
        gs = s.get_state()
        act_ids = np.sort(gs["id"][s.get_active()])
        ref_ids = np.sort(sim.id[r["active"]])
        common = np.intersect1d(act_ids, ref_ids).size
        act_diff = 1.0 - common / max(act_ids.size, ref_ids.size, 1)
        lv_g = np.empty(n, np.uint8)
        lv_g[gs["id"]] = gs["level"]
        lv_o = np.empty(n, np.uint8)
        lv_o[sim.id] = sim.level
        lvl_diff = float(np.mean(lv_g != lv_o))
        di = st["interactions"] - i0
        do = int(r["inter"].sum())
        rows.append({"T": r["T"], "active_diff": act_diff, "level_diff": lvl_diff,
                     "inter_rel_diff": abs(di - do) / max(do, 1)})
        assert act_diff <= 1e-3 and lvl_diff <= 1e-3, (tag, k, act_diff, lvl_diff)
    gs = s.get_state()
    pg = np.empty((n, 3))
    pg[gs["id"]] = gs["pos"]
    po = np.empty((n, 3))
    po[sim.id] = sim.r0
    dr = np.abs(pg - po).max(axis=1) / (np.abs(po).max(axis=1) + 1e-30)
    assert np.percentile(dr, 99) < 1e-5, np.percentile(dr, 99)
    assert s.status() == g.GT_OK
    s.close()
    rep = {"steps": nsteps, "max_active_diff": max(q["active_diff"] for q in rows),
           "max_level_diff": max(q["level_diff"] for q in rows),
           "max_interaction_rel_diff": max(q["inter_rel_diff"] for q in rows),
           "final_pos_rel_diff_p99": float(np.percentile(dr, 99))}
    print(f"\n[{tag}] free-running block steps: {rep}")
    return rep


# ------------------------------------------------------------------ NFW 2^20, 8 levels, 16 block steps
def test_nfw_2p20_sixteen_block_steps_teacher_forced(env):
    """NFW sphere (c = 10, r_s = 1, tapered beyond 10 r_s), N = 2^20, eps = r_s/256, 8
    levels, acceleration MAC with Delta_acc = 2^-7: 16 kick-drift-kick block steps."""
    torch, g, O = env
    pos, vel, mass, eps = ics.nfw(1 << 20, seed=2)
    prm = _params(g, eps, levels=8, rebuild_every=1, group_max=64, leaf_max=16)
    teacher_forced(env, pos, vel, mass, prm, 16, "nfw-2^20")


def test_nfw_2p20_sixteen_block_steps_free_running(env):
    """The same 16 block steps with the tree kept between rebuilds (every 4 steps on both
    sides, Sec. 2.6), each side on its own forces."""
    torch, g, O = env
    pos, vel, mass, eps = ics.nfw(1 << 20, seed=2)
    prm = _params(g, eps, levels=8, rebuild_every=4, group_max=64, leaf_max=16)
    free_running(env, pos, vel, mass, prm, 16, "nfw-2^20")


# ------------------------------------------------------------------ shared step (L = 1)
def test_shared_step_is_the_oracle_leapfrog(env):
    """L = 1: every particle is active at every step and the block step reduces to the
    kick-drift-kick leap-frog (Sec. 2.7); driven by the oracle's forces the GPU's state is
    the oracle's bit for bit (the oracle itself is pinned to an independent leap-frog)."""
    torch, g, O = env
    n = 1 << 13
    pos, vel, mass, eps = ics.plummer(n, seed=41)
    prm = _params(g, eps, levels=1, rebuild_every=1, group_max=32, dt_max=2.0 ** -7)
    reps = teacher_forced(env, pos, vel, mass, prm, 4, "plummer-L1")
    assert all(q["n_active"] == n for q in reps)
    assert [q["T"] for q in reps] == [1, 2, 3, 4]


def test_shared_step_free_running(env):
    torch, g, O = env
    n = 1 << 13
    pos, vel, mass, eps = ics.plummer(n, seed=42)
    prm = _params(g, eps, levels=1, rebuild_every=2, group_max=32, dt_max=2.0 ** -7)
    free_running(env, pos, vel, mass, prm, 6, "plummer-L1")


# ------------------------------------------------------------------ Andromeda-like 2^24, leaf 32
def test_andromeda_2p24_four_block_steps_teacher_forced(env):
    """The benchmark's workload (Andromeda-like model, N = 2^24, eps = 0.01, leaves of 32,
    8 levels): the first four block steps after the oracle's start-up, every active
    particle compared (the oracle walks them all)."""
    torch, g, O = env
    pos, vel, mass, eps = ics.andromeda_like(1 << 24, seed=3)
    prm = _params(g, eps, levels=8, rebuild_every=1, group_max=64, leaf_max=32)
    teacher_forced(env, pos, vel, mass, prm, 4, "m31-2^24")


def _state_of(s):
    st = s.get_state()
    return {k: st[k] for k in ("pos", "vel", "acc", "aold", "level", "t0", "id")}


def test_lookahead_matches_steps_without_it(env):
    """With the automatic rebuild interval a block step enqueues the next step's
    prediction (A8) before it returns.  The same steps without the look-ahead (a stream
    switch before every step drops it) give the same state bit for bit, through steps
    that refresh the pseudo j-particles on the old tree and one that rebuilds the tree
    from the prediction made ahead.  The first three steps' decisions do not depend on
    timings (one rebuild at the start; the group size fixed), the rest use a fixed
    interval, so both runs take the same steps."""
    torch, g, O = env
    pos, vel, mass, eps = ics.plummer(6144, seed=11)
    runs = []
    for switch in (False, True):
        s = g.System(len(mass), _params(g, eps, leaf_max=16, rebuild_every=0))
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        s.stream = streams[0].cuda_stream
        s.set_state(pos, vel, mass)
        s.start()
        trail = []
        for k in range(6):
            if k == 3:
                s.set_params(_params(g, eps, leaf_max=16, rebuild_every=3))
            if switch:  # another stream, after the last step has finished: nothing is predicted ahead
                torch.cuda.synchronize()
                s.stream = streams[(k + 1) % 2].cuda_stream
            s.block_step()
            st = s.stats()
            trail.append((st["T"], st["n_active"], st["interactions"], st["rebuilds"]))
        torch.cuda.synchronize()
        runs.append((trail, _state_of(s)))
        s.close()
    (ta, sa), (tb, sb) = runs
    assert ta == tb
    assert ta[3][3] == ta[2][3] + 1  # the fourth step rebuilt the tree
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)


def test_advance_with_lookahead_stops_at_the_end_time(env):
    """gt_advance reads the next block time from the words mirrored after each step and
    stops at the last block time not after T_end; the phase timers count every
    prediction, the one made ahead of a step included."""
    torch, g, O = env
    pos, vel, mass, eps = ics.plummer(4096, seed=12)
    s = g.System(len(mass), _params(g, eps, leaf_max=16, rebuild_every=0, levels=5))
    s.set_state(pos, vel, mass)
    s.start()
    s.profile(True)
    span = 1 << (5 - 1)
    k = s.advance(span)
    st = s.stats()
    assert st["T"] == span and k == st["block_steps"] and k >= 1
    tm = s.timers()
    assert tm["predict"][1] == k + 1  # the k steps' predictions and the one ahead of step k + 1
    assert tm["walk"][1] == k
    s.close()
