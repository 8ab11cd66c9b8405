"""Serving (gt_server_*): continuous batching of block-step requests.

A request's result -- its final state in the caller's particle order -- must be the
same bit for bit when it runs alone and when it shares ticks with other requests, and
the same as the single-system path (gt_start + gt_block_step) with the same
parameters.  Admission must respect the slot count and the memory cap.
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


def _params(g, eps, **kw):
    prm = g.gt_default_params()
    prm.eps = eps
    prm.levels = 5
    prm.rebuild_every = 2
    prm.walk_queue = 8192  # the servers below use this depth: same traversal order alone
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def _requests(g, count, seed, lo=10.0, hi=12.5):
    rng = np.random.default_rng(seed)
    out = []
    for m in ics.batch_systems(count, seed=seed, log2_lo=lo, log2_hi=hi):
        prm = _params(g, m["eps"], rebuild_every=int(rng.integers(1, 4)), group_max=int(rng.choice([16, 32])))
        out.append({"pos": m["pos"], "vel": m["vel"], "mass": m["mass"], "params": prm,
                    "nsteps": int(rng.integers(2, 7)), "n": m["n"]})
    return out


def _run(g, reqs, max_slots=8, hbm_cap=64 << 30, walk_queue=8192):
    """Submit in order (waiting for room when needed), collect every result."""
    srv = g.Server(hbm_cap, max_slots=max_slots, walk_queue=walk_queue)
    pending = list(range(len(reqs)))
    tickets, results = {}, {}
    waited = 0
    while pending or tickets:
        while pending:
            r = reqs[pending[0]]
            t = srv.submit(r["pos"], r["vel"], r["mass"], r["params"], r["nsteps"])
            if t is None:
                waited += 1
                break
            tickets[t] = pending.pop(0)
        for t in list(tickets):
            k = tickets[t]
            pos = np.zeros((reqs[k]["n"], 3))
            vel = np.zeros((reqs[k]["n"], 3))
            if srv.poll(t, pos, vel):
                results[k] = (pos, vel)
                del tickets[t]
    st = srv.stats()
    srv.close()
    return results, st, waited


def test_server_matches_single_system(env):
    torch, g = env
    pos, vel, mass, eps = ics.plummer(3000, seed=21)
    prm = _params(g, eps)
    nsteps = 6
    res, st, _ = _run(g, [{"pos": pos, "vel": vel, "mass": mass, "params": prm, "nsteps": nsteps, "n": 3000}])
    s = g.System(3000, prm)
    s.set_state(pos, vel, mass)
    s.start()
    for _ in range(nsteps):
        s.block_step()
    ref = s.get_state()
    s.close()
    order = ref["id"].astype(np.int64)
    rp = np.empty_like(ref["pos"])
    rv = np.empty_like(ref["vel"])
    rp[order] = ref["pos"]
    rv[order] = ref["vel"]
    assert np.array_equal(res[0][0], rp) and np.array_equal(res[0][1], rv)
    assert not np.array_equal(rp, pos)  # the request did advance
    assert st["ticks"] == nsteps + 1 and st["completed"] == 1


def test_server_alone_vs_mix_bit_identical(env):
    torch, g = env
    reqs = _requests(g, 12, seed=22)
    mixed, st, waited = _run(g, reqs, max_slots=5)
    assert len(mixed) == len(reqs) and st["completed"] == len(reqs)
    assert waited > 0  # some requests had to wait for a slot and joined later ticks
    assert st["walk_launches"] < sum(r["nsteps"] + 2 for r in reqs)  # walks were shared
    for k in (0, 3, 7, 11):
        alone, _, _ = _run(g, [reqs[k]], max_slots=1)
        assert np.array_equal(alone[0][0], mixed[k][0]), k
        assert np.array_equal(alone[0][1], mixed[k][1]), k


def test_server_device_outputs(env):
    torch, g = env
    reqs = _requests(g, 2, seed=23)
    host, _, _ = _run(g, reqs)
    srv = g.Server(64 << 30, max_slots=2, walk_queue=8192)
    t = [srv.submit(r["pos"], r["vel"], r["mass"], r["params"], r["nsteps"]) for r in reqs]
    outs = [(torch.zeros((r["n"], 3), dtype=torch.float64, device="cuda"),
             torch.zeros((r["n"], 3), dtype=torch.float64, device="cuda")) for r in reqs]
    done = [False, False]
    while not all(done):
        for k in range(2):
            if not done[k]:
                done[k] = srv.poll(t[k], outs[k][0], outs[k][1])
    srv.close()
    for k in range(2):
        assert np.array_equal(outs[k][0].cpu().numpy(), host[k][0])
        assert np.array_equal(outs[k][1].cpu().numpy(), host[k][1])


def test_server_admission_respects_memory_cap(env):
    torch, g = env
    reqs = _requests(g, 3, seed=24, lo=11.0, hi=11.0)
    probe = g.Server(64 << 30, max_slots=1, walk_queue=8192)
    region = probe.stats()["hbm_used"]
    r = reqs[0]
    t = probe.submit(r["pos"], r["vel"], r["mass"], r["params"], 1)
    per = probe.stats()["hbm_used"] - region
    assert t is not None and per > 0
    probe.close()
    srv = g.Server(region + per + per // 2, max_slots=8, walk_queue=8192)
    t0 = srv.submit(r["pos"], r["vel"], r["mass"], r["params"], 1)
    assert t0 is not None
    assert srv.submit(reqs[1]["pos"], reqs[1]["vel"], reqs[1]["mass"], reqs[1]["params"], 1) is None
    assert srv.stats()["hbm_used"] <= srv.stats()["hbm_cap"]
    while not srv.poll(t0):
        pass
    t1 = srv.submit(reqs[1]["pos"], reqs[1]["vel"], reqs[1]["mass"], reqs[1]["params"], 1)
    assert t1 is not None
    while not srv.poll(t1):
        pass
    assert srv.stats()["completed"] == 2
    srv.close()


def test_server_rejects_bad_requests(env):
    torch, g = env
    srv = g.Server(64 << 30, max_slots=2, walk_queue=8192)
    prm = _params(g, 1.0 / 64)
    with pytest.raises(g.GothicError):
        srv.submit(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, np.float32), prm, 2)
    bad = _params(g, 1.0 / 64, leaf_max=0)
    pos, vel, mass, _ = ics.plummer(1024, seed=25)
    with pytest.raises(g.GothicError):
        srv.submit(pos, vel, mass, bad, 2)
    with pytest.raises(g.GothicError):
        srv.poll(12345)
    assert srv.stats()["slots_used"] == 0
    srv.close()
