"""Multi-GPU partitioning, checked on CPU ranks (gloo, world size 2).

Independent systems shard by whole systems (no exchange); one system's force
evaluation can split over contiguous slices of its groups, each rank evaluating its
slice of the same tree.  In both cases the gathered result must equal the one-rank
result bit for bit; the ranks evaluate with the oracle, since a CPU rank has no GPU.
The shard planning that bench.py runs on every rank under torchrun (the batch's
systems, the serving stream's requests) is run here by two CPU ranks as it is.
"""
import os
import socket

import numpy as np
import pytest

from paper_1610_07279_gb300 import ics, partition


def test_assign_systems_is_a_balanced_partition():
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in rng.integers(1, 1000, 37)]
    for world in (1, 2, 3, 8):
        parts = partition.assign_systems(sizes, world)
        assert sorted(k for p in parts for k in p) == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)  # greedy LPT bound
    assert partition.assign_systems([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        partition.assign_systems([1], 0)


def test_group_slices_cover_every_group_once():
    for ng in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 5):
            cuts = [partition.group_slice(ng, r, world) for r in range(world)]
            assert cuts[0][0] == 0 and cuts[-1][1] == ng
            assert all(cuts[r][1] == cuts[r + 1][0] for r in range(world - 1))
            assert max(b - a for a, b in cuts) - min(b - a for a, b in cuts) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _p4(pos, mass):
    p4 = np.zeros((len(mass), 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    return p4


def _rank_groups(rank, world, port, q):
    """Rank `rank` walks its contiguous slice of the groups of one Plummer sphere."""
    import torch.distributed as dist
    import oracle as O
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    pos, vel, mass, eps = ics.plummer(4096, seed=31)
    prm = O.Params(eps=O.f32(eps))
    p4 = _p4(pos, mass)
    aold = O.bootstrap_aold(p4, prm)
    full = O.tree_force(p4, prm, aold=aold, group_ids=np.zeros(0, np.int64))  # the groups only
    ng = len(full["starts"]) - 1
    g0, g1 = partition.group_slice(ng, rank, world)
    r = O.tree_force(p4, prm, aold=aold, group_ids=np.arange(g0, g1, dtype=np.int64))
    a0, a1 = int(r["starts"][g0]), int(r["starts"][g1]) if g1 <= ng else len(mass)
    mine = (a0, r["acc"][a0:a1].copy(), r["inter"][a0:a1].copy())
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        acc = np.full((len(mass), 4), np.nan)
        inter = np.full(len(mass), -1, np.int64)
        for s, a, i in got:
            acc[s:s + len(a)] = a
            inter[s:s + len(i)] = i
        q.put((acc, inter))
    dist.barrier()
    dist.destroy_process_group()


def _rank_systems(rank, world, port, q):
    """Rank `rank` evaluates its share of a batch of independent systems."""
    import torch.distributed as dist
    import oracle as O
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mem = ics.batch_systems(6, seed=32, log2_lo=9.0, log2_hi=11.0)
    parts = partition.assign_systems([m["n"] for m in mem], world)
    mine = {}
    for k in parts[rank]:
        m = mem[k]
        prm = O.Params(eps=O.f32(m["eps"]))
        mine[k] = O.tree_force(_p4(m["pos"], m["mass"]), prm, mac=0)["acc"]
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        out = {}
        for d in got:
            out.update(d)
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def _run_ranks(target, world=2):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    return res


def test_two_ranks_over_group_slices_equal_one_rank():
    pytest.importorskip("torch")
    import oracle as O
    O.build()
    acc, inter = _run_ranks(_rank_groups)
    pos, vel, mass, eps = ics.plummer(4096, seed=31)
    prm = O.Params(eps=O.f32(eps))
    p4 = _p4(pos, mass)
    ref = O.tree_force(p4, prm, aold=O.bootstrap_aold(p4, prm))
    assert np.array_equal(acc, ref["acc"]) and np.array_equal(inter, ref["inter"])


def test_two_ranks_over_whole_systems_equal_one_rank():
    pytest.importorskip("torch")
    import oracle as O
    O.build()
    out = _run_ranks(_rank_systems)
    mem = ics.batch_systems(6, seed=32, log2_lo=9.0, log2_hi=11.0)
    assert sorted(out) == list(range(len(mem)))
    for k, m in enumerate(mem):
        ref = O.tree_force(_p4(m["pos"], m["mass"]), O.Params(eps=O.f32(m["eps"])), mac=0)["acc"]
        assert np.array_equal(out[k], ref), k


def _rank_plans(rank, world, port, q):
    """Rank `rank` plans its share of the benchmark's batch (64 systems) and serving
    stream with the same calls bench.py makes under torchrun, with no exchange; the
    plans are gathered only to check them."""
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mem = ics.batch_systems(64, seed=4, log2_lo=6.0, log2_hi=8.0)  # the bench's sizes scaled down
    ns = [m["n"] for m in mem]
    reqs = ics.serving_requests(512 * world, seed=5, rate=100.0 * world)
    mine = (rank, bench.batch_shard(ns, rank, world), bench.serving_shard(reqs, rank, world))
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        q.put((got, ns, [r["n"] * max(r["steps"], 1) for r in reqs]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_plan_disjoint_complete_shards():
    """The shards of the batch and of the serving stream that two ranks plan
    independently cover every system and request exactly once, are balanced, and are
    what each rank would have planned for the other."""
    pytest.importorskip("torch")
    got, ns, work = _run_ranks(_rank_plans)
    got = sorted(got)
    bat = [b for _, b, _ in got]
    srv = [s for _, _, s in got]
    assert sorted(k for b in bat for k in b) == list(range(len(ns)))
    assert sorted(k for s in srv for k in s) == list(range(len(work)))
    import bench
    assert bat == [bench.batch_shard(ns, r, 2) for r in range(2)]
    loads = [sum(ns[k] for k in b) for b in bat]
    assert max(loads) - min(loads) <= max(ns)
    wl = [sum(work[k] for k in s) for s in srv]
    assert max(wl) - min(wl) <= max(work)
    assert all(s == sorted(s) for s in srv)  # arrival order kept
