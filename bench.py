#!/usr/bin/env python3
"""Benchmark of the block-step oct-tree gravity path on the Andromeda-like model.

Workload: the three-component Andromeda-like model (Hernquist bulge 3 %, exponential
disk 5 %, tapered NFW halo 92 %) with N = 2^24 equal-mass particles, eps = 0.01,
acceleration MAC with Delta_acc = 2^-7, 8 block-step levels.  One benchmark step is
one full block-step cycle (block steps until the block time reaches the next
multiple of the longest step); the tree is rebuilt at the interval chosen by the
rebuild model of the paper's Sec. 2.6 (pseudo j-particles refreshed at every block
step): every step of the method (predict, keys, sort, permute, build, pseudo
j-particles, active set, walk, correct) runs in it.

Reported: interactions/s of the whole job (value), seconds per block step, the
end-to-end number through pinned host buffers, the walk kernel against the FP32
roofline, clocks sampled during the timed region, and the CPU oracle timed on a
bounded sample (rank 0, N = 1).  --impl reference times the CPU oracle instead.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one replica per GPU (the single system does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "block-step s & interactions/s at N=2^24; p50/p99 batched-solve latency"
# Flops per interaction by the paper's convention (Sec. 4, note to Table 3): 3 subtractions,
# 3 multiplications and 7 FMAs (the potential included) = 20, plus the reciprocal square
# root counted as the ratio of the add/multiply throughput to its own.
FLOPS_BASE = 20


def flops_per_interaction(rsqrt_flops: float) -> float:
    return FLOPS_BASE + rsqrt_flops


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--levels", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-groups", type=int, default=2048, help="groups walked by the CPU baseline sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-system batch workload")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-shared", action="store_true", help="skip the shared-step comparison")
    ap.add_argument("--no-nfw", action="store_true", help="skip the NFW 2^20 block-step workload")
    ap.add_argument("--no-error", action="store_true", help="skip the error report against FP64 direct sums")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-rho", type=str, default="0.5,0.8,1.0,1.2,2.0,burst",
                    help="load levels as multiples of the serial capacity; 'burst' = all requests at t = 0")
    return ap.parse_args()


# ------------------------------------------------------------------ workload
# Leaf size of the main 2^24 cycle: measured over whole block-step cycles of this model
# (automatic rebuild interval), leaves of 16, 24 and 32 particles took 437-439, 421-422 and
# 419 ms per cycle (fewer, larger leaves shorten the pseudo j pass and the tree; the walk
# evaluates more interactions).  The library default stays 16.
LEAF_MAX = 32


def workload(n: int):
    from paper_1610_07279_gb300 import ics
    pos, vel, mass, eps = ics.andromeda_like(n, seed=3)
    return pos, vel, mass, eps


def config_dict(args, eps):
    return {"workload": f"Andromeda-like three-component model (bulge 3%, disk 5%, NFW halo 92%), "
                        f"N={args.n}, one full block-step cycle per step, tree rebuilt at the automatic "
                        f"interval (Sec. 2.6)",
            "n": args.n, "levels": args.levels, "mac": "acceleration", "delta_acc": 2.0 ** -7,
            "eps": eps, "leaf_max": LEAF_MAX, "group_max": 64, "ij_share": "per group",
            "groups": "tree cells with at most 16, 32 or 64 actives, the size tuned per class of "
                      "block step (coarsest active level)",
            "l2": "inputs larger than L2 (particle state ~1.7 GB, nodes ~0.3 GB)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"gothic_clocks_{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle sample
def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_sample(pos, mass, eps, groups: int, seed: int = 7, single_core_groups: int = 0):
    """The oracle on a bounded sample of the workload: one full tree build (A1-A5)
    of all particles on all cores and the FP64 walk (A6-A7, acceleration MAC) of `groups`
    random groups on all cores; with single_core_groups > 0 also the walk of that many
    other random groups on one core.  Returns (interactions, seconds for the build share
    plus the walk, info)."""
    import oracle as O
    O.build()
    n = len(mass)
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    prm = O.Params(eps=O.f32(eps), leaf_max=LEAF_MAX, group_max=64)
    t0 = time.perf_counter()
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = np.ascontiguousarray(p4[order])
    tree = O.build_tree(skey, prm.leaf_max)
    jpos, bj = O.pseudo_j(tree, sp4)
    active = np.arange(n, dtype=np.uint32)
    starts = O.group_starts(tree, n, active, prm.group_max, prm.group_mode)
    t_build = time.perf_counter() - t0
    ng = len(starts) - 1
    rng = np.random.default_rng(seed)
    pick = rng.permutation(ng)
    gids = np.sort(pick[:min(groups, ng)]).astype(np.int64)
    gids1 = np.sort(pick[min(groups, ng):min(groups + single_core_groups, ng)]).astype(np.int64)

    def walk(ids):
        # |a_old| of the members from an opening-angle pass (setup, not timed)
        gI, gamin = O.groups(starts, active, sp4, None)
        boot, _, _ = O.walk(tree, jpos, bj, sp4, active, starts, gI, gamin, 0, prm.theta,
                            prm.delta_acc, prm.eps, prm.G, group_ids=ids)
        aold = np.zeros(n, np.float32)
        rows = np.isfinite(boot[:, 0])
        aold[rows] = O.aold_of(boot[rows].astype(np.float32))
        gI, gamin = O.groups(starts, active, sp4, aold)
        t1 = time.perf_counter()
        acc, inter, _ = O.walk(tree, jpos, bj, sp4, active, starts, gI, gamin, 1, prm.theta,
                               prm.delta_acc, prm.eps, prm.G, group_ids=ids)
        return int(inter[inter >= 0].sum()), time.perf_counter() - t1

    threads = O.num_threads()
    n_inter, t_walk = walk(gids)
    info = {"t_build_s": t_build, "t_walk_s": t_walk, "groups": int(len(gids)), "groups_total": int(ng),
            "threads": threads, "walk_rate_all_cores": n_inter / t_walk}
    if len(gids1):
        O.set_num_threads(1)
        try:
            i1, w1 = walk(gids1)
        finally:
            O.set_num_threads(threads)
        info.update({"single_core_groups": int(len(gids1)), "t_walk_1core_s": w1, "walk_rate_1_core": i1 / w1})
    share = len(gids) / ng
    secs = t_walk + t_build * share
    return n_inter, secs, info


def cpu_baseline_entry(pos, mass, eps, groups):
    n_inter, secs, info = cpu_sample(pos, mass, eps, groups, single_core_groups=max(32, groups // 16))
    aff = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else []
    return {"value": n_inter / secs, "unit": "interactions/s", "cores": info["threads"], "kind": "oracle",
            "sample": (f"one oracle tree build of all {len(mass)} particles (A1-A5, {info['t_build_s']:.2f} s, "
                       f"charged pro rata to the sampled groups) plus the FP64 walk of {info['groups']} of "
                       f"{info['groups_total']} random groups ({info['t_walk_s']:.2f} s, acceleration MAC), "
                       f"all cores"),
            "interactions": n_inter, "cpu_model": cpu_model(), "affinity_cpus": len(aff),
            "omp_threads": info["threads"],
            "walk_interactions_per_s": {"all_cores": info["walk_rate_all_cores"],
                                        "one_core": info.get("walk_rate_1_core"),
                                        "one_core_sample_groups": info.get("single_core_groups")},
            "build_s_all_cores": info["t_build_s"]}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pos, vel, mass, eps = workload(args.n)
    import oracle as O
    O.build()
    vals, times = [], []
    for k in range(args.warmup + args.steps):
        n_inter, secs, info = cpu_sample(pos, mass, eps, max(64, args.cpu_groups // 4), seed=100 + k)
        if k >= args.warmup:
            vals.append(n_inter / secs)
            times.append(secs)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(args, eps),
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": info["threads"],
                             "kind": "oracle",
                             "sample": "per step: the oracle's full tree build charged pro rata plus the FP64 walk "
                                       f"of {info['groups']} random groups, all cores",
                             "cpu_model": cpu_model(),
                             "affinity_cpus": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                             else None},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



# ------------------------------------------------------------------ block vs shared step
def run_shared_comparison(g, torch, pos, vel, mass, eps, block_cycle_ms, block_inter, dt_max, levels,
                          steps: int = 16):
    """Sec. 3.3: the same model advanced with one shared step equal to the block run's
    finest step (every particle active at every step); a cycle of the block run spans
    2^(L-1) such steps.  The speed-up is the shared time per cycle over the block time."""
    dt_min = dt_max / 2 ** (levels - 1)
    prm = g.gt_default_params()
    prm.eps = eps
    prm.leaf_max = LEAF_MAX
    prm.levels = 1
    prm.dt_max = dt_min
    s = g.System(len(mass), prm)
    s.set_state(pos, vel, mass)
    s.start()
    for _ in range(4):
        s.block_step()
    s.sync()
    st = torch.cuda.current_stream()
    i0 = s.stats()["interactions"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        s.block_step()
    e1.record(st)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / steps
    inter = (s.stats()["interactions"] - i0) / steps
    s.close()
    ticks = 2 ** (levels - 1)
    return {"workload": "the same model with one shared step = the block run's finest step (L = 1), "
                        "every particle active every step; one block cycle spans 2^(L-1) shared steps",
            "shared_step_ms": step_ms, "shared_steps_per_cycle": ticks, "shared_cycle_ms": step_ms * ticks,
            "block_cycle_ms": block_cycle_ms, "speedup_block_vs_shared": step_ms * ticks / block_cycle_ms,
            "interactions_per_cycle": {"shared": inter * ticks, "block": block_inter}}


# ------------------------------------------------------------------ ranks
class Comm:
    """Max, sum and gather over the ranks of the job (identity on one rank)."""

    def __init__(self, rank: int = 0, world: int = 1):
        self.rank, self.world = rank, world

    def _reduce(self, x, op):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.MAX if self.world > 1 else None)

    def sum(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.SUM if self.world > 1 else None)

    def gather(self, obj) -> list:
        if self.world == 1:
            return [obj]
        import torch.distributed as dist
        out = [None] * self.world
        dist.all_gather_object(out, obj)
        return out


def batch_shard(ns, rank: int, world: int) -> list[int]:
    """This rank's systems of a batch: whole systems, balanced by particle count."""
    from paper_1610_07279_gb300 import partition
    return partition.assign_systems(ns, world)[rank]


def serving_shard(reqs, rank: int, world: int) -> list[int]:
    """This rank's requests of a serving stream: balanced by particles x block steps."""
    from paper_1610_07279_gb300 import partition
    return partition.shard_requests([r["n"] * max(r["steps"], 1) for r in reqs], world)[rank]


# ------------------------------------------------------------------ batch workload
def direct_fp64(pos, mass, eps, G, targets):
    """Eq. (1) in FP64 for the target rows (plain numpy, chunked): the accuracy yardstick
    of the batch report."""
    pos = np.asarray(pos, np.float64)
    m = np.asarray(mass, np.float64)
    out = np.zeros((len(targets), 3))
    e2 = float(eps) ** 2
    for a in range(0, len(targets), 16):
        t = targets[a:a + 16]
        d = pos[None, :, :] - pos[t][:, None, :]
        r2 = (d * d).sum(-1) + e2
        w = m[None, :] / (r2 * np.sqrt(r2))
        out[a:a + 16] = G * (w[:, :, None] * d).sum(1)
    return out


def run_batch(g, torch, steps: int, comm: Comm | None = None):
    """64 independent systems (Plummer or NFW, N log-uniform in [2^12, 2^18]): one force
    evaluation of all of them per step, as a captured graph of forked builds and one
    walk launch, knobs from the autotuner; against the same members through the
    single-system calls one after another.  On several GPUs the 64 systems are shared
    out whole (balanced by size, no exchange) and the job's time is the slowest rank's."""
    from paper_1610_07279_gb300 import ics
    comm = comm or Comm()
    allmem = ics.batch_systems(64, seed=4)
    mine = batch_shard([m["n"] for m in allmem], comm.rank, comm.world)
    mem = [allmem[k] for k in mine]
    prms = []
    for m in mem:
        p = g.gt_default_params()
        p.eps = m["eps"]
        prms.append(p)
    b = g.Batch([m["n"] for m in mem], prms)
    for s, m in zip(b.systems, mem):
        s.set_state(m["pos"], m["vel"], m["mass"])
    b.accel(bootstrap=True)
    b.sync()
    tune = b.autotune(leaf_max=(8, 16, 32), group_max=(16, 32), walk_queue=(8192, 16384), reps=3)
    b.capture(bootstrap=False)
    b.launch()
    b.sync()
    st = torch.cuda.ExternalStream(b.stream)
    reps = max(10, steps)
    i0 = int(b.sync().sum())
    l0 = g.gt_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        b.launch()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    inter = (int(b.sync().sum()) - i0) / reps
    launches = (g.gt_kernel_launches() - l0) / reps
    # serial: the same members, build + walk of every particle, one system after another
    accs = [torch.empty((max(m["n"], 1), 4), dtype=torch.float32, device="cuda") for m in mem]
    for s, a in zip(b.systems, accs):  # warm-up
        s.build_tree()
        s.accel_active(None, None, a)
    b.sync()
    i0 = int(b.sync().sum())
    e0.record(st)
    for _ in range(reps):
        for s, a in zip(b.systems, accs):
            s.build_tree()
            s.accel_active(None, None, a)
    e1.record(st)
    e1.synchronize()
    ms_serial = e0.elapsed_time(e1) / reps
    inter_serial = (int(b.sync().sum()) - i0) / reps
    # accuracy: FP32 forces of the batch vs FP64 direct sums on 128 random particles per system
    b.launch()
    b.sync()
    rng = np.random.default_rng(40)
    per = []
    for k, m in enumerate(mem):
        acc, ids = b.get_acc(k)
        rows = rng.choice(m["n"], min(128, m["n"]), replace=False)
        ref = direct_fp64(m["pos"], m["mass"], m["eps"], 1.0, ids[rows].astype(np.int64))
        rel = np.linalg.norm(acc[rows, :3] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        per.append({"kind": m["kind"], "n": m["n"], "median": float(np.median(rel)),
                    "p99": float(np.percentile(rel, 99))})
    b.close()
    ms, ms_serial = comm.max(ms), comm.max(ms_serial)
    inter, inter_serial = comm.sum(inter), comm.sum(inter_serial)
    per = [q for part in comm.gather(per) for q in part]
    return {"workload": "64 systems, Plummer or NFW by seeded coin, N = round(2^(12 + 6u)), own eps; "
                        "one force evaluation of every system per step (tree build + every particle "
                        "active, acceleration MAC with a_old from an opening-angle start-up pass)",
            "total_particles": int(sum(m["n"] for m in allmem)), "ranks": comm.world,
            "scaling": "strong (the 64 systems shared out whole across the ranks)",
            "autotuned": {"leaf_max": tune["leaf_max"], "group_max": tune["group_max"],
                          "walk_queue": tune["walk_queue"], "candidates_ms": tune["ms"]},
            "batched": {"ms_per_step": ms, "interactions_per_s": inter / (ms * 1e-3),
                        "systems_per_s": 64 / (ms * 1e-3), "gpu_launches_per_step": launches,
                        "path": "captured CUDA graph: forked builds + one persistent walk launch"},
            "serial": {"ms_per_step": ms_serial, "interactions_per_s": inter_serial / (ms_serial * 1e-3),
                       "systems_per_s": 64 / (ms_serial * 1e-3),
                       "path": "gt_build_tree + gt_accel_active per system, one after another"},
            "speedup_vs_serial": ms_serial / ms,
            "error_vs_fp64_direct": {"sample": "128 random particles per system vs FP64 direct summation",
                                     "median_of_medians": float(np.median([p["median"] for p in per])),
                                     "max_median": float(max(p["median"] for p in per)),
                                     "max_p99": float(max(p["p99"] for p in per)), "per_system": per}}


# ------------------------------------------------------------------ serving workload
class RequestSource:
    """Inputs of the serving stream: one 2^20-particle sample per model, a request of N
    particles takes its first N (the samples are iid, so a prefix is a sample of the
    model; masses rescaled to total 1)."""

    def __init__(self):
        from paper_1610_07279_gb300 import ics
        self.master = {"plummer": ics.plummer(1 << 20, seed=51), "nfw": ics.nfw(1 << 20, seed=52)}

    def get(self, req):
        pos, vel, mass, eps = self.master[req["kind"]]
        n = req["n"]
        m = np.full(n, np.float32(1.0 / n))
        return np.ascontiguousarray(pos[:n]), np.ascontiguousarray(vel[:n]), m, eps


def serve_params(g, eps):
    p = g.gt_default_params()
    p.eps = eps
    p.rebuild_every = 4        # a server cannot sync per step for the automatic interval
    p.group_max = 32           # nor tune the group size per step
    p.group_mode = g.GT_GROUP_CELLS
    p.walk_queue = 8192
    return p


def run_serving(g, torch, nreq: int, rhos, comm: Comm | None = None):
    """The serving stream; on several GPUs every rank serves its shard of a stream of
    nreq requests per GPU at the per-GPU load (weak scaling), and latencies are pooled."""
    from paper_1610_07279_gb300 import ics
    comm = comm or Comm()
    src = RequestSource()
    # serial capacity: requests alone through the single-system path, one after another
    probe = ics.serving_requests(48, seed=55, rate=1.0)
    t_serial = []
    for r in probe:
        pos, vel, mass, eps = src.get(r)
        t0 = time.perf_counter()
        s = g.System(r["n"], serve_params(g, eps))
        s.set_state(pos, vel, mass)
        s.start()
        for _ in range(r["steps"]):
            s.block_step()
        out = s.get_state()
        s.close()
        t_serial.append(time.perf_counter() - t0)
    cap = 1.0 / float(np.mean(t_serial[4:]))  # requests/s, first few are warm-up
    cap = comm.sum(cap) / comm.world            # the ranks' mean serial capacity
    runs = []
    for rho in rhos:
        burst = rho == "burst"
        whole = ics.serving_requests(nreq * comm.world, seed=5,
                                     rate=(cap if burst else float(rho) * cap) * comm.world)
        reqs = [whole[k] for k in serving_shard(whole, comm.rank, comm.world)]
        if burst:
            for r in reqs:
                r["arrival"] = 0.0
        srv = g.Server(150 * 10**9, max_slots=128, walk_queue=8192)
        outs = {}
        lat_arr, lat_sub = [], []
        nxt, pending, tickets = 0, [], {}
        t_start = time.perf_counter()
        while nxt < len(reqs) or pending or tickets:
            now = time.perf_counter() - t_start
            while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
                pending.append(nxt)
                nxt += 1
            while pending:
                r = reqs[pending[0]]
                pos, vel, mass, eps = src.get(r)
                t = srv.submit(pos, vel, mass, serve_params(g, eps), r["steps"])
                if t is None:
                    break
                tickets[t] = (pending.pop(0), time.perf_counter() - t_start)
            for t in list(tickets):
                k, t_sub = tickets[t]
                if srv.poll(t):
                    done = time.perf_counter() - t_start
                    lat_arr.append(done - reqs[k]["arrival"])
                    lat_sub.append(done - t_sub)
                    del tickets[t]
            if not tickets and pending == [] and nxt < len(reqs):
                time.sleep(max(0.0, min(0.002, reqs[nxt]["arrival"] - (time.perf_counter() - t_start))))
        span = comm.max(time.perf_counter() - t_start)
        st = srv.stats()
        srv.close()
        lat_arr = [x for part in comm.gather(lat_arr) for x in part]
        lat_sub = [x for part in comm.gather(lat_sub) for x in part]
        nall = len(lat_arr)
        runs.append({"rho": rho, "arrival_rate_per_s": None if burst else float(rho) * cap * comm.world,
                     "requests": nall,
                     "p50_latency_s": float(np.percentile(lat_arr, 50)),
                     "p99_latency_s": float(np.percentile(lat_arr, 99)),
                     "p50_submit_to_done_s": float(np.percentile(lat_sub, 50)),
                     "p99_submit_to_done_s": float(np.percentile(lat_sub, 99)),
                     "throughput_req_per_s": nall / span, "makespan_s": span,
                     "ticks": int(comm.sum(st["ticks"])), "batched_walk_launches": int(comm.sum(st["walk_launches"]))})
    return {"workload": f"Poisson arrivals of Plummer/NFW systems, N log-uniform in [2^12, 2^20], 4-32 block "
                        f"steps each (8 levels, acceleration MAC, rebuild every 4 steps), {nreq} requests per "
                        f"load level and GPU, HBM admission cap 150 GB per GPU, up to 128 resident per GPU",
            "ranks": comm.world, "scaling": "weak (each GPU serves its shard of a stream of nreq x ranks)",
            "serial_capacity_req_per_s": cap,
            "serial_path": "gt_system_create + gt_set_state + gt_start + block steps + gt_get_state, one "
                           "request at a time (48 sampled requests)",
            "latency": "from arrival (queueing included); submit-to-done also given",
            "runs": runs,
            "max_throughput_vs_serial": max(r["throughput_req_per_s"] for r in runs) / (cap * comm.world)}


# ------------------------------------------------------------------ NFW 2^20, 16 block steps
def run_nfw_block_steps(g, torch, reps: int = 3, steps: int = 16):
    """The NFW sphere (c = 10, r_s = 1, tapered beyond 10 r_s), N = 2^20, eps = r_s/256, 8
    levels, acceleration MAC with Delta_acc = 2^-7: 16 kick-drift-kick block steps after the
    start-up, timed with CUDA events (the start-up, with its tree and two full walks, is
    not timed).  The first repetition is a warm-up."""
    from paper_1610_07279_gb300 import ics
    pos, vel, mass, eps = ics.nfw(1 << 20, seed=2)
    prm = g.gt_default_params()
    prm.eps = eps
    prm.levels = 8
    s = g.System(len(mass), prm)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    for r in range(reps + 1):
        s.set_state(pos, vel, mass)
        s.start()
        s.sync()
        s0 = s.stats()
        e0.record(st)
        for _ in range(steps):
            s.block_step()
        e1.record(st)
        torch.cuda.synchronize()
        s1 = s.stats()
        if r:
            ms = e0.elapsed_time(e1)
            runs.append({"ms": ms, "interactions": s1["interactions"] - s0["interactions"], "T": s1["T"],
                         "rebuilds": s1["rebuilds"] - s0["rebuilds"]})
    s.close()
    ms = float(np.mean([q["ms"] for q in runs]))
    inter = float(np.mean([q["interactions"] for q in runs]))
    return {"workload": "NFW sphere, N=2^20, c=10, r_s=1, tapered beyond 10 r_s, eps=r_s/256, 8 levels, "
                        "acceleration MAC (Delta_acc=2^-7), 16 kick-drift-kick block steps after the start-up, "
                        "automatic rebuild interval, group size tuned per class of step",
            "block_steps": steps, "block_step_s": ms * 1e-3 / steps, "interactions_per_s": inter / (ms * 1e-3),
            "interactions_per_block_step": inter / steps, "T_end_ticks": runs[-1]["T"],
            "rebuilds": runs[-1]["rebuilds"], "reps": reps}


# ------------------------------------------------------------------ error against FP64 direct sums
def _rel_err(a, ref):
    a = np.asarray(a, np.float64)
    num = np.linalg.norm(a[:, :3] - ref[:, :3], axis=1)
    den = np.linalg.norm(ref[:, :3], axis=1)
    return num / np.where(den > 0, den, 1.0)


def _dist(x):
    return {"median": float(np.median(x)), "p99": float(np.percentile(x, 99)), "max": float(np.max(x))}


def error_report(g, torch, kind: str, n: int, seed: int, leaf: int, target: int, model=None):
    """One force evaluation with the acceleration MAC (Delta_acc = 2^-7) on the GPU; on a
    seeded sample of whole groups (>= target particles) it is compared with the oracle's
    tree code (O2, same lists: parity) and with FP64 direct summation (O1: the error of the
    method).  The sampled members' |a_old| come from the oracle's opening-angle pass on
    both sides; the GPU's other groups use its own."""
    import oracle as O
    from paper_1610_07279_gb300 import ics
    gen = {"plummer": ics.plummer, "nfw": ics.nfw, "m31": ics.andromeda_like}[kind]
    pos, vel, mass, eps = model if model is not None else gen(n, seed=seed)
    t_all = time.perf_counter()
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    prm = g.gt_default_params()
    prm.eps = eps
    prm.leaf_max = leaf
    prm.group_mode = g.GT_GROUP_CELLS
    oprm = O.Params(eps=O.f32(eps), leaf_max=leaf, group_max=prm.group_max)
    key, _ = O.keys(p4)
    order, skey = O.sort(key)
    sp4 = np.ascontiguousarray(p4[order])
    tree = O.build_tree(skey, leaf)
    jpos, bj = O.pseudo_j(tree, sp4)
    active = np.arange(n, dtype=np.uint32)
    starts = O.group_starts(tree, n, active, oprm.group_max, oprm.group_mode)
    ng = len(starts) - 1
    rng = np.random.default_rng(seed + 1000)
    perm = rng.permutation(ng)
    sizes = np.diff(starts.astype(np.int64))[perm]
    k = int(np.searchsorted(np.cumsum(sizes), target)) + 1
    gids = np.sort(perm[:min(k, ng)]).astype(np.int64)
    rows = np.concatenate([np.arange(starts[q], starts[q + 1]) for q in gids])
    gI, gamin = O.groups(starts, active, sp4, None)
    boot, _, _ = O.walk(tree, jpos, bj, sp4, active, starts, gI, gamin, 0, oprm.theta, oprm.delta_acc,
                        oprm.eps, oprm.G, group_ids=gids)
    aold_o = O.aold_of(boot[rows].astype(np.float32))
    aold_s = np.zeros(n, np.float32)
    aold_s[rows] = aold_o
    gI, gamin = O.groups(starts, active, sp4, aold_s)
    o2, inter_o, _ = O.walk(tree, jpos, bj, sp4, active, starts, gI, gamin, 1, oprm.theta, oprm.delta_acc,
                            oprm.eps, oprm.G, group_ids=gids)
    o1 = O.direct(sp4, eps, 1.0, rows)
    # GPU: its own opening-angle pass for a_old, the oracle's values on the sampled members
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    s.build_tree()
    acc = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    prm_bh = g.gt_default_params()
    prm_bh.eps, prm_bh.leaf_max, prm_bh.group_mode, prm_bh.mac = eps, leaf, g.GT_GROUP_CELLS, 0
    s.set_params(prm_bh)
    s.accel_active(None, None, acc)
    a = acc.double()
    aold = torch.sqrt((a[:, 0] * a[:, 0] + a[:, 1] * a[:, 1] + a[:, 2] * a[:, 2]).float())
    aold[torch.from_numpy(rows).cuda()] = torch.from_numpy(aold_o).cuda()
    s.set_params(prm)
    i0 = s.stats()["interactions"]
    s.accel_active(None, aold.contiguous(), acc)
    s.sync()
    inter_gpu = s.stats()["interactions"] - i0
    ga = acc.cpu().numpy()[rows]
    s.close()
    return {"model": kind, "n": n, "leaf_max": leaf, "sample_particles": int(len(rows)),
            "sample_groups": int(len(gids)), "groups_total": int(ng),
            "gpu_vs_direct_fp64": _dist(_rel_err(ga, o1)),
            "gpu_vs_oracle_tree": _dist(_rel_err(ga, o2[rows])),
            "oracle_tree_vs_direct_fp64": _dist(_rel_err(o2[rows], o1)),
            "interactions_per_particle": float(inter_gpu / n),
            "seconds": time.perf_counter() - t_all}


def accuracy_sweeps(g, torch, reps: int = 5):
    """Plummer sphere N = 2^13 (G = M = a = 1, eps = 1/64), one force evaluation of every
    particle: the opening-angle MAC for theta = 0.9 ... 0.1 and the acceleration MAC for
    Delta_acc = 2^-2 ... 2^-19 (a_old from the oracle's theta = 0.5 pass), each timed on
    the GPU (walk only, CUDA events, mean of reps) and compared with FP64 direct summation
    over all particles (paper Sec. 3.2, Figs. 3-4)."""
    import oracle as O
    from paper_1610_07279_gb300 import ics
    n = 1 << 13
    pos, vel, mass, eps = ics.plummer(n, seed=1)
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    oprm = O.Params(eps=O.f32(eps), leaf_max=16, group_max=64)
    boot = O.bootstrap_aold(p4, oprm)
    direct = O.direct(p4, eps, 1.0)
    prm = g.gt_default_params()
    prm.eps = eps
    prm.group_mode = g.GT_GROUP_CELLS
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    s.build_tree()
    order = s.get_tree()["order"]
    d_aold = torch.from_numpy(boot[order]).cuda()
    acc = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ref = direct[order]

    def run(mac, theta, dacc):
        p = g.gt_default_params()
        p.eps, p.group_mode, p.mac, p.theta, p.delta_acc = eps, g.GT_GROUP_CELLS, mac, theta, dacc
        s.set_params(p)
        s.accel_active(None, d_aold, acc)
        s.sync()
        i0 = s.stats()["interactions"]
        e0.record(st)
        for _ in range(reps):
            s.accel_active(None, d_aold, acc)
        e1.record(st)
        torch.cuda.synchronize()
        inter = (s.stats()["interactions"] - i0) / reps
        err = _rel_err(acc.cpu().numpy(), ref)
        return {"ms": e0.elapsed_time(e1) / reps, "interactions": inter, **_dist(err)}

    theta = [{"theta": t, **run(0, t, 2.0 ** -7)} for t in (0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3, 0.2, 0.1)]
    dacc = [{"delta_acc_log2": -k, **run(1, 0.5, 2.0 ** -k)} for k in range(2, 20)]
    s.close()
    return {"workload": "Plummer N=2^13, eps=1/64, every particle, error |a - a_direct| / |a_direct| vs "
                        "FP64 direct summation over all particles; ms = one walk launch (tree built once)",
            "opening_angle": theta, "acceleration_mac": dacc}


# ------------------------------------------------------------------ our arm
def walk_traffic_entry(interactions_per_launch: float):
    """DRAM bytes of an average walk launch: the bytes per interaction of the committed ncu
    capture (profiles/walk_traffic.json) scaled by the interactions one launch does here,
    or None once walk.cu has changed since the capture."""
    path = os.path.join(ROOT, "profiles", "walk_traffic.json")
    src = os.path.join(ROOT, "paper_1610_07279_gb300", "csrc", "walk.cu")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("walk_cu_sha256") == h:
            return rec["dram_bytes_per_interaction"] * interactions_per_launch
    except Exception:
        pass
    return None


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1610_07279_gb300 import build as gbuild
    from paper_1610_07279_gb300 import gothic as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    gbuild.build()
    g.load()

    pos, vel, mass, eps = workload(args.n)
    prm = g.gt_default_params()
    prm.eps = eps
    prm.leaf_max = LEAF_MAX
    prm.levels = args.levels
    sysm = g.System(args.n, prm)
    sysm.set_state(pos, vel, mass)
    sysm.start()
    sysm.sync()
    for _ in range(args.warmup):
        sysm.advance_cycle()
    sysm.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    def allreduce(x, op):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=op)
        return float(t.item())

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    # ---- device-resident timed region
    sysm.profile(True)
    st0 = sysm.stats()
    l0 = g.gt_kernel_launches()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    block_steps = 0
    for _ in range(args.steps):
        block_steps += sysm.advance_cycle()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = sysm.stats()
    timers = sysm.timers()
    launches = g.gt_kernel_launches() - l0
    sysm.profile(False)
    inter = st1["interactions"] - st0["interactions"]
    ms_max = allreduce(ms, dist.ReduceOp.MAX if world > 1 else None)
    inter_all = allreduce(float(inter), dist.ReduceOp.SUM if world > 1 else None)
    value = inter_all / (ms_max * 1e-3)

    walk_ms, walk_launches = timers["walk"]
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nsm = props.multi_processor_count
    sm_max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    derived = nsm * 128 * 2 * sm_max_mhz * 1e6 / 1e12  # FP32 lanes x FMA x clock
    rates = g.gt_measure_fp32_rates(stream.cuda_stream)
    fpi = flops_per_interaction(rates["rsqrt_flops"])
    peak = rates["peak_flops"] / 1e12
    achieved = inter * fpi / (walk_ms * 1e-3) / 1e12 if walk_ms > 0 else 0.0
    traffic = walk_traffic_entry(inter / max(walk_launches, 1))
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_basis": "DRAM bytes per interaction of the committed ncu capture of k_walk "
                                 "(profiles/walk_traffic.json) x interactions per launch here",
                "kernel": "k_walk (tree walk + force loop)",
                "flops_per_interaction": fpi,
                "flops_basis": "20 (3 sub, 3 mul, 7 FMA) + rsqrt counted as the measured add/mul : rsqrt "
                               "throughput ratio (the paper's rule, Sec. 4)",
                "peak_basis": "measured: 2 x the faster of the scalar and packed (f32x2) FMA chains on all SMs "
                              "(gt_measure_fp32_rates); the walk's force loop issues the packed form",
                "measured_rates_per_s": {k: rates[k] for k in ("fma_per_s", "fma2_per_s", "add_per_s",
                                                              "mul_per_s", "rsqrt_per_s", "fp64_fma_per_s")},
                "rsqrt_flops_measured": rates["rsqrt_flops"],
                "frac_at_20_flops": inter * FLOPS_BASE / (walk_ms * 1e-3) / 1e12 / peak if walk_ms > 0 else 0.0,
                "derived_peak_tflops": derived,
                "derived_peak_basis": f"{nsm} SMs x 128 FP32 lanes x 2 flops x {sm_max_mhz:.0f} MHz",
                "walk_launches": walk_launches, "walk_ms_avg": walk_ms / max(walk_launches, 1)}

    # ---- end to end through pinned host buffers
    e2e = None
    if not args.no_e2e:
        n = args.n
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True)
        host = {"pos": pin((n, 3), torch.float64), "vel": pin((n, 3), torch.float64),
                "mass": pin((n,), torch.float32), "acc": pin((n, 4), torch.float32),
                "aold": pin((n,), torch.float32), "level": pin((n,), torch.uint8),
                "t0": pin((n,), torch.int64), "id": pin((n,), torch.int32)}
        sysm.get_state(out=host)
        s_e = sysm.stats()
        T, dt_max = s_e["T"], s_e["dt_max"]
        h2d = n * (24 + 24 + 4 + 16 + 4 + 1 + 8)
        d2h = n * (24 + 24 + 4 + 16 + 4 + 1 + 8 + 4)
        barrier()
        torch.cuda.synchronize()
        i0 = sysm.stats()["interactions"]
        t_start = time.perf_counter()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        # the legs of every step, by CUDA events on the stream: inputs in, the cycle, results out
        legs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        for k in range(args.steps):
            legs[k][0].record(stream)
            sysm.set_state(host["pos"], host["vel"], host["mass"])
            sysm.set_integrator_state(host["level"], host["t0"], host["aold"], host["acc"], dt_max, T)
            legs[k][1].record(stream)
            sysm.advance_cycle()
            legs[k][2].record(stream)
            sysm.get_state(out=host)
            legs[k][3].record(stream)
            T = sysm.stats()["T"]
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t_start
        ms_e = f0.elapsed_time(f1)
        i_e = sysm.stats()["interactions"] - i0
        ms_e_max = allreduce(ms_e, dist.ReduceOp.MAX if world > 1 else None)
        i_e_all = allreduce(float(i_e), dist.ReduceOp.SUM if world > 1 else None)
        leg_ms = [sum(legs[k][j].elapsed_time(legs[k][j + 1]) for k in range(args.steps)) / args.steps
                  for j in range(3)]
        e2e = {"value": i_e_all / (ms_e_max * 1e-3), "unit": "interactions/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "wall_s": wall,
               "legs_ms_per_step": {"in": leg_ms[0], "cycle": leg_ms[1], "out": leg_ms[2],
                                    "in_GBps": h2d / (leg_ms[0] * 1e6) if leg_ms[0] > 0 else None,
                                    "out_GBps": d2h / (leg_ms[2] * 1e6) if leg_ms[2] > 0 else None},
               "path": "gt_set_state + gt_set_integrator_state from pinned host, one block-step cycle, "
                       "gt_get_state to pinned host, every step"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_entry(pos, mass, eps, args.cpu_groups)
    dt_max_run = sysm.stats()["dt_max"]
    sysm.close()
    del sysm
    shared = None
    if not args.no_shared:
        shared = run_shared_comparison(g, torch, pos, vel, mass, eps, ms_max / args.steps, inter / args.steps,
                                       dt_max_run, args.levels)
    nfw = errors = None
    if not args.no_nfw:
        nfw = run_nfw_block_steps(g, torch)
    if not args.no_error and rank == 0:
        errors = {"plummer_2p13": error_report(g, torch, "plummer", 1 << 13, 1, 16, 1 << 13),
                  "nfw_2p20": error_report(g, torch, "nfw", 1 << 20, 2, 16, 1 << 13),
                  "m31_2p24": error_report(g, torch, "m31", args.n, 3, LEAF_MAX, 1 << 10,
                                           model=(pos, vel, mass, eps)),
                  "sweeps_plummer_2p13": accuracy_sweeps(g, torch)}
    batch = serving = None
    if not args.no_batch:
        batch = run_batch(g, torch, args.steps, Comm(rank, world))
    if not args.no_serve:
        serving = run_serving(g, torch, args.serve_requests, comm=Comm(rank, world), rhos=
                              [x if x == "burst" else float(x) for x in args.serve_rho.split(",")])

    if rank == 0:
        breakdown = {k: {"ms_total": v[0], "launches": v[1]} for k, v in timers.items()}
        line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config_dict(args, eps),
                "block_step_s": ms_max * 1e-3 / max(block_steps, 1), "block_steps": block_steps,
                "rebuilds": st1["rebuilds"] - st0["rebuilds"],
                "interactions": inter, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "cpu_baseline": cpu, "clocks": clk, "phase_ms": breakdown,
                "block_vs_shared": shared, "nfw_2p20_block_steps": nfw, "error": errors,
                "batch": batch, "serving": serving,
                "gflops_paper_convention": {str(f): inter_all * f / (ms_max * 1e-3) / 1e9
                                            for f in (20, 24, 28, 38, round(fpi, 2))}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
