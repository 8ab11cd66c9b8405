"""Small, fixed cases for profiling single kernels under a profiler.

    python -m paper_1610_07279_gb300.profile_cases walk  --model m31 --n 4194304
    python -m paper_1610_07279_gb300.profile_cases build --model m31 --n 2097152 --repeat 3
    python -m paper_1610_07279_gb300.profile_cases steps --model m31 --n 2097152 --steps 16

walk:  tree build, one opening-angle walk of every particle (the start-up pass), then
       one acceleration-MAC walk of every particle (the second k_walk launch).
build: the tree build (keys, sort, permute, octree, cell lists, pseudo j) repeated.
steps: start-up and block steps with the automatic rebuild interval.
Each case prints one line with its timings and counts; inputs are the seeded models of
``ics`` (the same generators the benchmark uses).
"""
from __future__ import annotations

import argparse

from . import build as _build
from . import gothic as g
from . import ics

def _uniform(n: int, seed: int = 7):
    """Particles uniform in the unit cube at rest (a shallow tree of nearly equal leaves)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32).astype(np.float64)
    return pos, np.zeros_like(pos), np.full(n, np.float32(1.0 / n)), 1.0 / 256


MODELS = {"m31": ics.andromeda_like, "nfw": ics.nfw, "plummer": ics.plummer, "uniform": _uniform}


KNOBS = {}  # parameter overrides from the command line


def _system(model: str, n: int, seed: int):
    pos, vel, mass, eps = MODELS[model](n, seed=seed)
    prm = g.gt_default_params()
    prm.eps = eps
    for k, v in KNOBS.items():
        setattr(prm, k, v)
    s = g.System(n, prm)
    s.set_state(pos, vel, mass)
    return s, prm


def case_walk(model: str, n: int, seed: int, repeat: int = 1) -> str:
    import torch
    s, prm = _system(model, n, seed)
    s.build_tree()
    acc = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    boot = g.gt_params.from_buffer_copy(prm)
    boot.mac = g.GT_MAC_OPENING_ANGLE
    s.set_params(boot)
    s.accel_active(None, None, acc)
    s.sync()
    aold = torch.linalg.norm(acc[:, :3].double(), dim=1).float().contiguous()
    s.set_params(prm)
    st0 = s.stats()
    s.accel_active(None, aold, acc)
    s.sync()
    st1 = s.stats()
    inter = st1["interactions"] - st0["interactions"]
    tests = st1["mac_tests"] - st0["mac_tests"]
    # the same walk timed again with CUDA events (mean of `repeat` launches)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(repeat):
        s.accel_active(None, aold, acc)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(repeat, 1)
    s.close()
    return (f"walk {model} n={n} nodes={st1['n_nodes']} depth={st1['depth']} interactions={inter} "
            f"mac_tests={tests} acc_walk_ms={ms:.4f} ns_per_interaction={ms * 1e6 / max(inter, 1):.4f}")


def case_build(model: str, n: int, seed: int, repeat: int) -> str:
    s, _ = _system(model, n, seed)
    s.profile(True)
    for _ in range(repeat):
        s.build_tree()
    s.sync()
    tm = s.timers()
    st = s.stats()
    s.close()
    return (f"build {model} n={n} nodes={st['n_nodes']} depth={st['depth']} "
            + " ".join(f"{k}_ms={v[0] / max(v[1], 1):.3f}" for k, v in tm.items() if v[1]))


def case_steps(model: str, n: int, seed: int, steps: int) -> str:
    s, _ = _system(model, n, seed)
    s.start()
    s.profile(True)
    for _ in range(steps):
        s.block_step()
    s.sync()
    tm = s.timers()
    st = s.stats()
    s.close()
    return (f"steps {model} n={n} block_steps={st['block_steps']} rebuilds={st['rebuilds']} "
            + " ".join(f"{k}_ms={v[0]:.3f}" for k, v in tm.items() if v[1]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["walk", "build", "steps"])
    ap.add_argument("--model", choices=sorted(MODELS), default="m31")
    ap.add_argument("--n", type=int, default=1 << 21)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--group-max", type=int, default=0)
    ap.add_argument("--leaf-max", type=int, default=0)
    ap.add_argument("--rebuild-every", type=int, default=-1, help="fixed rebuild interval (0: automatic)")
    a = ap.parse_args(argv)
    if a.group_max:
        KNOBS["group_max"] = a.group_max
    if a.leaf_max:
        KNOBS["leaf_max"] = a.leaf_max
    if a.rebuild_every >= 0:
        KNOBS["rebuild_every"] = a.rebuild_every
    _build.build()
    g.load()
    if a.case == "walk":
        print(case_walk(a.model, a.n, a.seed, a.repeat), flush=True)
    elif a.case == "build":
        print(case_build(a.model, a.n, a.seed, a.repeat), flush=True)
    else:
        print(case_steps(a.model, a.n, a.seed, a.steps), flush=True)


if __name__ == "__main__":
    main()
