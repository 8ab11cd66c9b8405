"""Work partitioning across GPUs (one process per GPU).

Independent systems (a batch, a serving stream) shard with no exchange at all: each
rank takes whole systems, balanced by the device memory they need.  A single system
does not shard in the paper's design (one GPU); the split available to it is over
the groups of i-particles of a replicated tree (Sec. 2.3: groups are independent),
which needs one gather of the ranks' accelerations per force evaluation.
"""
from __future__ import annotations


def assign_systems(nbytes, world: int) -> list[list[int]]:
    """Whole systems to ranks, largest first onto the least-loaded rank (greedy
    longest-processing-time); returns, per rank, its system indices in ascending
    order.  Deterministic: ties go to the lower rank and the lower index."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(nbytes)), key=lambda k: (-int(nbytes[k]), k))
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(nbytes[k])
    return [sorted(v) for v in out]


def shard_requests(work, world: int) -> list[list[int]]:
    """Requests of a serving stream to ranks, in arrival order, each onto the rank with
    the least work assigned so far (work[k]: an estimate such as particles x steps);
    returns, per rank, its request indices in arrival order.  Every rank computes the
    same plan from the same stream, so no exchange is needed to agree on it."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for k, w in enumerate(work):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += float(w)
    return out


def group_slice(n_groups: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous groups [g0, g1) of one rank: the first n_groups % world ranks take
    one group more."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(int(n_groups), world)
    g0 = rank * base + min(rank, extra)
    return g0, g0 + base + (1 if rank < extra else 0)
