"""A cache of the batch autotuner's choices, one JSON file, keyed by the device and the
size of the work (the paper tunes its walk parameters per GPU and per problem size,
Sec. 2.4-2.5 and Table 2; a tuning measured once is reused by later batches of the
same kind instead of being timed again).

Key: the device's name and SM count, the number of systems and the total number of
particles, both rounded down to a power of two, and the candidate lists searched (a
different search space is a different question).  The file is rewritten whole through
a temporary file and a rename, so a reader never sees half of it; an unreadable file
counts as empty and is replaced on the next store.
"""
from __future__ import annotations

import json
import os
import tempfile


def bucket(v: int) -> int:
    """The largest power of two not above v (0 for v < 1)."""
    v = int(v)
    return 0 if v < 1 else 1 << (v.bit_length() - 1)


def make_key(device: str, n_sm: int, ns, leaf_max=(), group_max=(), walk_queue=(), reps: int = 3) -> str:
    ns = [int(n) for n in ns]
    parts = [device.strip(), f"sm{int(n_sm)}", f"sys{bucket(len(ns))}", f"n{bucket(sum(ns))}",
             "leaf" + ",".join(str(int(v)) for v in leaf_max),
             "group" + ",".join(str(int(v)) for v in group_max),
             "queue" + ",".join(str(int(v)) for v in walk_queue), f"reps{int(reps)}"]
    return "|".join(parts)


class TuneCache:
    def __init__(self, path: str):
        self.path = path

    def _read(self) -> dict:
        try:
            with open(self.path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            return {}
        return data if isinstance(data, dict) else {}

    def get(self, key: str) -> dict | None:
        v = self._read().get(key)
        if not isinstance(v, dict) or not all(isinstance(v.get(k), int) for k in ("leaf_max", "group_max", "walk_queue")):
            return None
        return v

    def put(self, key: str, result: dict) -> None:
        data = self._read()
        data[key] = {k: result[k] for k in ("leaf_max", "group_max", "walk_queue", "best_ms") if k in result}
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune", dir=d)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise
