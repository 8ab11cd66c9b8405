"""CPU oracle for the block-step oct-tree gravity method (GOTHIC, arXiv:1610.07279).

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this package: only the
tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares no code
with the CUDA path; both take their inputs from the seeded generators only.

The arithmetic lives in ``gothic_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module compiles it, loads it with ctypes and strings
its steps together in the paper's order:

  keys (Sec. 2.1, App. A) -> stable sort (Sec. 2.1) -> breadth-first octree
  (Sec. 2.1) -> pseudo j-particles (Sec. 2.1, Fig. 1) -> groups and pseudo
  i-particles (Sec. 2.3, Fig. 2, App. B) -> tree walk with the MAC (Sec. 2.2-2.3,
  Eqs. 2, 5-7) and Eq. (1) sums -> block-step prediction/correction (Sec. 2.7,
  Eqs. 15-17).

Readings where the paper is silent (bounding cube, leaf size, b_J of a cell,
rounding directions, |a_old| of a group, step criterion, level changes) are
stated next to the C routine that takes them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gothic_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

KEY_LEVELS = 21


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    P = C.c_void_p
    I64, I32, D, F = C.c_int64, C.c_int, C.c_double, C.c_float
    L.or_num_threads.restype = I32
    L.or_set_num_threads.argtypes = [I32]
    L.or_direct.argtypes = [I64, P, D, D, I64, P, P]
    L.or_keys.argtypes = [I64, P, P, P]
    L.or_sort.argtypes = [I64, P, P, P]
    L.or_sort.restype = I32
    L.or_build.argtypes = [I64, P, I32, I64, P, P, P, P, P, P, P]
    L.or_build.restype = I64
    L.or_pseudo_j.argtypes = [I64, P, P, P, P, P, P, P, P]
    L.or_pseudo_j.restype = I32
    L.or_active_prefix.argtypes = [I64, I64, P, P]
    L.or_group_starts.argtypes = [I64, P, P, P, P, P, I32, P, F, P]
    L.or_group_starts.restype = I64
    L.or_groups.argtypes = [I64, P, P, P, P, I32, P, P]
    L.or_walk.argtypes = [I64, P, P, P, P, P, P, P, I64, P, P, P, P, I32, F, F, F, F,
                          I64, P, P, P, P, P]
    L.or_walk.restype = I32
    L.or_dtmax_exponent.argtypes = [I64, P, D, D]
    L.or_dtmax_exponent.restype = I32
    L.or_a2.argtypes = [I64, P, P]
    L.or_aold.argtypes = [I64, P, P]
    L.or_init_levels.argtypes = [I64, P, P, D, D, I32, I32, D, P, P, P, P]
    L.or_predict.argtypes = [I64, P, P, P, P, I64, D, P]
    L.or_correct.argtypes = [I64, P, P, I64, D, I32, I32, D, D, P, P, P, P, P, P]
    L.or_morton3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.or_morton3.restype = C.c_uint64
    L.or_hilbert3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.or_hilbert3.restype = C.c_uint64
    L.or_keys_curve.argtypes = [I64, P, P, P, I32]
    L.or_mac_accept.argtypes = [I32, F, F, F, F, P, P, F, F]
    L.or_mac_accept.restype = I32
    L.or_level_from_a2.argtypes = [D, D, D, I32, I32]
    L.or_level_from_a2.restype = I32


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    lib().or_set_num_threads(int(k))


# ------------------------------------------------------------------ parameters
@dataclass
class Params:
    """Method parameters (the oracle's own copy; mirrors the library's struct)."""
    mac: int = 1               # 0 opening angle (Eq. 2), 1 acceleration (Eq. 5), 2 multipole (Warren-Salmon)
    theta: float = 0.5         # opening angle; also the bootstrap pass's angle
    delta_acc: float = 2.0 ** -7
    eps: float = 1.0 / 64.0
    G: float = 1.0
    leaf_max: int = 16
    group_max: int = 32
    levels: int = 8
    eta: float = 0.025
    dt_max: float = 0.0        # 0: derived at start as a power of two
    group_mode: int = 1        # 1: groups bounded by tree cells; 0: runs of group_max actives
    r_crit: float = 0.0        # critical separation of a group cell's radius (Sec. 2.4); <= 0: none
    rebuild_every: int = 1     # block steps per tree build (Sec. 2.6); the topology is kept between
    sphere: int = 0            # pseudo i-particle: 0 GEO, 1 Ritter's efficient bounding sphere (App. B)
    key_curve: int = 0         # 0 Morton, 1 Peano-Hilbert (Sec. 2.1, App. A)


def f32(x):
    return float(np.float32(x))


# ------------------------------------------------------------------ primitives
def direct(p4: np.ndarray, eps: float, G: float = 1.0, idx=None) -> np.ndarray:
    """Eq. (1) by direct summation in FP64 (potential as 4th column)."""
    p4 = _c(p4, np.float32)
    n = p4.shape[0]
    if idx is None:
        ni, ip = n, None
    else:
        ip = _c(idx, np.int64)
        ni = ip.shape[0]
    out = np.zeros((ni, 4), np.float64)
    lib().or_direct(n, _p(p4), float(eps), float(G), ni, _p(ip), _p(out))
    return out


def keys(p4: np.ndarray, curve: int = 0):
    """63-bit keys of the quantised positions: curve 0 Morton, 1 Peano-Hilbert."""
    p4 = _c(p4, np.float32)
    n = p4.shape[0]
    key = np.zeros(n, np.uint64)
    box = np.zeros(5, np.float64)
    lib().or_keys_curve(n, _p(p4), _p(key), _p(box), int(curve))
    return key, box


def sort(key: np.ndarray):
    key = _c(key, np.uint64)
    n = key.shape[0]
    order = np.zeros(n, np.uint32)
    skey = np.zeros(n, np.uint64)
    if lib().or_sort(n, _p(key), _p(order), _p(skey)) != 0:
        raise MemoryError("oracle sort")
    return order, skey


def build_tree(skey: np.ndarray, leaf_max: int, cap: int | None = None) -> dict:
    skey = _c(skey, np.uint64)
    n = skey.shape[0]
    if cap is None:
        cap = 2 * n + 64
    first = np.zeros(cap, np.uint32)
    count = np.zeros(cap, np.uint32)
    child = np.zeros(cap, np.int32)
    nchild = np.zeros(cap, np.uint8)
    level = np.zeros(cap, np.uint8)
    parent = np.zeros(cap, np.int32)
    lstart = np.zeros(KEY_LEVELS + 2, np.int64)
    nn = lib().or_build(n, _p(skey), int(leaf_max), int(cap), _p(first), _p(count), _p(child),
                        _p(nchild), _p(level), _p(parent), _p(lstart))
    if nn < 0:
        raise OverflowError("oracle tree: node capacity exceeded")
    return {"n_nodes": int(nn), "first": first[:nn].copy(), "count": count[:nn].copy(),
            "child": child[:nn].copy(), "nchild": nchild[:nn].copy(),
            "level": level[:nn].copy(), "parent": parent[:nn].copy(), "level_start": lstart}


def pseudo_j(tree: dict, sp4: np.ndarray, with_b2: bool = False):
    """(jpos, bj), or (jpos, bj, b2) with the second moments B_2 of the multipole MAC."""
    sp4 = _c(sp4, np.float32)
    nn = tree["n_nodes"]
    jpos = np.zeros((nn, 4), np.float32)
    bj = np.zeros(nn, np.float32)
    b2 = np.zeros(nn, np.float32) if with_b2 else None
    rc = lib().or_pseudo_j(nn, _p(tree["first"]), _p(tree["count"]), _p(tree["child"]),
                           _p(tree["nchild"]), _p(sp4), _p(jpos), _p(bj), _p(b2))
    if rc != 0:
        raise MemoryError("oracle pseudo_j")
    return (jpos, bj, b2) if with_b2 else (jpos, bj)


def active_prefix(n: int, active) -> np.ndarray:
    active = _c(active, np.uint32)
    P = np.zeros(n + 1, np.uint32)
    lib().or_active_prefix(n, active.shape[0], _p(active), _p(P))
    return P


def group_starts(tree: dict, n: int, active, gmax: int, mode: int = 1, bj=None, r_crit: float = 0.0) -> np.ndarray:
    """First active position of every group, plus n_active at the end.

    mode 1: groups bounded by tree cells (Sec. 2.4): the cells holding at most gmax
    actives that are leaves or have b_J <= r_crit (r_crit <= 0: no radius limit);
    mode 0: consecutive runs of gmax."""
    active = _c(active, np.uint32)
    na = active.shape[0]
    if mode == 0 or tree["n_nodes"] == 0:
        return np.append(np.arange(0, na, gmax, dtype=np.uint32), np.uint32(na))
    P = active_prefix(n, active)
    starts = np.zeros(na + 1, np.uint32)
    bjv = None if bj is None else _c(bj, np.float32)
    ng = lib().or_group_starts(tree["n_nodes"], _p(tree["first"]), _p(tree["count"]), _p(tree["child"]),
                               _p(tree["parent"]), _p(P), int(gmax), _p(bjv), f32(r_crit), _p(starts))
    return starts[:ng + 1].copy()


def groups(starts, active, sp4: np.ndarray, aold=None, sphere: int = 0):
    """Pseudo i-particles (x, y, z, b_I) and min |a_old| per group; sphere 0: GEO centre,
    1: the centre of Ritter's efficient bounding sphere (Appendix B)."""
    starts = _c(starts, np.uint32)
    active = _c(active, np.uint32)
    sp4 = _c(sp4, np.float32)
    ng = starts.shape[0] - 1
    gI = np.zeros((ng, 4), np.float32)
    gamin = np.zeros(ng, np.float32)
    ao = None if aold is None else _c(aold, np.float32)
    lib().or_groups(ng, _p(starts), _p(active), _p(sp4), _p(ao), int(sphere), _p(gI), _p(gamin))
    return gI, gamin


def walk(tree: dict, jpos, bj, sp4, active, starts, gI, gamin, mac: int, theta: float,
         delta_acc: float, eps: float, G: float, group_ids=None, b2=None):
    """Tree walk for the listed groups (all if None).  Returns (acc, inter, ntest).
    mac 2 (multipole) needs b2 and takes Delta_mul in delta_acc."""
    if mac == 2 and b2 is None:
        raise ValueError("the multipole MAC needs the B_2 moments")
    active = _c(active, np.uint32)
    starts = _c(starts, np.uint32)
    sp4 = _c(sp4, np.float32)
    na = active.shape[0]
    ng = starts.shape[0] - 1
    gids = None if group_ids is None else _c(group_ids, np.int64)
    n_eval = ng if gids is None else gids.shape[0]
    acc = np.full((na, 4), np.nan, np.float64)
    inter = np.full(na, -1, np.int64)
    ntest = np.zeros(n_eval, np.int64)
    rc = lib().or_walk(tree["n_nodes"], _p(_c(jpos, np.float32)), _p(_c(bj, np.float32)),
                       _p(tree["first"]), _p(tree["count"]), _p(tree["child"]), _p(tree["nchild"]),
                       _p(sp4), na, _p(active), _p(starts), _p(_c(gI, np.float32)),
                       _p(_c(gamin, np.float32)), int(mac), f32(theta), f32(delta_acc), f32(eps),
                       f32(G), n_eval, _p(gids), _p(None if b2 is None else _c(b2, np.float32)), _p(acc), _p(inter), _p(ntest))
    if rc != 0:
        raise MemoryError("oracle walk")
    return acc, inter, ntest


def predict(r0, vh, t0, mass, T: int, dt_min: float) -> np.ndarray:
    n = r0.shape[0]
    p4 = np.zeros((n, 4), np.float32)
    lib().or_predict(n, _p(_c(r0, np.float64)), _p(_c(vh, np.float64)), _p(_c(t0, np.int64)),
                     _p(_c(mass, np.float32)), int(T), float(dt_min), _p(p4))
    return p4


def a2(acc4) -> np.ndarray:
    """|a|^2 in FP64 from FP32 components, (ax^2 + ay^2) + az^2."""
    acc4 = _c(acc4, np.float32)
    out = np.zeros(acc4.shape[0], np.float64)
    lib().or_a2(acc4.shape[0], _p(acc4), _p(out))
    return out


def aold_of(acc4) -> np.ndarray:
    """|a_old| = sqrtf((float)|a|^2)."""
    acc4 = _c(acc4, np.float32)
    out = np.zeros(acc4.shape[0], np.float32)
    lib().or_aold(acc4.shape[0], _p(acc4), _p(out))
    return out


def dtmax_exponent(acc4, eta: float, eps: float) -> int:
    acc4 = _c(acc4, np.float32)
    return int(lib().or_dtmax_exponent(acc4.shape[0], _p(acc4), float(eta), float(eps)))


def init_levels(acc4, vel, eta, eps, M, L, dt_max):
    acc4 = _c(acc4, np.float32)
    vel = _c(vel, np.float64)
    n = acc4.shape[0]
    level = np.zeros(n, np.uint8)
    t0 = np.zeros(n, np.int64)
    vh = np.zeros((n, 3), np.float64)
    aold = np.zeros(n, np.float32)
    lib().or_init_levels(n, _p(acc4), _p(vel), float(eta), float(eps), int(M), int(L),
                         float(dt_max), _p(level), _p(t0), _p(vh), _p(aold))
    return level, t0, vh, aold


def correct(active, acc4, T, dt_max, M, L, eta, eps, r0, vh, t0, level, aold, acc_store=None):
    """In-place update of r0, vh, t0, level, aold (and acc_store) for the active set."""
    active = _c(active, np.uint32)
    acc4 = _c(acc4, np.float32)
    for a, dt in ((r0, np.float64), (vh, np.float64), (t0, np.int64), (level, np.uint8),
                  (aold, np.float32)):
        assert a.dtype == dt and a.flags.c_contiguous
    lib().or_correct(active.shape[0], _p(active), _p(acc4), int(T), float(dt_max), int(M), int(L),
                     float(eta), float(eps), _p(r0), _p(vh), _p(t0), _p(level), _p(aold),
                     _p(acc_store))


def hilbert3(qx: int, qy: int, qz: int) -> int:
    return int(lib().or_hilbert3(qx, qy, qz))


def morton3(qx: int, qy: int, qz: int) -> int:
    return int(lib().or_morton3(qx, qy, qz))


def mac_accept(mac: int, theta: float, delta_acc: float, amin: float, G: float, gI, jpos, bJ,
               B2: float = 0.0) -> bool:
    gi = _c(gI, np.float32)
    jp = _c(jpos, np.float32)
    return bool(lib().or_mac_accept(int(mac), f32(theta), f32(delta_acc), f32(amin), f32(G),
                                    _p(gi), _p(jp), f32(bJ), f32(B2)))


def level_from_a2(a2: float, eta: float, eps: float, M: int, L: int) -> int:
    return int(lib().or_level_from_a2(float(a2), float(eta), float(eps), int(M), int(L)))


# ------------------------------------------------------------------ pipelines
def tree_force(p4: np.ndarray, prm: Params, aold=None, active=None, mac=None, theta=None,
               group_ids=None) -> dict:
    """Steps A1-A7 for FP32 particles p4 (n x 4, unsorted).

    aold: |a_old| per particle in the *input* order (needed by the acceleration MAC).
    active: sorted-order indices of the i-particles (all particles if None).
    Returns a dict with the sorted order, keys, tree, pseudo particles, groups and
    the accelerations (rows follow ``active``; column 3 is the potential).
    """
    p4 = _c(p4, np.float32)
    n = p4.shape[0]
    key, box = keys(p4, prm.key_curve)
    order, skey = sort(key)
    sp4 = p4[order]
    tree = build_tree(skey, prm.leaf_max)
    m = prm.mac if mac is None else mac
    jpos, bj, b2 = pseudo_j(tree, sp4, with_b2=True)
    if active is None:
        active = np.arange(n, dtype=np.uint32)
    saold = None if aold is None else _c(aold, np.float32)[order]
    starts = group_starts(tree, n, active, prm.group_max, prm.group_mode, bj, prm.r_crit)
    gI, gamin = groups(starts, active, sp4, saold, prm.sphere)
    th = prm.theta if theta is None else theta
    acc, inter, ntest = walk(tree, jpos, bj, sp4, active, starts, gI, gamin, m, th,
                             prm.delta_acc, prm.eps, prm.G, group_ids, b2)
    return {"key": key, "box": box, "order": order, "skey": skey, "sp4": sp4, "tree": tree,
            "jpos": jpos, "bj": bj, "b2": b2, "active": active, "starts": starts, "gI": gI, "gamin": gamin,
            "acc": acc, "inter": inter, "ntest": ntest}


def bootstrap_aold(p4: np.ndarray, prm: Params) -> np.ndarray:
    """|a| of an opening-angle pass (theta = prm.theta), in input order.

    The acceleration MAC needs |a_old|, which does not exist at t = 0 (the paper is
    silent); the first pass uses the opening-angle MAC and its |a| seeds a_old.
    """
    r = tree_force(p4, prm, mac=0)
    am = aold_of(r["acc"].astype(np.float32))
    out = np.empty_like(am)
    out[r["order"]] = am
    return out


class BlockStepSim:
    """Block time-step integration (Sec. 1; Sec. 2.7) driving the oracle tree force.

    State is kept in sorted (key) order.  Every rebuild_every block steps (Sec. 2.6) the
    predicted positions are keyed and sorted and the tree is built anew; at the other
    steps the previous order and topology are kept and only the pseudo j-particles are
    formed again from the predicted positions.
    """

    def __init__(self, pos, vel, mass, prm: Params):
        self.prm = prm
        n = pos.shape[0]
        self.n = n
        self.L = int(prm.levels)
        self.id = np.arange(n, dtype=np.uint32)
        self.r0 = _c(pos, np.float64).copy()
        self.vh = _c(vel, np.float64).copy()
        self.mass = _c(mass, np.float32).copy()
        self.t0 = np.zeros(n, np.int64)
        self.level = np.zeros(n, np.uint8)
        self.aold = np.zeros(n, np.float32)
        self.acc = np.zeros((n, 4), np.float32)
        self.T = 0
        self.steps = 0
        self.interactions = 0

    # positions as FP32 particles (x, y, z, m)
    def _p4_now(self):
        p4 = np.empty((self.n, 4), np.float32)
        p4[:, :3] = self.r0
        p4[:, 3] = self.mass
        return p4

    def _permute(self, order):
        for name in ("id", "r0", "vh", "mass", "t0", "level", "aold", "acc"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name)[order]))

    def start(self, aold_boot=None):
        """Bootstrap pass, acceleration pass, dt_max, levels and the first half kick."""
        prm = self.prm
        p4 = self._p4_now()
        if aold_boot is None:
            aold_boot = bootstrap_aold(p4, prm)
        r = tree_force(p4, prm, aold=aold_boot)
        self._permute(r["order"])
        acc32 = r["acc"].astype(np.float32)
        self.interactions += int(r["inter"].sum())
        if prm.dt_max > 0:
            self.M = int(np.frexp(prm.dt_max)[1] - 1)
        else:
            self.M = dtmax_exponent(acc32, prm.eta, prm.eps)
        self.dt_max = float(np.ldexp(1.0, self.M))
        vel = self.vh
        self.level, self.t0, self.vh, self.aold = init_levels(acc32, vel, prm.eta, prm.eps,
                                                              self.M, self.L, self.dt_max)
        self.acc = acc32.copy()
        return r

    def ticks(self, level):
        return np.left_shift(np.int64(1), (self.L - 1 - level.astype(np.int64)))

    def next_time(self) -> int:
        return int((self.t0 + self.ticks(self.level)).min())

    def step(self) -> dict:
        prm = self.prm
        T = self.next_time()
        dt_min = float(np.ldexp(self.dt_max, -(self.L - 1)))
        p4 = predict(self.r0, self.vh, self.t0, self.mass, T, dt_min)
        if self.steps % max(1, int(prm.rebuild_every)) == 0 or getattr(self, "tree", None) is None:
            key, _ = keys(p4, prm.key_curve)
            order, skey = sort(key)
            self._permute(order)
            sp4 = np.ascontiguousarray(p4[order])
            tree = build_tree(skey, prm.leaf_max)
            self.tree, self.skey = tree, skey
        else:
            order = np.arange(self.n, dtype=np.uint32)
            sp4, tree, skey = p4, self.tree, self.skey
        jpos, bj, b2 = pseudo_j(tree, sp4, with_b2=True)
        active = np.nonzero(self.t0 + self.ticks(self.level) == T)[0].astype(np.uint32)
        starts = group_starts(tree, self.n, active, prm.group_max, prm.group_mode, bj, prm.r_crit)
        gI, gamin = groups(starts, active, sp4, self.aold, prm.sphere)
        acc, inter, _ = walk(tree, jpos, bj, sp4, active, starts, gI, gamin, prm.mac,
                             prm.theta, prm.delta_acc, prm.eps, prm.G, b2=b2)
        acc32 = acc.astype(np.float32)
        correct(active, acc32, T, self.dt_max, self.M, self.L, prm.eta, prm.eps, self.r0,
                self.vh, self.t0, self.level, self.aold, self.acc)
        self.T = T
        self.steps += 1
        self.interactions += int(inter.sum())
        return {"T": T, "active": active, "acc": acc, "inter": inter, "skey": skey,
                "order": order, "tree": tree, "sp4": sp4, "jpos": jpos, "bj": bj}
