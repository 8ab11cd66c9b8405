"""Python binding of libgothic's C ABI (include/gothic.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The functions keep the C names; ``System`` wraps one ``gt_system`` together with
its device workspace (a torch byte tensor) and the current torch stream.

The library must have been built (``paper_1610_07279_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import re

import numpy as np

from . import build as _build

GT_OK = 0
GT_EINVAL = -1
GT_ENOMEM = -2
GT_EOVERFLOW = -3
GT_ETIMEOUT = -4
GT_ECUDA = -5
GT_EAGAIN = -6
GT_EPENDING = -7
GT_ENOTIMPL = -8
GT_ESTATE = -9
GT_MAC_OPENING_ANGLE = 0
GT_MAC_ACCELERATION = 1
GT_MAC_MULTIPOLE = 2
GT_KEY_MORTON, GT_KEY_HILBERT = 0, 1


class gt_params(C.Structure):
    _fields_ = [("mac", C.c_int32), ("theta", C.c_float), ("delta_acc", C.c_float),
                ("eps", C.c_float), ("G", C.c_float), ("leaf_max", C.c_int32),
                ("group_max", C.c_int32), ("ij_share", C.c_int32), ("levels", C.c_int32),
                ("rebuild_every", C.c_int32), ("walk_queue", C.c_int32), ("node_factor", C.c_int32),
                ("eta", C.c_double), ("dt_max", C.c_double), ("group_mode", C.c_int32),
                ("r_crit", C.c_float), ("key_curve", C.c_int32), ("reserved2", C.c_int32)]


GT_GROUP_RUNS = 0
GT_GROUP_CELLS = 1
GT_GROUP_CELLS_TUNED = 2
GT_SPHERE_EBS = 0x100


class gt_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("T", C.c_int64), ("n_active", C.c_int64),
                ("n_groups", C.c_int64), ("n_nodes", C.c_int64), ("depth", C.c_int64),
                ("interactions", C.c_int64), ("mac_tests", C.c_int64),
                ("block_steps", C.c_int64), ("rebuilds", C.c_int64), ("dt_max", C.c_double),
                ("err", C.c_int32), ("err_where", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gt_fp32_rates(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("fma_per_s", "fma2_per_s", "add_per_s", "mul_per_s", "rsqrt_per_s",
                                          "peak_flops", "rsqrt_flops", "fp64_fma_per_s")]


class GothicError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {gt_strerror(status)} ({status})")
        self.status = status


class gt_tune_space(C.Structure):
    _fields_ = [("n_leaf", C.c_int32), ("leaf_max", C.c_int32 * 8),
                ("n_group", C.c_int32), ("group_max", C.c_int32 * 8),
                ("n_queue", C.c_int32), ("walk_queue", C.c_int32 * 4),
                ("reps", C.c_int32)]


class gt_tune_result(C.Structure):
    _fields_ = [("leaf_max", C.c_int32), ("group_max", C.c_int32), ("walk_queue", C.c_int32),
                ("n_tried", C.c_int32), ("best_ms", C.c_double), ("ms", C.c_double * 256)]


BRENT_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)
GT_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
GT_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
GT_SERVER_MAX_SLOTS = 256
GT_REQ_UNKNOWN, GT_REQ_RUNNING, GT_REQ_DONE = 0, 1, 2


class gt_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("p_pos", C.c_void_p), ("p_vel", C.c_void_p), ("p_mass", C.c_void_p),
                ("params", gt_params), ("nsteps", C.c_int32), ("reserved", C.c_int32)]


class gt_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("ticks", "admitted", "completed", "slots_used", "hbm_used",
                                         "hbm_cap", "walk_launches", "reserved")]


_lib = None


def lib_path() -> str:
    return _build.LIB


def declared_symbols() -> list[str]:
    """Entry points declared in include/gothic.h."""
    with open(os.path.join(_build.INCLUDE, "gothic.h")) as f:
        text = f.read()
    return re.findall(r"^GT_API\s+[\w\s\*]*?\b(gt_\w+)\s*\(", text, flags=re.M)


def load(path: str | None = None):
    """Load libgothic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path or _build.LIB)
    return _lib


def open_library(p: str):
    """Open one build of the library (the release one, or a variant such as the debug
    build) with every entry point declared; ``using`` makes the bindings call it."""
    if not os.path.exists(p):
        raise ImportError(f"libgothic is not built ({p}); run paper_1610_07279_gb300.build.build()")
    L = C.CDLL(p)
    P, I64, I32 = C.c_void_p, C.c_int64, C.c_int
    L.gt_strerror.restype = C.c_char_p
    L.gt_strerror.argtypes = [I32]
    L.gt_default_params.argtypes = [C.POINTER(gt_params)]
    L.gt_workspace_bytes.argtypes = [I64, C.POINTER(gt_params), C.POINTER(C.c_size_t)]
    L.gt_system_create.argtypes = [C.POINTER(P), I64, C.POINTER(gt_params), P, C.c_size_t]
    L.gt_system_destroy.argtypes = [P]
    L.gt_set_params.argtypes = [P, C.POINTER(gt_params)]
    L.gt_set_state.argtypes = [P, P, P, P, P]
    L.gt_build_tree.argtypes = [P, P]
    L.gt_accel_active.argtypes = [P, P, I64, P, P, P]
    L.gt_start.argtypes = [P, P, P]
    L.gt_block_step.argtypes = [P, P]
    L.gt_set_integrator_state.argtypes = [P, P, P, P, P, C.c_double, I64, P]
    L.gt_predict.argtypes = [P, I64, P, P]
    L.gt_correct.argtypes = [P, P, I64, P, I64, P]
    L.gt_get_state.argtypes = [P, P, P, P, P, P, P, P, P, P]
    L.gt_advance.argtypes = [P, I64, C.POINTER(I64), P]
    L.gt_profile.argtypes = [P, I32]
    L.gt_get_timers.argtypes = [P, C.POINTER(C.c_double), C.POINTER(I64), P]
    L.gt_kernel_launches.argtypes = [C.POINTER(I64)]
    L.gt_sort_pairs_noalloc.argtypes = [P, P, I64, P]
    L.gt_sort_noalloc_status.argtypes = [P]
    L.gt_set_wait_limit.argtypes = [P, C.c_uint32, P]
    L.gt_probe_bounded_wait.argtypes = [P, C.c_uint32, P]
    L.gt_rebuild_interval.argtypes = [C.POINTER(C.c_double), I32, C.c_double, C.POINTER(I32),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.gt_get_tree.argtypes = [P, P, P, P, P, P, C.POINTER(I64), P]
    L.gt_get_active.argtypes = [P, P, C.POINTER(I64), P]
    L.gt_sync_status.argtypes = [P, P]
    L.gt_get_stats.argtypes = [P, C.POINTER(gt_stats), P]
    L.gt_measure_fp32_peak.argtypes = [C.POINTER(C.c_double), P]
    L.gt_measure_fp32_rates.argtypes = [C.POINTER(gt_fp32_rates), P]
    L.gt_brent_minimize.argtypes = [BRENT_FN, P, C.c_double, C.c_double, C.c_double, I32,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(I32)]
    L.gt_batch_workspace_bytes.argtypes = [I32, P, P, I32, C.POINTER(C.c_size_t)]
    L.gt_batch_create.argtypes = [C.POINTER(P), I32, P, P, I32, P, C.c_size_t]
    L.gt_batch_destroy.argtypes = [P]
    L.gt_batch_system.argtypes = [P, I32, C.POINTER(P)]
    L.gt_batch_set_knobs.argtypes = [P, I32, I32, I32]
    L.gt_batch_accel.argtypes = [P, I32, P]
    L.gt_batch_capture.argtypes = [P, I32, P]
    L.gt_batch_launch.argtypes = [P, P]
    L.gt_batch_get_acc.argtypes = [P, I32, P, P, P]
    L.gt_batch_sync_status.argtypes = [P, P, P]
    L.gt_batch_autotune.argtypes = [P, C.POINTER(gt_tune_space), C.POINTER(gt_tune_result), P]
    L.gt_server_create.argtypes = [C.POINTER(P), C.c_size_t, I32, I32, GT_ALLOC_FN, GT_FREE_FN, P]
    L.gt_server_destroy.argtypes = [P]
    L.gt_submit.argtypes = [P, C.POINTER(gt_request), C.POINTER(C.c_uint64)]
    L.gt_server_progress.argtypes = [P, C.POINTER(I32)]
    L.gt_poll.argtypes = [P, C.c_uint64, C.POINTER(I32), P, P]
    L.gt_server_get_stats.argtypes = [P, C.POINTER(gt_server_stats)]
    for name in declared_symbols():
        getattr(L, name).restype = C.c_char_p if name == "gt_strerror" else C.c_int
    return L


@contextlib.contextmanager
def using(lib):
    """Make every binding of this module call ``lib`` (from open_library) inside the block."""
    global _lib
    saved = load()
    _lib = lib
    try:
        yield lib
    finally:
        _lib = saved


def _check(rc: int, where: str):
    if rc != GT_OK:
        raise GothicError(rc, where)


# --------------------------------------------------------------- same-named calls
def gt_strerror(status: int) -> str:
    return load().gt_strerror(int(status)).decode()


def gt_default_params() -> gt_params:
    p = gt_params()
    _check(load().gt_default_params(C.byref(p)), "gt_default_params")
    return p


def gt_workspace_bytes(n: int, prm: gt_params) -> int:
    b = C.c_size_t(0)
    _check(load().gt_workspace_bytes(int(n), C.byref(prm), C.byref(b)), "gt_workspace_bytes")
    return int(b.value)


def gt_measure_fp32_peak(stream: int | None = None) -> float:
    f = C.c_double(0.0)
    _check(load().gt_measure_fp32_peak(C.byref(f), stream), "gt_measure_fp32_peak")
    return float(f.value)


def gt_measure_fp32_rates(stream: int | None = None) -> dict:
    """FP32 instruction throughputs (lane operations/s), the FP32 peak in flop/s and the
    flops one rsqrt counts for under the paper's convention."""
    r = gt_fp32_rates()
    _check(load().gt_measure_fp32_rates(C.byref(r), stream), "gt_measure_fp32_rates")
    return {k: float(getattr(r, k)) for k, _ in gt_fp32_rates._fields_}


PHASES = ("predict", "keys_sort", "permute", "build", "pseudo_j", "active", "walk", "correct")


def gt_kernel_launches() -> int:
    c = C.c_int64(0)
    _check(load().gt_kernel_launches(C.byref(c)), "gt_kernel_launches")
    return int(c.value)


def gt_rebuild_interval(t_walk, t_make: float):
    """(model, n_opt, coef) of the rebuild-interval fit (host only, no GPU needed)."""
    t = np.ascontiguousarray(t_walk, np.float64)
    model = C.c_int(0)
    nopt = C.c_double(0.0)
    coef = (C.c_double * 3)()
    _check(load().gt_rebuild_interval(t.ctypes.data_as(C.POINTER(C.c_double)), int(t.size), float(t_make),
                                      C.byref(model), C.byref(nopt), coef), "gt_rebuild_interval")
    return int(model.value), float(nopt.value), [float(c) for c in coef]


def gt_brent_minimize(f, lo: float, hi: float, tol: float = 1e-8, max_evals: int = 100):
    """(x_min, f_min, evaluations) of Brent's minimisation of f on [lo, hi] (host only)."""
    cb = BRENT_FN(lambda x, ctx: float(f(x)))
    x, fx, ev = C.c_double(0.0), C.c_double(0.0), C.c_int32(0)
    _check(load().gt_brent_minimize(cb, None, float(lo), float(hi), float(tol), int(max_evals), C.byref(x),
                                    C.byref(fx), C.byref(ev)), "gt_brent_minimize")
    return float(x.value), float(fx.value), int(ev.value)


GT_NOALLOC_SORT_MAX = 1 << 20


def gt_sort_pairs_noalloc(d_keys, d_vals, n: int, stream: int | None = None):
    """Stable in-place sort of n (uint64 key, uint32 value) device pairs by key, using
    the library's static scratch instead of any allocation (n <= GT_NOALLOC_SORT_MAX)."""
    st = stream if stream is not None else _current_stream()
    _check(load().gt_sort_pairs_noalloc(_ptr(d_keys), _ptr(d_vals), int(n), st), "gt_sort_pairs_noalloc")


def gt_sort_noalloc_status(stream: int | None = None) -> int:
    """Latched device status of the no-allocation sort on this device (read and cleared)."""
    st = stream if stream is not None else _current_stream()
    return int(load().gt_sort_noalloc_status(st))


def _ptr(a):
    """Device or host address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(type(a))


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class System:
    """One N-body system: a gt_system living in a torch-allocated workspace."""

    def __init__(self, n: int, params: gt_params | None = None, stream: int | None = None):
        import torch
        self.n = int(n)
        self.params = params if params is not None else gt_default_params()
        nbytes = gt_workspace_bytes(self.n, self.params)
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        self.stream = stream
        self._h = C.c_void_p()
        _check(load().gt_system_create(C.byref(self._h), self.n, C.byref(self.params),
                                       self.ws.data_ptr(), self.ws.numel()), "gt_system_create")

    @classmethod
    def _member(cls, handle, n: int, params: gt_params, owner, stream):
        """A view of a batch member (owned and destroyed by the batch)."""
        s = cls.__new__(cls)
        s.n, s.params, s.ws, s.stream, s._h, s._owner = int(n), params, None, stream, handle, owner
        return s

    # stream defaults to torch's current stream at call time
    def _s(self):
        return self.stream if self.stream is not None else _current_stream()

    def close(self):
        if getattr(self, "_owner", None) is not None:  # a batch member: the batch destroys it
            self._h = C.c_void_p()
            return
        if self._h:
            load().gt_system_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: gt_params):
        _check(load().gt_set_params(self._h, C.byref(params)), "gt_set_params")
        self.params = params

    def set_state(self, pos, vel, mass):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, np.float64)
            vel = np.ascontiguousarray(vel, np.float64)
            mass = np.ascontiguousarray(mass, np.float32)
        self._keep = (pos, vel, mass)
        _check(load().gt_set_state(self._h, _ptr(pos), _ptr(vel), _ptr(mass), self._s()), "gt_set_state")

    def build_tree(self):
        _check(load().gt_build_tree(self._h, self._s()), "gt_build_tree")

    def accel_active(self, active, aold, acc_out, n_active: int | None = None):
        na = self.n if active is None else (int(n_active) if n_active is not None else int(active.numel()))
        _check(load().gt_accel_active(self._h, _ptr(active), na, _ptr(aold), _ptr(acc_out), self._s()),
               "gt_accel_active")

    def start(self, aold_boot=None):
        if isinstance(aold_boot, np.ndarray):
            aold_boot = np.ascontiguousarray(aold_boot, np.float32)
        _check(load().gt_start(self._h, _ptr(aold_boot), self._s()), "gt_start")

    def block_step(self):
        _check(load().gt_block_step(self._h, self._s()), "gt_block_step")

    def set_integrator_state(self, level, t0, aold, acc, dt_max: float, T: int):
        def host(a, dt):
            if a is None or hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dt)
        arrs = [host(level, np.uint8), host(t0, np.int64), host(aold, np.float32), host(acc, np.float32)]
        _check(load().gt_set_integrator_state(self._h, *[_ptr(a) for a in arrs], float(dt_max), int(T),
                                              self._s()), "gt_set_integrator_state")

    def predict(self, T: int, posm_out):
        _check(load().gt_predict(self._h, int(T), _ptr(posm_out), self._s()), "gt_predict")

    def correct(self, active, acc, T: int):
        _check(load().gt_correct(self._h, _ptr(active), int(active.numel()), _ptr(acc), int(T), self._s()),
               "gt_correct")

    def advance(self, T_end: int) -> int:
        k = C.c_int64(0)
        _check(load().gt_advance(self._h, int(T_end), C.byref(k), self._s()), "gt_advance")
        return int(k.value)

    def advance_cycle(self) -> int:
        """Block steps up to the next multiple of 2^(L-1) ticks (one full cycle)."""
        span = 1 << (self.params.levels - 1)
        T = self.stats()["T"]
        return self.advance((T // span + 1) * span)

    def profile(self, enable: bool = True):
        _check(load().gt_profile(self._h, int(bool(enable))), "gt_profile")

    def timers(self) -> dict:
        ms = (C.c_double * len(PHASES))()
        cnt = (C.c_int64 * len(PHASES))()
        _check(load().gt_get_timers(self._h, ms, cnt, self._s()), "gt_get_timers")
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def get_state(self, out: dict | None = None) -> dict:
        """State in internal order (host numpy arrays, or the caller's buffers in ``out``)."""
        n = self.n
        if out is None:
            out = {"pos": np.zeros((n, 3)), "vel": np.zeros((n, 3)), "mass": np.zeros(n, np.float32),
                   "acc": np.zeros((n, 4), np.float32),
                   "aold": np.zeros(n, np.float32), "level": np.zeros(n, np.uint8),
                   "t0": np.zeros(n, np.int64), "id": np.zeros(n, np.uint32)}
        _check(load().gt_get_state(self._h, _ptr(out.get("pos")), _ptr(out.get("vel")), _ptr(out.get("mass")),
                                   _ptr(out.get("acc")),
                                   _ptr(out.get("aold")), _ptr(out.get("level")), _ptr(out.get("t0")),
                                   _ptr(out.get("id")), self._s()), "gt_get_state")
        self.sync()
        return out

    def get_tree(self) -> dict:
        n = self.n
        cnt = C.c_int64(0)
        _check(load().gt_get_tree(self._h, None, None, None, None, None, C.byref(cnt), self._s()), "gt_get_tree")
        nn = int(cnt.value)
        keys = np.zeros(n, np.uint64)
        order = np.zeros(n, np.uint32)
        nodes = np.zeros((max(nn, 1), 4), np.uint32)
        jpos = np.zeros((max(nn, 1), 4), np.float32)
        bj = np.zeros(max(nn, 1), np.float32)
        cnt = C.c_int64(max(nn, 1))
        _check(load().gt_get_tree(self._h, _ptr(keys), _ptr(order), _ptr(nodes), _ptr(jpos), _ptr(bj),
                                  C.byref(cnt), self._s()), "gt_get_tree")
        nn = int(cnt.value)
        return {"keys": keys, "order": order, "first": nodes[:nn, 0].copy(), "count": nodes[:nn, 1].copy(),
                "child": nodes[:nn, 2].view(np.int32).copy(), "nchild": nodes[:nn, 3].copy(),
                "jpos": jpos[:nn].copy(), "bj": bj[:nn].copy(), "n_nodes": nn}

    def get_active(self) -> np.ndarray:
        cnt = C.c_int64(0)
        _check(load().gt_get_active(self._h, None, C.byref(cnt), self._s()), "gt_get_active")
        buf = np.zeros(max(int(cnt.value), 1), np.uint32)
        cnt = C.c_int64(buf.size)
        _check(load().gt_get_active(self._h, _ptr(buf), C.byref(cnt), self._s()), "gt_get_active")
        return buf[:int(cnt.value)].copy()

    def sync(self):
        _check(load().gt_sync_status(self._h, self._s()), "device")

    def status(self) -> int:
        return int(load().gt_sync_status(self._h, self._s()))

    def set_wait_limit(self, iterations: int):
        _check(load().gt_set_wait_limit(self._h, int(iterations), self._s()), "gt_set_wait_limit")

    def probe_bounded_wait(self, iterations: int) -> int:
        """Status of a look-back whose predecessor never publishes (GT_ETIMEOUT expected)."""
        return int(load().gt_probe_bounded_wait(self._h, int(iterations), self._s()))

    def stats(self) -> dict:
        st = gt_stats()
        _check(load().gt_get_stats(self._h, C.byref(st), self._s()), "gt_get_stats")
        return st.as_dict()


class Batch:
    """Many independent systems: forked tree builds and one walk launch over all of
    them (gt_batch_*).  The batch runs on a stream of its own (capture needs a stream
    other than the legacy default one); its members use the same stream."""

    def __init__(self, ns, params, stream: int | None = None):
        import torch
        self.ns = [int(n) for n in ns]
        k = len(self.ns)
        plist = list(params) if isinstance(params, (list, tuple)) else [params]
        if len(plist) not in (1, k):
            raise ValueError("one params for all systems, or one per system")
        self.params = plist
        self._nn = np.ascontiguousarray(self.ns, np.int64)
        self._pp = (gt_params * len(plist))(*plist)
        b = C.c_size_t(0)
        _check(load().gt_batch_workspace_bytes(k, self._nn.ctypes.data, C.addressof(self._pp), len(plist),
                                               C.byref(b)), "gt_batch_workspace_bytes")
        self.ws = torch.empty(max(int(b.value), 256), dtype=torch.uint8, device="cuda")
        if stream is None:
            self._torch_stream = torch.cuda.Stream()
            stream = self._torch_stream.cuda_stream
        self.stream = stream
        self._h = C.c_void_p()
        _check(load().gt_batch_create(C.byref(self._h), k, self._nn.ctypes.data, C.addressof(self._pp),
                                      len(plist), self.ws.data_ptr(), self.ws.numel()), "gt_batch_create")
        self.systems = []
        for i in range(k):
            h = C.c_void_p()
            _check(load().gt_batch_system(self._h, i, C.byref(h)), "gt_batch_system")
            self.systems.append(System._member(h, self.ns[i], plist[0 if len(plist) == 1 else i], self, stream))

    def close(self):
        if self._h:
            for s in self.systems:
                s.close()
            load().gt_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.ns)

    def set_knobs(self, leaf_max: int = 0, group_max: int = 0, walk_queue: int = 0):
        _check(load().gt_batch_set_knobs(self._h, int(leaf_max), int(group_max), int(walk_queue)),
               "gt_batch_set_knobs")

    def accel(self, bootstrap: bool = False):
        _check(load().gt_batch_accel(self._h, int(bool(bootstrap)), self.stream), "gt_batch_accel")

    def capture(self, bootstrap: bool = False):
        _check(load().gt_batch_capture(self._h, int(bool(bootstrap)), self.stream), "gt_batch_capture")

    def launch(self):
        _check(load().gt_batch_launch(self._h, self.stream), "gt_batch_launch")

    def get_acc(self, k: int, out=None, ids=None):
        """(acc (n, 4) float32, id (n,) uint32) of member k in internal order."""
        n = self.ns[k]
        acc = out if out is not None else np.zeros((max(n, 1), 4), np.float32)
        idv = ids if ids is not None else np.zeros(max(n, 1), np.uint32)
        _check(load().gt_batch_get_acc(self._h, int(k), _ptr(acc), _ptr(idv), self.stream), "gt_batch_get_acc")
        return acc, idv

    def sync(self) -> np.ndarray:
        """Raise on any member's device error; interactions counted so far per member."""
        inter = np.zeros(len(self.ns), np.int64)
        _check(load().gt_batch_sync_status(self._h, inter.ctypes.data, self.stream), "device")
        return inter

    def autotune(self, leaf_max=(), group_max=(), walk_queue=(), reps: int = 3, cache: str | None = None) -> dict:
        """Time every candidate and keep the fastest (gt_batch_autotune).  With ``cache`` (a
        JSON file path) a choice stored for the same device, size class and candidates is
        set on the batch without timing, and a new one is stored."""
        key = None
        if cache:
            import torch
            from . import tune_cache
            dev = torch.cuda.get_device_properties(torch.cuda.current_device())
            key = tune_cache.make_key(dev.name, dev.multi_processor_count, self.ns, leaf_max, group_max,
                                      walk_queue, reps)
            hit = tune_cache.TuneCache(cache).get(key)
            if hit is not None:
                self.set_knobs(hit["leaf_max"], hit["group_max"], hit["walk_queue"])
                return {"leaf_max": hit["leaf_max"], "group_max": hit["group_max"],
                        "walk_queue": hit["walk_queue"], "best_ms": hit.get("best_ms"), "ms": [], "cached": True}
        sp = gt_tune_space()
        sp.n_leaf, sp.n_group, sp.n_queue, sp.reps = len(leaf_max), len(group_max), len(walk_queue), int(reps)
        for i, v in enumerate(leaf_max):
            sp.leaf_max[i] = int(v)
        for i, v in enumerate(group_max):
            sp.group_max[i] = int(v)
        for i, v in enumerate(walk_queue):
            sp.walk_queue[i] = int(v)
        r = gt_tune_result()
        _check(load().gt_batch_autotune(self._h, C.byref(sp), C.byref(r), self.stream), "gt_batch_autotune")
        out = {"leaf_max": r.leaf_max, "group_max": r.group_max, "walk_queue": r.walk_queue,
               "best_ms": r.best_ms, "ms": [float(r.ms[i]) for i in range(r.n_tried)], "cached": False}
        if key is not None:
            from . import tune_cache
            tune_cache.TuneCache(cache).put(key, out)
        return out


class Server:
    """Continuous batching of block-step requests (gt_server_*), device memory from
    torch's caching allocator through the library's allocation callbacks."""

    def __init__(self, hbm_cap: int, max_slots: int = 64, walk_queue: int = 16384):
        import torch
        self._blocks = {}

        def _alloc(nbytes, ctx):
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            except RuntimeError:
                return None
            self._blocks[t.data_ptr()] = t
            return t.data_ptr()

        def _free(ptr, ctx):
            self._blocks.pop(int(ptr), None)

        self._alloc_cb, self._free_cb = GT_ALLOC_FN(_alloc), GT_FREE_FN(_free)
        self._h = C.c_void_p()
        _check(load().gt_server_create(C.byref(self._h), int(hbm_cap), int(max_slots), int(walk_queue),
                                       self._alloc_cb, self._free_cb, None), "gt_server_create")

    def close(self):
        if self._h:
            load().gt_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, pos, vel, mass, params: gt_params, nsteps: int):
        """Ticket of the admitted request, or None when it must wait (no slot / memory)."""
        pos = np.ascontiguousarray(pos, np.float64) if isinstance(pos, np.ndarray) else pos
        vel = np.ascontiguousarray(vel, np.float64) if isinstance(vel, np.ndarray) else vel
        mass = np.ascontiguousarray(mass, np.float32) if isinstance(mass, np.ndarray) else mass
        r = gt_request()
        r.n = int(mass.shape[0])
        r.p_pos, r.p_vel, r.p_mass = _ptr(pos), _ptr(vel), _ptr(mass)
        r.params = params
        r.nsteps = int(nsteps)
        t = C.c_uint64(0)
        rc = load().gt_submit(self._h, C.byref(r), C.byref(t))
        if rc == GT_EAGAIN:
            return None
        _check(rc, "gt_submit")
        return int(t.value)

    def progress(self) -> int:
        running = C.c_int32(0)
        _check(load().gt_server_progress(self._h, C.byref(running)), "gt_server_progress")
        return int(running.value)

    def poll(self, ticket: int, pos_out=None, vel_out=None):
        """True once the request is done (its state written to the outputs), else False."""
        state = C.c_int32(0)
        rc = load().gt_poll(self._h, C.c_uint64(ticket), C.byref(state), _ptr(pos_out), _ptr(vel_out))
        if rc == GT_EPENDING:
            return False
        _check(rc, "gt_poll")
        return state.value == GT_REQ_DONE

    def stats(self) -> dict:
        st = gt_server_stats()
        _check(load().gt_server_get_stats(self._h, C.byref(st)), "gt_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in gt_server_stats._fields_ if k != "reserved"}

