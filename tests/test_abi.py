"""The C-ABI library builds, loads and exports every entry point of include/gothic.h
(no GPU needed: only symbol lookup, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1610_07279_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    from paper_1610_07279_gb300 import gothic
    names = gothic.declared_symbols()
    for must in ("gt_build_tree", "gt_accel_active", "gt_block_step", "gt_start", "gt_get_state",
                 "gt_workspace_bytes", "gt_system_create", "gt_sync_status"):
        assert must in names
    assert len(names) == len(set(names))


def test_library_exports_every_declared_symbol(libpath):
    from paper_1610_07279_gb300 import gothic
    lib = ctypes.CDLL(libpath)
    for name in gothic.declared_symbols():
        assert hasattr(lib, name), name


def test_debug_build_exports_the_same_abi_and_using_switches_back(libpath):
    """The debug variant (index checks, its own directory) builds, exports every declared
    entry point, and gothic.using() points the bindings at it and back."""
    from paper_1610_07279_gb300 import build, gothic
    dpath = build.build(variant="debug")
    assert os.path.dirname(dpath) != os.path.dirname(libpath)
    dbg = gothic.open_library(dpath)
    for name in gothic.declared_symbols():
        assert hasattr(dbg, name), name
    rel = gothic.load()
    with gothic.using(dbg):
        assert gothic.load() is dbg
        assert gothic.gt_strerror(0) == "ok"
        assert gothic.gt_default_params().leaf_max > 0
    assert gothic.load() is rel


def test_binding_loads_and_strerror(libpath):
    from paper_1610_07279_gb300 import gothic
    gothic.load()
    assert gothic.gt_strerror(0) == "ok"
    assert "overflow" in gothic.gt_strerror(gothic.GT_EOVERFLOW)


def test_struct_layout_matches_header(libpath):
    from paper_1610_07279_gb300 import gothic
    assert ctypes.sizeof(gothic.gt_params) == 80 and gothic.gt_params.node_factor.offset == 44
    assert gothic.gt_params.key_curve.offset == 72
    assert gothic.gt_params.group_mode.offset == 64
    assert gothic.gt_params.eta.offset == 48
    assert ctypes.sizeof(gothic.gt_stats) == 96
    assert ctypes.sizeof(gothic.gt_tune_space) == 96 and ctypes.sizeof(gothic.gt_tune_result) == 2072
    assert gothic.gt_tune_result.best_ms.offset == 16 and gothic.gt_tune_space.reps.offset == 92
    assert ctypes.sizeof(gothic.gt_request) == 120 and gothic.gt_request.nsteps.offset == 112
    assert ctypes.sizeof(gothic.gt_server_stats) == 64


def test_default_params_host_only(libpath):
    from paper_1610_07279_gb300 import gothic
    p = gothic.gt_default_params()
    assert p.mac == gothic.GT_MAC_ACCELERATION and p.delta_acc == 2.0 ** -7
    assert p.leaf_max == 16 and p.group_max == 64 and p.ij_share == 0
    assert p.group_mode == gothic.GT_GROUP_CELLS_TUNED and p.r_crit == 0.0


def test_no_cpu_fallback_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1610_07279_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), fn
