"""The key quantisation's integer evaluation (Sec. 2.1 keys; csrc/keys_quant.cuh) equals
the FP64 expression it replaces, checked on the host: the header is compiled with g++
(contraction off) next to a driver that compares both on ~5e6 operand sets."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1610_07279_gb300", "csrc")


def test_integer_quantisation_matches_fp64(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "keys_quant_check")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-I", CSRC, os.path.join(HERE, "keys_quant_check.cpp"),
                    "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    line = r.stdout.strip().splitlines()[-1]
    cases, handled, bad = (int(w) for w in line.replace("cases", "").replace("handled", "").replace("mismatches", "").split())
    assert bad == 0 and handled > cases // 2, line
