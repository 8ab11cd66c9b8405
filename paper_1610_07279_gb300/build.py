"""Build libgothic.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each translation unit is compiled with nvcc in parallel, then linked into
``paper_1610_07279_gb300/_lib/libgothic.so`` against the shared CUDA runtime (the
same libcudart.so.13 PyTorch loads, so streams and device pointers are shared).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libgothic.so")
# The debug variant (index checks in the walk and the pseudo j-particle pass that latch
# GT_EINVAL instead of reading outside the tree; -DGT_DEBUG=1) lives in its own directory.
VARIANTS = {"": (OUT_DIR, []), "debug": (os.path.join(OUT_DIR, "debug"), ["-DGT_DEBUG=1"])}


def lib_of(variant: str = "") -> str:
    return os.path.join(VARIANTS[variant][0], "libgothic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgothic")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


# Extra nvcc flags for tuning builds (compile-time knobs such as -DGT_WALK_MINB=4); the
# library is rebuilt whenever they change.
FLAGS_STAMP = os.path.join(OUT_DIR, "flags.txt")


def _extra_flags(variant: str = "") -> list[str]:
    return VARIANTS[variant][1] + os.environ.get("GOTHIC_NVCC_FLAGS", "").split()


def up_to_date(variant: str = "") -> bool:
    lib = lib_of(variant)
    if not os.path.exists(lib):
        return False
    try:
        if open(os.path.join(VARIANTS[variant][0], "flags.txt")).read() != " ".join(_extra_flags(variant)):
            return False
    except OSError:
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, variant: str = "") -> str:
    """Compile every .cu under csrc/ and link libgothic.so (of the variant); returns its path."""
    if not force and up_to_date(variant):
        return lib_of(variant)
    nvcc = _nvcc()
    out_dir = VARIANTS[variant][0]
    LIB = lib_of(variant)
    os.makedirs(out_dir, exist_ok=True)
    obj_dir = os.path.join(out_dir, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "-Xcompiler", "-fvisibility=hidden"] + _extra_flags(variant)
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src: str):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, sources()))
    if verbose or ptxas_verbose:
        for obj, log in results:
            if log.strip():
                print(f"--- {os.path.basename(obj)}\n{log}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + [
        "-cudart", "shared", "-Xlinker", "-rpath," + _cuda_lib_dir(nvcc)]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(os.path.join(out_dir, "flags.txt"), "w") as f:
        f.write(" ".join(_extra_flags(variant)))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv,
                variant="debug" if "--debug" in sys.argv else ""))
