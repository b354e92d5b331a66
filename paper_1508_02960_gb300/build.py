"""Build the CUDA library ``_build/liblbm_gb300.so`` for sm_103a.

Every ``csrc/*.cu`` is compiled to an object in parallel (one ``-gencode`` target,
``-lineinfo``) and linked with nvcc into a shared library that exports only the
``lbm_*`` C ABI of ``include/lbm_gb300.h``.  Objects are rebuilt when their source or
any header is newer.

Variants build the same sources with extra preprocessor definitions into
``_build_<variant>/``: ``checked`` (``LBM_CHECKED=1``) bounds-checks every index the
step kernels use and reports a violation instead of making the access.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblbm_gb300.so")
VARIANTS = {"": [], "checked": ["-DLBM_CHECKED=1"]}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-fvisibility=hidden,-O2", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_dir(variant: str = "") -> str:
    return BUILD if not variant else BUILD + "_" + variant


def lib_path(variant: str = "") -> str:
    return os.path.join(build_dir(variant), "liblbm_gb300.so")


def _compile(src: str, obj: str, verbose: bool, defines=()) -> str:
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(defines) + ["-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, variant: str = "",
          defines=None) -> str:
    """Compile and link the library (or one of its variants) if needed; return its path.
    defines: the variant's -D flags (default: those of VARIANTS[variant])."""
    if defines is None:
        defines = VARIANTS[variant]
    out = build_dir(variant)
    lib = lib_path(variant)
    os.makedirs(out, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(out, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            todo.append((s, o))
    if todo:
        jobs = jobs or min(len(todo), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = {ex.submit(_compile, s, o, verbose, defines): s for s, o in todo}
            for f in cf.as_completed(futs):
                log = f.result()
                if verbose and log:
                    sys.stderr.write(log)
    if force or todo or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
