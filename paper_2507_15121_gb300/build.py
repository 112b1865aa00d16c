"""Build the GB300 sparse MTTKRP library (libamped.so) in place.

Compiles every CUDA translation unit for sm_103a with nvcc (in parallel) and
links them with the host reorder into ``paper_2507_15121_gb300/libamped.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libamped.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp", "-I" + os.path.join(HERE, "..", "include")]
# extra nvcc flags (e.g. -D definitions of the kernels' compile-time constants); part of the
# object files' staleness key so a change rebuilds
EXTRA = os.environ.get("AMPED_NVCC_FLAGS", "").split()


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _flags_file(build_dir, flags):
    """A file whose content is the extra flags; rewritten only when they change."""
    path = os.path.join(build_dir, "extra_flags.txt")
    text = " ".join(flags)
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def _compile(src, build_dir, flags, verbose=False):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if not _stale(obj, [src, os.path.join(build_dir, "extra_flags.txt")] + _headers()):
        return obj
    cmd = [NVCC] + ARCH + COMMON + flags + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, flags: list | None = None,
          lib_path: str | None = None, build_dir: str | None = None) -> str:
    """Compile and link the library.  `flags` (default: AMPED_NVCC_FLAGS) are
    extra nvcc flags, e.g. ["-DAMPED_CHECKS=1"] for the bounds-checked build;
    `lib_path` / `build_dir` place a variant build outside the package."""
    flags = EXTRA if flags is None else list(flags)
    lib = lib_path or LIB
    bdir = build_dir or BUILD
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    if force:
        for f in glob.glob(os.path.join(bdir, "*.o")):
            os.remove(f)
    _flags_file(bdir, flags)
    with cf.ThreadPoolExecutor(max_workers=jobs or min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(lambda s: _compile(s, bdir, flags, verbose), srcs))
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
