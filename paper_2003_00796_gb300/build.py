"""Build the CUDA library libgbmc.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into paper_2003_00796_gb300/_build/libgbmc.so. Rebuilds only when a source or
header is newer than the library. The checked variant (the same sources with
GBMC_CHECKED defined: index checks in every kernel, see gbmc.h) is linked into
_build/libgbmc_checked.so; build_all() compiles both in one parallel pool.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgbmc.so")
LIB_CHECKED = os.path.join(BUILD, "libgbmc_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "--use_fast_math", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def lib_path(checked: bool = False) -> str:
    return LIB_CHECKED if checked else LIB


def up_to_date(checked: bool = False) -> bool:
    path = lib_path(checked)
    if not os.path.exists(path):
        return False
    t = os.path.getmtime(path)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile_jobs(checked: bool, extra):
    """(source, object, command) of every translation unit of one variant."""
    cc = nvcc()
    odir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(odir, exist_ok=True)
    flags = [*ARCH, *NVCC_FLAGS, *(["-DGBMC_CHECKED"] if checked else []), *extra,
             "-I", os.path.join(ROOT, "include")]
    jobs = []
    for src in sources():
        obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
        jobs.append((src, obj, [cc, *flags, "-c", src, "-o", obj]))
    return jobs


def _link(checked: bool, objs) -> str:
    path = lib_path(checked)
    tmp = path + f".tmp{os.getpid()}"
    # the checked library binds its own symbols first, so that it can be
    # loaded beside libgbmc.so (same exported names) in one process
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart",
           *(["-Xlinker", "-Bsymbolic"] if checked else [])]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, path)
    return path


def build_variants(variants, force: bool = False, verbose: bool = False, extra=None):
    """Compile the given variants (False: libgbmc.so, True: the checked one)
    in one pool; returns their library paths."""
    extra = list(extra or [])
    todo = [v for v in variants if force or not up_to_date(v)]
    if todo:
        os.makedirs(BUILD, exist_ok=True)
        jobs = {v: _compile_jobs(v, extra) for v in todo}

        def compile_one(job):
            src, obj, cmd = job
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            return r.stderr

        flat = [j for v in todo for j in jobs[v]]
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
            errs = list(ex.map(compile_one, flat))
        if verbose:
            for err in errs:
                if err.strip():
                    sys.stderr.write(err)
        for v in todo:
            _link(v, [obj for _, obj, _ in jobs[v]])
    return [lib_path(v) for v in variants]


def build(force: bool = False, verbose: bool = False, extra=None, checked: bool = False) -> str:
    return build_variants([checked], force=force, verbose=verbose, extra=extra)[0]


def build_all(force: bool = False, verbose: bool = False) -> list:
    """libgbmc.so and libgbmc_checked.so."""
    return build_variants([False, True], force=force, verbose=verbose)


if __name__ == "__main__":
    print(build_variants([False, True] if "--all" in sys.argv else ["--checked" in sys.argv],
                         force="--force" in sys.argv, verbose=True,
                         extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None))
