"""Build ``libvi.so`` (the CUDA library behind ``include/vi.h``) in place, and
its checked variant ``libvi_checked.so``.

Each translation unit is compiled by nvcc for sm_103a in parallel, then linked
into one shared library next to this file.  The checked variant is the same
sources compiled with ``-DVI_DEBUG_BOUNDS=1``: every kernel tests its memory
indices before each access and counts violations (``vi_debug_bounds``).  Usage:
``python -m paper_2008_06134_gb300.build [--force] [--verbose] [--release-only]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["vi_api.cu", "vi_sweep.cu", "vi_march.cu", "vi_grid.cu", "vi_server.cu", "vi_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# variant -> (library, object folder, extra defines)
VARIANTS = {
    "release": (os.path.join(HERE, "libvi.so"), os.path.join(HERE, "_build"), []),
    "checked": (os.path.join(HERE, "libvi_checked.so"), os.path.join(HERE, "_build_checked"),
                ["-DVI_DEBUG_BOUNDS=1"]),
}
LIB = VARIANTS["release"][0]
LIB_CHECKED = VARIANTS["checked"][0]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvi.so")


def _flags(verbose: bool, defines):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                "-I", os.path.join(HERE, "..", "include")] + list(defines)
    # Optional tuning defines, e.g. VI_NVCC_DEFINES="-DVI_BRICK_SHIFT=2".
    f += os.environ.get("VI_NVCC_DEFINES", "").split()
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(HERE, "..", "include", "vi.h"), os.path.abspath(__file__)]


def up_to_date(variant: str = "release") -> bool:
    lib = VARIANTS[variant][0]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Build the release library (and, with ``checked``, the checked one) if a
    source is newer; all translation units compile in one parallel pool.
    Returns the release library's path."""
    variants = [v for v in (("release", "checked") if checked else ("release",))
                if force or not up_to_date(v)]
    if not variants:
        return LIB
    cc = nvcc()
    jobs = []
    for v in variants:
        _, obj_dir, defines = VARIANTS[v]
        os.makedirs(obj_dir, exist_ok=True)
        jobs += [(v, src, _flags(verbose, defines)) for src in SOURCES]

    def compile_one(job):
        v, src, flags = job
        obj = os.path.join(VARIANTS[v][1], os.path.splitext(src)[0] + ".o")
        cmd = [cc, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} ({v}):\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return v, obj

    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for v in variants:
        lib = VARIANTS[v][0]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for w, o in objs if w == v], "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed ({v}):\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                checked="--release-only" not in sys.argv))
