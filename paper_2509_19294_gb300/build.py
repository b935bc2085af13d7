"""Build libnbody.so in-tree with nvcc for sm_103a (no torch extension machinery).

Every ``csrc/*.cu`` is compiled to an object in parallel, then linked with the
static CUDA runtime into ``paper_2509_19294_gb300/libnbody.so``, the force
library.  ``probe/*.cu`` (the benchmark's pipe-rate probes) is linked the same
way into ``libnbody_probe.so``.  A rebuild only happens when a source or header
is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libnbody.so")
PROBE = os.path.join(PKG, "probe")
PROBE_LIB = os.path.join(PKG, "libnbody_probe.so")
OBJ = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fno-fast-math", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnbody.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def probe_sources():
    return sorted(glob.glob(os.path.join(PROBE, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def _probe_deps():
    return _deps() + probe_sources() + glob.glob(os.path.join(PROBE, "*.h"))


def _fresh(lib, deps) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps)


def up_to_date() -> bool:
    return _fresh(LIB, _deps()) and _fresh(PROBE_LIB, _probe_deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Build libnbody.so and libnbody_probe.so (whichever is stale); returns
    the path of libnbody.so."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)

    def compile_one(src, inc=()):
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + list(inc) + list(extra) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    def link(objs, lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {lib} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)

    need_lib = force or not _fresh(LIB, _deps())
    need_probe = force or not _fresh(PROBE_LIB, _probe_deps())
    jobs = ([(src, ()) for src in sources()] if need_lib else []) + (
        [(src, ("-I", PROBE)) for src in probe_sources()] if need_probe else [])
    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(lambda j: compile_one(*j), jobs))
    n_lib = len(sources()) if need_lib else 0
    if need_lib:
        link(objs[:n_lib], LIB)
    if need_probe:
        link(objs[n_lib:], PROBE_LIB)
    return LIB


ABLATION_LIB = os.path.join(PKG, "libnbody_ablate_tile_sums.so")


def build_ablation() -> str:
    """The force library with the cross-tile Kahan compensation switched off
    (NBODY_TILE_SUM_COMPENSATION=0), for the accuracy ablation in bench.py
    only; it is never built by default and nothing else loads it."""
    if _fresh(ABLATION_LIB, _deps()):
        return ABLATION_LIB
    nvcc = _nvcc()
    obj_dir = os.path.join(OBJ, "ablate_tile_sums")
    os.makedirs(obj_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-DNBODY_TILE_SUM_COMPENSATION=0", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = ABLATION_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs,
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {ABLATION_LIB} failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, ABLATION_LIB)
    return ABLATION_LIB


if __name__ == "__main__":
    verbose = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if verbose else []
    print(build(force="-f" in sys.argv or verbose, verbose=verbose, extra=extra))
