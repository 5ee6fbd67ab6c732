"""Build the CUDA library ``libptg.so`` (sm_103a) in-tree.

The stepper is compiled once per (precision, task kind) pair so the translation units
build in parallel; the objects are linked with the assembly kernels and the C ABI layer
into ``paper_2411_19030_gb300/libptg.so``.  Objects go to ``paper_2411_19030_gb300/_build``.
A rebuild happens only when a source or header is newer than the library.

Variants: ``release`` (the default, ``libptg.so``), ``nvtx`` (``libptg_nvtx.so``, compiled with
``-DPTG_NVTX``: NVTX ranges around every C-ABI call, for a profiler's timeline) and ``debug``
(``libptg_debug.so``, ``-DPTG_DEBUG``: every launch's index ranges checked against the op's
allocations first; a failed check skips the launch and reports PTG_EBOUNDS).  The binding loads
the variant named by the environment variable ``PTG_LIBRARY`` (default ``release``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libptg.so")
VARIANTS = {"release": [], "nvtx": ["-DPTG_NVTX"], "debug": ["-DPTG_DEBUG"]}
# the translation units whose code depends on a variant's macros (trace.h reads PTG_NVTX; the
# launch checks of launch_check.h run in api.cu); a variant compiles these and links them with
# the release objects of the others
VARIANT_SOURCES = {"nvtx": ("api.cu", "design.cu", "noalloc.cu"), "debug": ("api.cu",)}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _units() -> list[tuple[str, list[str], str]]:
    """(source, extra flags, object name) for every translation unit."""
    units = []
    for tag, real in (("f32", "float"), ("f64", "double")):
        for kind in range(6):
            units.append((os.path.join(CSRC, "stepper_inst.cu"),
                          [f"-DPTG_REAL={real}", f"-DPTG_TAG={tag}", f"-DPTG_KIND={kind}"],
                          f"stepper_{tag}_k{kind}.o"))
    for kind in range(6):
        units.append((os.path.join(CSRC, "stream_inst.cu"), [f"-DPTG_KIND={kind}"], f"stream_k{kind}.o"))
    for name in ("plan.cu", "assemble.cu", "coarse.cu", "api.cu", "noalloc.cu", "design.cu", "mesh.cu", "stream.cu",
                 "mg.cu", "mma.cpp"):
        units.append((os.path.join(CSRC, name), [], name.rsplit(".", 1)[0] + ".o"))
    return units


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ptg.h"))
    files.append(os.path.abspath(__file__))
    return files


def library_path(variant: str = "release") -> str:
    """Path of the shared library of a build variant."""
    if variant not in VARIANTS:
        raise ValueError(f"unknown build variant {variant!r}; one of {sorted(VARIANTS)}")
    return LIB if variant == "release" else os.path.join(PKG, f"libptg_{variant}.so")


def _build_dir(variant: str) -> str:
    return BUILD if variant == "release" else os.path.join(BUILD, variant)


def needs_build(variant: str = "release") -> bool:
    lib = library_path(variant)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build_library(force: bool = False, verbose: bool = False, jobs: int | None = None,
                  variant: str = "release") -> str:
    """Compile and link the library of a build variant; returns its path."""
    lib = library_path(variant)
    if not force and not needs_build(variant):
        return lib
    nvcc = _nvcc()
    build_dir = _build_dir(variant)
    os.makedirs(build_dir, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    extra = ["-Xptxas", "-v"] if verbose else []
    defines = VARIANTS[variant]

    def compile_one(u):
        src, flags, obj = u
        out = os.path.join(build_dir, obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *inc, *defines, *flags, *extra, "-c", src, "-o", out]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return out, r.stderr

    units = _units()
    reused = []
    if variant != "release":
        build_library(verbose=verbose, jobs=jobs)          # the release objects of the other units
        own = set(VARIANT_SOURCES[variant])
        reused = [os.path.join(BUILD, obj) for src, _, obj in units if os.path.basename(src) not in own]
        units = [u for u in units if os.path.basename(u[0]) in own]
    jobs = jobs or min(len(units), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, units))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = reused + [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import time
    t0 = time.time()
    var = next((a.split("=", 1)[1] for a in sys.argv if a.startswith("--variant=")), "release")
    path = build_library(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=var)
    print(f"built {path} in {time.time() - t0:.1f} s")
