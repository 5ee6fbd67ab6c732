"""CPU-side checks of the C ABI: the library builds, loads without a GPU and exports every
function that include/ptg.h declares; argument errors are caught before any launch."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2411_19030_gb300 import _ffi
from paper_2411_19030_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> list[str]:
    src = open(os.path.join(ROOT, "include", "ptg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _ffi.load()


def test_header_declares_the_paths_entry_points():
    names = declared_functions()
    for required in ("ptg_fe_assemble_operator", "ptg_fine_propagate_slices", "ptg_coarse_sweep",
                     "ptg_parareal_correct", "ptg_adjoint_sweep", "ptg_sensitivities"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _ffi.SIGNATURES, f"{name} has no ctypes signature"


def test_version_string(lib):
    assert lib.ptg_version().decode().startswith("ptg ")


def _args(nx=4, ny=4, Nt=4, Ntau=2, p=8.0, prec=0):
    g = _ffi.ptg_grid(nx, ny, 1.0 / nx)
    m = _ffi.ptg_material(1.0, 1e-3, 3.0, 1.0, 1.0, 1.0)
    t = _ffi.ptg_time(Nt, Ntau, 0.1, p)
    s = _ffi.ptg_solve(prec, 1e-13, 0.0, 100, 4)
    d = np.zeros((nx + 1) * (ny + 1), np.uint8)
    return g, m, t, s, d


@pytest.mark.parametrize("bad", ["ntau", "p_odd", "p_frac", "nx", "precision", "objective", "guess_high",
                                 "guess_negative", "local_steps", "coarse_stream"])
def test_invalid_problem_rejected_on_host(lib, bad):
    g, m, t, s, d = _args()
    if bad == "ntau":
        t.Ntau = 3
    elif bad == "p_odd":
        t.p = 7.0
    elif bad == "p_frac":
        t.p = 8.5
    elif bad == "nx":
        g.nx = 1
    elif bad == "precision":
        s.precision = 7
    elif bad == "objective":
        t.objective = 2
    elif bad == "guess_high":
        s.initial_guess = 5
    elif bad == "guess_negative":
        s.initial_guess = -1
    elif bad == "local_steps":
        s.local_steps = 4
    elif bad == "coarse_stream":
        s.coarse_stream = 3
    h = ctypes.c_void_p()
    rc = lib.ptg_op_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(t), ctypes.byref(s), d.ctypes.data,
                           None, None, 0, ctypes.byref(h))
    assert rc == _ffi.PTG_EINVAL and not h.value


def test_null_op_rejected(lib):
    assert lib.ptg_fe_assemble_operator(None, None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_fine_propagate_slices(None, 0, 0, 1, None, None, None, 0, 0, None, None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_get_stats(None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_objective_from_modified(None, None, None, None, None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_parareal_correct(None, 1, None, None, None, None, None, None, None, None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_batch_oneshot_pass(None, 0, None) == _ffi.PTG_EINVAL


@pytest.mark.parametrize("field", ["k0", "kmin", "c0", "cmin"])
def test_noalloc_rejects_non_positive_materials_on_host(lib, field):
    """The entry point without allocation applies ptg_op_create's material rule before it touches
    the device (the pointers here are never dereferenced)."""
    m = _ffi.ptg_material(1.0, 1e-3, 3.0, 1.0, 0.5, 2.0)
    setattr(m, field, 0.0)
    fake = ctypes.c_void_p(16)
    rc = lib.ptg_sensitivities_noalloc(4, 4, 0.25, 4, 0.1, ctypes.byref(m), fake, fake, 1, 4, fake, 0, 5, fake, None)
    assert rc == _ffi.PTG_EINVAL
    assert b"positive" in lib.ptg_last_error()


def test_binding_constants_match_the_header():
    """Every integer constant of include/ptg.h has the same value in the ctypes binding, and every
    error code has a name there (the header's PTG_NOALLOC_SCRATCH_DOUBLES is a size, not a code)."""
    src = open(os.path.join(ROOT, "include", "ptg.h")).read()
    defs = dict(re.findall(r"^#define (PTG_[A-Z0-9_]+)\s+(-?\d+)\b", src, flags=re.M))
    assert len(defs) >= 20
    for name, value in defs.items():
        assert getattr(_ffi, name) == int(value), name
        if name.startswith("PTG_E") or name == "PTG_OK":
            assert _ffi.ERROR_NAMES[int(value)] == name


def test_ctypes_structures_match_the_header_layout(tmp_path):
    """The ctypes mirrors of the header's structures have the C layout: for every field of every
    mirror, the offset that g++ gives it through include/ptg.h, and the size of the whole struct
    (a field missing on either side changes one of them or fails the compile)."""
    import shutil
    import subprocess

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    structs = [_ffi.ptg_grid, _ffi.ptg_material, _ffi.ptg_time, _ffi.ptg_solve, _ffi.ptg_stats,
               _ffi.ptg_pass_buffers]
    lines = ['#include <cstdio>', '#include <cstddef>', '#include "ptg.h"', "int main() {"]
    for st in structs:
        lines.append(f'  std::printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for f in st._fields_:
            lines.append(f'  std::printf("{st.__name__} {f[0]} %zu\\n", offsetof({st.__name__}, {f[0]}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.cpp"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("no CUDA headers for ptg.h")
    subprocess.run([gxx, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for f in st._fields_:
            assert got[(st.__name__, f[0])] == getattr(st, f[0]).offset, (st.__name__, f[0])


def test_product_path_fails_loudly_without_its_library_or_a_gpu(tmp_path):
    """There is no CPU fallback: a missing library raises OSError on load, and an operator cannot
    be made without a CUDA device (this test runs where torch sees none)."""
    import torch

    with pytest.raises(OSError, match="missing"):
        _ffi.load(str(tmp_path / "libptg.so"))
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2411_19030_gb300 import Operator
    with pytest.raises(Exception):
        Operator(4, 4, 0.25, dict(k0=1.0, kmin=1e-3, pk=3.0, c0=1.0, cmin=1.0, pc=1.0), 4, 2, 0.1, 8.0,
                 np.zeros(25, np.uint8))
