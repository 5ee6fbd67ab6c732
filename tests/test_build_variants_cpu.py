"""The build variant with NVTX ranges around the C-ABI calls (``build_library(variant="nvtx")``,
libptg_nvtx.so): it compiles for sm_103a, loads without a GPU, exports every function that
include/ptg.h declares, names itself in the version string, and its traced entry points run
their host-side checks with the NVTX calls live (no profiler attached, so they return at once).
The binding opens it when PTG_LIBRARY is "nvtx"."""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2411_19030_gb300 import _ffi
from paper_2411_19030_gb300.build import build_library, library_path
from tests.test_abi_cpu import declared_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nvtx_lib():
    path = build_library(variant="nvtx")
    assert path == library_path("nvtx") and path != library_path("release")
    return _ffi.load(path)


def test_nvtx_variant_exports_every_declared_symbol(nvtx_lib):
    for name in declared_functions():
        assert hasattr(nvtx_lib, name), name


def test_version_names_the_variant(nvtx_lib):
    assert nvtx_lib.ptg_version().decode().endswith(" nvtx")
    release = _ffi.load(library_path("release"))
    assert not release.ptg_version().decode().endswith(" nvtx")


def test_traced_entry_points_keep_their_host_checks(nvtx_lib):
    g = _ffi.ptg_grid(4, 4, 0.25)
    m = _ffi.ptg_material(1.0, 1e-3, 3.0, 1.0, 1.0, 1.0)
    t = _ffi.ptg_time(4, 3, 0.1, 8.0)                       # Ntau does not divide Nt
    s = _ffi.ptg_solve(0, 1e-13, 0.0, 100, 4)
    d = np.zeros(25, np.uint8)
    h = ctypes.c_void_p()
    rc = nvtx_lib.ptg_op_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(t), ctypes.byref(s),
                                d.ctypes.data, None, None, 0, ctypes.byref(h))
    assert rc == _ffi.PTG_EINVAL and not h.value
    assert nvtx_lib.ptg_fe_assemble_operator(None, None, None) == _ffi.PTG_EINVAL
    assert nvtx_lib.ptg_batch_oneshot_pass(None, 0, None) == _ffi.PTG_EINVAL
    assert nvtx_lib.ptg_design_forward(None, None, None, None, None) == _ffi.PTG_EINVAL


def test_binding_opens_the_variant_named_by_the_environment(nvtx_lib):
    code = ("from paper_2411_19030_gb300 import _ffi; import sys; "
            "sys.stdout.write(_ffi.default_library() + '|' + _ffi.load().ptg_version().decode())")
    env = dict(os.environ, PTG_LIBRARY="nvtx")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    path, version = out.stdout.split("|")
    assert path == library_path("nvtx") and version.endswith(" nvtx")


def test_unknown_variant_is_rejected():
    with pytest.raises(ValueError):
        library_path("profiling")
