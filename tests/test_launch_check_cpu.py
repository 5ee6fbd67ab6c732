"""The launch checks of the debug build (csrc/launch_check.h, compiled into libptg_debug.so's
ABI layer): valid launches of every plan kind pass, and each planted fault (slices past N_tau,
history rows outside the window, streamed groups or vectors beyond the workspace, multigrid
levels past a group's workspace, node rows no CTA owns) is caught at its own site.  The header
is plain C++, compiled here with g++ into tests/launch_check_driver.cpp; the debug library
itself is built, loaded and checked for its exports without a GPU."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2411_19030_gb300 import _ffi
from paper_2411_19030_gb300.build import CSRC, build_library, library_path
from tests.test_abi_cpu import declared_functions

HERE = os.path.dirname(os.path.abspath(__file__))

EXPECTED = {
    "ok_fine_primal": 0, "ok_fine_chained": 0, "ok_coarse_adjoint": 0, "ok_adjoint_sweep": 0,
    "ok_adjoint_sweep_plt": 0, "ok_slice_range": 0, "ok_streamed_coarse": 0, "ok_streamed_sweep": 0,
    "slices_past_the_end": 1, "slices_negative_start": 1, "chained_run_of_two_tasks": 1, "sweep_of_two_tasks": 1,
    "coarse_adjoint_without_history": 2, "coarse_adjoint_history_short": 2, "adjoint_sweep_history_offset": 2,
    "streamed_groups_over_workspace": 3, "streamed_sweep_two_groups": 3,
    "streamed_vector_too_short": 4,
    "multigrid_workspace_short": 5, "multigrid_too_many_levels": 5,
    "rows_not_covered": 6, "cluster_of_seventeen": 6,
}


@pytest.fixture(scope="module")
def sites() -> dict:
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "launch_check_driver")
        subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                        os.path.join(HERE, "launch_check_driver.cpp"), "-o", exe], check=True, timeout=120)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60).stdout
    return {name: int(site) for name, site in (line.split() for line in out.splitlines())}


def test_every_case_ran(sites):
    assert set(sites) == set(EXPECTED)


@pytest.mark.parametrize("case", sorted(EXPECTED))
def test_launch_check_site(sites, case):
    assert sites[case] == EXPECTED[case], (case, sites[case])


def test_debug_library_builds_and_loads_without_a_gpu():
    path = build_library(variant="debug")
    assert path == library_path("debug")
    lib = _ffi.load(path)
    assert lib.ptg_version().decode().endswith(" debug")
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.ptg_fe_assemble_operator(None, None, None) == _ffi.PTG_EINVAL
    assert _ffi.ERROR_NAMES[_ffi.PTG_EBOUNDS] == "PTG_EBOUNDS"
