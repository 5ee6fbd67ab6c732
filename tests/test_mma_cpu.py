"""The host MMA of the library (ptg_mma_*, C++) against the oracle's MMA: the same iterates on
a separable convex problem and on a problem whose constraint switches between active and
inactive; argument checks of the design entry points.  CPU only (the MMA runs on the host)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from oracle.design import MMA
from paper_2411_19030_gb300 import _ffi
from paper_2411_19030_gb300.build import build_library


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _ffi.load()


def host_mma(lib, n, lo, hi, move):
    h = ctypes.c_void_p()
    assert lib.ptg_mma_create(n, lo, hi, move, ctypes.byref(h)) == 0
    return h


def step(lib, h, x, f0, df0, f1, df1):
    x, df0, df1 = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, df0, df1))
    out = np.empty_like(x)
    assert lib.ptg_mma_update(h, x.ctypes.data, f0, df0.ctypes.data, f1, df1.ctypes.data, out.ctypes.data) == 0
    return out


def test_host_mma_follows_the_oracle_on_a_separable_problem(lib):
    rng = np.random.default_rng(7)
    n, V = 300, 0.4
    c = rng.uniform(0.1, 3.0, n)
    ref, h = MMA(n, 0.0, 1.0, 0.2), host_mma(lib, n, 0.0, 1.0, 0.2)
    x_ref = x_lib = np.full(n, V)
    for _ in range(30):
        x_ref = ref.update(x_ref, float(np.sum(c / (x_ref + 0.05))), -c / (x_ref + 0.05) ** 2, float(x_ref.mean() - V),
                           np.full(n, 1.0 / n))
        x_lib = step(lib, h, x_lib, float(np.sum(c / (x_lib + 0.05))), -c / (x_lib + 0.05) ** 2,
                     float(x_lib.mean() - V), np.full(n, 1.0 / n))
        assert np.max(np.abs(x_lib - x_ref)) < 1e-12
    lib.ptg_mma_destroy(h)


def test_host_mma_follows_the_oracle_with_a_switching_constraint(lib):
    """Objective pulls towards t, the constraint sum(x)/n <= V binds only in some steps."""
    rng = np.random.default_rng(8)
    n, V = 120, 0.5
    t = rng.uniform(-0.3, 1.3, n)
    ref, h = MMA(n, 0.0, 1.0, 0.1), host_mma(lib, n, 0.0, 1.0, 0.1)
    x_ref = x_lib = rng.uniform(0.2, 0.8, n)
    for k in range(40):
        w = 1.0 + 0.5 * np.sin(0.3 * k)          # the target moves, so the multiplier changes
        x_ref = ref.update(x_ref, float(w * np.sum((x_ref - t) ** 2)), 2 * w * (x_ref - t), float(x_ref.mean() - V),
                           np.full(n, 1.0 / n))
        x_lib = step(lib, h, x_lib, float(w * np.sum((x_lib - t) ** 2)), 2 * w * (x_lib - t),
                     float(x_lib.mean() - V), np.full(n, 1.0 / n))
        assert np.max(np.abs(x_lib - x_ref)) < 1e-11, k
    lib.ptg_mma_destroy(h)


def test_design_and_mma_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.ptg_mma_create(0, 0.0, 1.0, 0.2, ctypes.byref(h)) == _ffi.PTG_EINVAL
    assert lib.ptg_mma_create(10, 1.0, 0.0, 0.2, ctypes.byref(h)) == _ffi.PTG_EINVAL
    assert lib.ptg_mma_update(None, None, 0.0, None, 0.0, None, None) == _ffi.PTG_EINVAL
    assert lib.ptg_design_create(8, 8, 0.1, -1.0, 8.0, 0.5, 0, ctypes.byref(h)) == _ffi.PTG_EINVAL
    assert lib.ptg_design_create(8, 8, 0.1, 0.2, 8.0, 1.5, 0, ctypes.byref(h)) == _ffi.PTG_EINVAL
    assert lib.ptg_design_forward(None, None, None, None, None) == _ffi.PTG_EINVAL


def test_mma_state_saved_to_a_file_resumes_bit_for_bit(lib, tmp_path):
    """The optimiser half of the design loop's save / resume: the MMA state (update count, last
    two iterates, asymptotes) written with np.savez, as the loop's save() does, and restored into
    a fresh optimiser continues with the same iterates as the optimiser that never stopped."""
    from paper_2411_19030_gb300.design import MMAUpdate

    rng = np.random.default_rng(9)
    n, V = 200, 0.45
    t = rng.uniform(-0.2, 1.2, n)

    def grads(x, k):
        w = 1.0 + 0.5 * np.sin(0.4 * k)
        return float(w * np.sum((x - t) ** 2)), 2 * w * (x - t), float(x.mean() - V), np.full(n, 1.0 / n)

    a = MMAUpdate(n, 0.0, 1.0, 0.15)
    x = rng.uniform(0.2, 0.8, n)
    for k in range(7):
        x = a.update(x, *grads(x, k))
    path = tmp_path / "state.npz"
    np.savez(path, x=x, **{"mma_" + key: v for key, v in a.get_state().items()})
    d = np.load(path)
    b = MMAUpdate(n, 0.0, 1.0, 0.15)
    b.set_state({key: d["mma_" + key] for key in ("k", "x1", "x2", "L", "U")})
    xa, xb = x, d["x"].copy()
    for k in range(7, 15):
        xa = a.update(xa, *grads(xa, k))
        xb = b.update(xb, *grads(xb, k))
        assert np.array_equal(xa, xb), k
    with pytest.raises(ValueError):
        MMAUpdate(n + 1, 0.0, 1.0, 0.15).set_state(a.get_state())
