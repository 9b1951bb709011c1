"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every function include/hydro.h declares, and rejects bad arguments
before touching the device."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hy():
    from paper_1510_05061_gb300 import build, hydro

    build.build()
    hydro.load()
    return hydro


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hydro.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(hy):
    names = declared_functions()
    assert len(names) >= 10
    lib = C.CDLL(hy.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hy.EXPORTS)


def test_sizes(hy):
    from paper_1510_05061_gb300 import inputs

    prob, _ = inputs.rayleigh_taylor(8, nz=16, perturb=False)
    cp = hy.make_problem(prob)
    assert hy.hydro_state_bytes(cp) == 5 * 8 * 8 * 16 * 8
    cp.precision = 1
    assert hy.hydro_state_bytes(cp) == 5 * 8 * 8 * 16 * 4
    assert hy.hydro_workspace_bytes(cp) % 256 == 0 and hy.hydro_workspace_bytes(cp) > 0
    prob2, _ = inputs.sod(16)
    assert hy.hydro_state_bytes(hy.make_problem(prob2)) == 4 * 16 * 16 * 8


@pytest.mark.parametrize("field,value", [
    ("ndim", 4), ("gamma", 1.0), ("cfl", 0.0), ("precision", 7), ("hse_subtract", 2),
])
def test_invalid_problems_rejected(hy, field, value):
    from paper_1510_05061_gb300 import inputs

    prob, _ = inputs.sod(16)
    cp = hy.make_problem(prob)
    setattr(cp, field, value)
    assert hy.hydro_state_bytes(cp) == 0
    assert hy.hydro_workspace_bytes(cp) == 0


def test_invalid_shapes_rejected(hy):
    from paper_1510_05061_gb300 import inputs

    prob, _ = inputs.sod(16)
    cp = hy.make_problem(prob)
    cp.n[1] = 1                      # an active axis needs >= 2 cells
    assert hy.hydro_state_bytes(cp) == 0
    cp = hy.make_problem(prob)
    cp.bc_lo[0] = 1                  # periodic on one side only
    assert hy.hydro_state_bytes(cp) == 0
    cp = hy.make_problem(prob)
    cp.hse_subtract = 1              # hse needs 3D
    assert hy.hydro_state_bytes(cp) == 0


def test_plane_size_limit(hy):
    """A z plane (nx * ny) is indexed with 32-bit offsets: 2^31 - 1 cells
    is the largest accepted plane, and the byte counts of such a grid are
    computed in 64 bits."""
    from paper_1510_05061_gb300 import inputs

    prob, _ = inputs.rayleigh_taylor(8, nz=4, perturb=False)
    cp = hy.make_problem(prob)
    cp.hse_subtract = 0
    cp.n[0], cp.n[1], cp.n[2] = 65536, 32768, 2           # plane = 2^31
    assert hy.hydro_state_bytes(cp) == 0
    cp.n[0], cp.n[1], cp.n[2] = 46341, 46340, 2           # plane = 2147441940 < 2^31
    assert hy.hydro_state_bytes(cp) == 5 * 46341 * 46340 * 2 * 8
    cp.precision = 1
    assert hy.hydro_state_bytes(cp) == 5 * 46341 * 46340 * 2 * 4
    assert hy.hydro_workspace_bytes(cp) > 0


def test_init_argument_errors_before_device(hy):
    from paper_1510_05061_gb300 import inputs

    prob, W = inputs.sod(16)
    cp = hy.make_problem(prob)
    L = hy.load()
    h = C.c_void_p()
    W = np.ascontiguousarray(W)
    Wp = W.ctypes.data_as(C.POINTER(C.c_double))
    # null buffers, misaligned buffers, same buffer twice, null handle slot
    assert L.hydro_init(C.byref(cp), None, None, None, Wp, None, None, C.byref(h)) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_init(C.byref(cp), C.c_void_p(256), C.c_void_p(1024 + 8), C.c_void_p(4096), Wp, None,
                        None, C.byref(h)) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_init(C.byref(cp), C.c_void_p(256), C.c_void_p(256), C.c_void_p(4096), Wp, None,
                        None, C.byref(h)) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_init(C.byref(cp), C.c_void_p(256), C.c_void_p(512), C.c_void_p(4096), Wp, None,
                        None, None) == hy.HYDRO_ERR_INVALID_ARG
    # hse without tables
    p3, W3 = inputs.rayleigh_taylor(8, nz=16, hse_subtract=1)
    c3 = hy.make_problem(p3)
    W3 = np.ascontiguousarray(W3)
    assert L.hydro_init(C.byref(c3), C.c_void_p(256), C.c_void_p(512), C.c_void_p(4096),
                        W3.ctypes.data_as(C.POINTER(C.c_double)), None, None,
                        C.byref(h)) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_step(None, None) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_destroy(None) == hy.HYDRO_ERR_INVALID_ARG
    assert L.hydro_strerror(hy.HYDRO_ERR_NONPHYSICAL).startswith(b"non-physical")


def test_background_table_order(hy):
    from paper_1510_05061_gb300 import inputs

    prob, _ = inputs.rayleigh_taylor(8, nz=16, hse_subtract=1)
    t = hy.background_tables(prob)
    assert t.size == 2 * 20 + 2 * 21
    np.testing.assert_array_equal(t[:20], prob.bg_rho_c)
    np.testing.assert_array_equal(t[40:61], prob.bg_rho_f)


def test_per_device_setup_runs_once_per_device(hy):
    """The launchers' attribute/occupancy set-up is kept per device ordinal:
    one process driving several devices configures each of them once, a
    failed set-up is retried, and concurrent host threads do not repeat it."""
    devs = [0, 1, 0, 1, 1, 0, 2, 3, 2, 0]
    once, vcalls, vals = hy.hydro_selftest_device_once(devs, ndev=4)
    assert once.tolist() == [1, 1, 1, 1]
    assert vcalls.tolist() == [1, 1, 1, 1]
    assert vals.tolist() == [100, 101, 102, 103]
    # a device never seen is never configured
    once, vcalls, vals = hy.hydro_selftest_device_once([0, 2, 2], ndev=4)
    assert once.tolist() == [1, 0, 1, 0] and vals.tolist() == [100, 0, 102, 0]
    # device 1's first set-up fails: its next use retries it, the others are unaffected
    once, vcalls, vals = hy.hydro_selftest_device_once(devs, fail_dev=1, ndev=4)
    assert once.tolist() == [1, 2, 1, 1] and vcalls.tolist() == [1, 2, 1, 1]
    assert vals.tolist() == [100, 101, 102, 103]
    # eight host threads walking the same devices at once
    for _ in range(20):
        once, vcalls, vals = hy.hydro_selftest_device_once(devs * 10, threads=8, ndev=4)
        assert once.tolist() == [1, 1, 1, 1] and vcalls.tolist() == [1, 1, 1, 1]
        assert vals.tolist() == [100, 101, 102, 103]
    with pytest.raises(hy.HydroError):
        hy.hydro_selftest_device_once([5], ndev=4)


def test_conserved_init_argument_checks(hy):
    from paper_1510_05061_gb300 import inputs

    prob, W = inputs.sod(16)
    cp = hy.make_problem(prob)
    h = C.c_void_p()
    # a missing initial state and a null output are refused before any CUDA call
    assert hy.load().hydro_init_conserved(C.byref(cp), C.c_void_p(256), C.c_void_p(512),
                                          C.c_void_p(1024), None, None, None,
                                          C.byref(h)) == hy.HYDRO_ERR_INVALID_ARG
    assert hy.load().hydro_init_conserved(C.byref(cp), C.c_void_p(256), C.c_void_p(512),
                                          C.c_void_p(1024), W.ctypes.data_as(C.POINTER(C.c_double)),
                                          None, None, None) == hy.HYDRO_ERR_INVALID_ARG
