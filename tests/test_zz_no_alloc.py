"""hydro_totals_noalloc: conserved totals for callers that must not allocate
device memory (their host application's memory manager owns the device, or
their loop cannot take the synchronisation an allocation may cause).  It must
return the same sums as the workspace-based hydro_reduce(HYDRO_RED_TOTALS),
on repeated calls, with its scratch in the library's static device array.

This file is named so that pytest collects it after every other test file.
"""

import ctypes as C

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hy():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05061_gb300 import build, hydro

    build.build()
    hydro.load()
    return hydro


CASES = [
    ("rt_fp64", lambda: inputs.rayleigh_taylor(24, nz=40, amplitude=0.05)),
    ("rt_fp64_hse", lambda: inputs.rayleigh_taylor(24, nz=40, amplitude=0.05, hse_subtract=1)),
    ("rt_fp32_hse", lambda: inputs.rayleigh_taylor(24, nz=40, amplitude=0.05, hse_subtract=1,
                                                   precision=inputs.FP32)),
    ("kh2d_fp64", lambda: inputs.kelvin_helmholtz(200, ndim=2, precision=inputs.FP64)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_totals_match_workspace_totals(hy, name, make):
    import torch

    prob, W = make()
    sim = hy.Simulation(prob, W)
    sim.run_steps(4)
    ref = sim.totals()                       # existing entry point, caller workspace
    cp = hy.make_problem(prob)
    bg = hy.background_tables(prob)
    stream = torch.cuda.current_stream().cuda_stream
    scale = np.abs(ref).max()
    for _ in range(2):                       # two calls in a row share the scratch
        got = hy.hydro_totals_noalloc(cp, sim.current_ptr(), bg, stream, prob.nvar)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * scale)
    # after the state moves on, the static scratch gives the new totals
    sim.run_steps(2)
    ref2 = sim.totals()
    got2 = hy.hydro_totals_noalloc(cp, sim.current_ptr(), bg, stream, prob.nvar)
    np.testing.assert_allclose(got2, ref2, rtol=1e-12, atol=1e-12 * scale)
    sim.close()


def test_noalloc_rejects_oversized_background(hy):
    import torch

    prob, _ = inputs.rayleigh_taylor(4, nz=5000, perturb=False, hse_subtract=1)
    cp = hy.make_problem(prob)
    bg = hy.background_tables(prob)
    # a real device buffer of the problem's state size: should the size check
    # ever regress, the call still reads only memory it was given
    nbytes = hy.load().hydro_state_bytes(C.byref(cp))
    assert nbytes > 0
    U = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out = np.zeros(5)
    rc = hy.load().hydro_totals_noalloc(C.byref(cp), C.c_void_p(U.data_ptr()),
                                        bg.ctypes.data_as(C.POINTER(C.c_double)), None,
                                        out.ctypes.data_as(C.POINTER(C.c_double)))
    torch.cuda.synchronize()
    assert rc == hy.HYDRO_ERR_INVALID_ARG
