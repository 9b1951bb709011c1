"""Parity of the PPM reconstruction on the GPU (SSP-RK2 stages with
piecewise parabolic face states, 2D and 3D) with the FP64 CPU oracle's PPM
mode, through the C ABI.  Same bar as the other paths: L1-relative 1e-10 per
conserved variable in FP64."""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, PPM, SSPRK2, Problem

from test_gpu_parity import assert_parity, l1rel, smooth_random

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


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def ppm(prob):
    return prob.replace(scheme=SSPRK2, recon=PPM)


def gpu(hy, prob, W, steps=None, t_end=None, variant=None, zchunk=0):
    sim = hy.Simulation(prob, W)
    if variant is not None:
        sim.configure(variant, zchunk)
    if t_end is not None:
        n, t = sim.advance_to(t_end)
    else:
        sim.run_steps(steps)
        n = steps
    return dict(U=sim.conserved(), t=sim.t, n=n, sim=sim)


def ref(orc, prob, W, steps=None, t_end=None):
    o = orc.Oracle(prob)
    kw = dict(max_steps=steps) if t_end is None else dict(t_end=t_end)
    V, t, s, dl = o.run(o.state_from_prim(W), **kw)
    return dict(U=o.total(V), t=t, n=s)


def test_ppm_sod(hy, orc):
    prob, W = inputs.sod(128)
    prob = ppm(prob)
    g = gpu(hy, prob, W, t_end=0.2)
    o = ref(orc, prob, W, t_end=0.2)
    assert g["t"] == 0.2 and g["n"] == o["n"]
    assert_parity(g["U"], o["U"], label="sod ppm")
    P = g["sim"].primitive()
    assert (P[0] == P[0, :, :1, :]).all() and np.abs(P[2]).max() == 0.0


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, 0), (BC_REFLECT, BC_PERIODIC, 0), (0.0, -0.5, 0.0)),
    ((BC_REFLECT, BC_OUTFLOW, 0), (BC_OUTFLOW, BC_REFLECT, 0), (0.3, 0.2, 0.0)),
])
def test_ppm_2d_ragged(hy, orc, bcl, bch, g):
    prob = ppm(Problem(ndim=2, n=(131, 67, 1), hi=(1.3, 0.7, 1.0), bc_lo=bcl, bc_hi=bch, grav=g))
    W = smooth_random(prob, 17)
    gr = gpu(hy, prob, W, steps=25)
    o = ref(orc, prob, W, steps=25)
    assert_parity(gr["U"], o["U"], label=f"ppm 2d {bcl} {bch}")


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), (BC_REFLECT, BC_PERIODIC, BC_REFLECT), (0.0, 0.0, -1.0)),
    ((BC_PERIODIC, BC_REFLECT, BC_OUTFLOW), (BC_PERIODIC, BC_OUTFLOW, BC_OUTFLOW), (0.2, -0.3, 0.5)),
])
def test_ppm_3d_ragged(hy, orc, bcl, bch, g):
    prob = ppm(Problem(ndim=3, n=(37, 29, 23), hi=(1.0, 0.8, 0.6), bc_lo=bcl, bc_hi=bch, grav=g))
    W = smooth_random(prob, 23)
    gr = gpu(hy, prob, W, steps=12)
    o = ref(orc, prob, W, steps=12)
    assert_parity(gr["U"], o["U"], label=f"ppm 3d {bcl} {bch}")


@pytest.mark.parametrize("shape", [(3, 3, 3), (5, 4, 7), (33, 3, 9)])
def test_ppm_smallest_grids(hy, orc, shape):
    prob = ppm(Problem(ndim=3, n=shape, bc_lo=(BC_REFLECT, BC_PERIODIC, BC_OUTFLOW),
                       bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.1, -0.4)))
    W = smooth_random(prob, 5, jump=False)
    gr = gpu(hy, prob, W, steps=5)
    o = ref(orc, prob, W, steps=5)
    assert_parity(gr["U"], o["U"], label=str(shape))


def test_ppm_rayleigh_taylor_and_fp32(hy, orc):
    prob, W = inputs.rayleigh_taylor(24, nz=32, amplitude=0.05)
    prob = ppm(prob)
    gr = gpu(hy, prob, W, steps=15)
    o = ref(orc, prob, W, steps=15)
    assert_parity(gr["U"], o["U"], label="ppm rt")
    g32 = gpu(hy, prob.replace(precision=inputs.FP32), W, steps=15)
    assert l1rel(g32["U"][0], o["U"][0]) <= 1e-5


@pytest.mark.parametrize("variant,zchunk", [(1, 3), (2, 0), (0, 32)])
def test_ppm_tile_and_chunk_invariance(hy, variant, zchunk):
    prob, W = inputs.kelvin_helmholtz(35, ndim=3, U=1.2, ratio=2.0, precision=inputs.FP64)
    prob = ppm(prob)
    base = gpu(hy, prob, W, steps=4)["sim"].get_state()
    other = gpu(hy, prob, W, steps=4, variant=variant, zchunk=zchunk)["sim"].get_state()
    assert np.array_equal(base, other)


@pytest.mark.parametrize("variant,zchunk", [(0, 0), (3, 7), (2, 40)])
def test_ppm_fp32_tile_and_chunk_invariance(hy, variant, zchunk):
    """FP32 PPM stages: the 32 x 16 tile (spare ring slot) and the 32 x 8 and
    16 x 16 tiles (no spare slot) give the same bits."""
    prob, W = inputs.kelvin_helmholtz(35, ndim=3, U=1.2, ratio=2.0, precision=inputs.FP32)
    prob = ppm(prob)
    base = gpu(hy, prob, W, steps=4)["sim"].get_state()
    other = gpu(hy, prob, W, steps=4, variant=variant, zchunk=zchunk)["sim"].get_state()
    assert np.array_equal(base, other)


def test_ppm_rejected_combinations(hy):
    prob, W = inputs.sod(16)
    with pytest.raises(hy.HydroError):
        hy.Simulation(prob.replace(recon=PPM), W)            # MUSCL-Hancock
    p2 = ppm(prob.replace(n=(16, 2, 1)))
    with pytest.raises(hy.HydroError):
        hy.Simulation(p2, np.ones(p2.shape))                  # fewer than 3 cells
    prt, Wrt = inputs.rayleigh_taylor(8, nz=8, hse_subtract=1)
    with pytest.raises(hy.HydroError):
        hy.Simulation(ppm(prt), Wrt)                           # background mode
