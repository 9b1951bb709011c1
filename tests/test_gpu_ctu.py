"""Parity of the corner transport upwind step on the GPU (one fused kernel
per step) with the FP64 CPU oracle's CTU mode, through the C ABI.  Same bar
as the other paths: L1-relative 1e-10 per conserved variable in FP64."""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, CTU, Problem

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


def ctu(prob):
    return prob.replace(scheme=CTU)


def gpu(hy, prob, W, steps=None, t_end=None):
    sim = hy.Simulation(prob, W)
    l0 = sim.launches()
    if t_end is not None:
        n, t = sim.advance_to(t_end)
    else:
        sim.run_steps(steps)
        n = steps
    launches = sim.launches() - l0
    return dict(U=sim.conserved(), t=sim.t, n=n, launches=launches, sim=sim)


def ref(orc, prob, W, steps=None, t_end=None):
    o = orc.Oracle(prob)
    kw = dict(max_steps=steps) if t_end is None else dict(t_end=t_end)
    V, t, s, dl, dts = o.run(o.state_from_prim(W), record_dt=True, **kw)
    return dict(U=o.total(V), t=t, n=s, dts=dts)


def test_ctu_sod(hy, orc):
    prob, W = inputs.sod(128)
    prob = ctu(prob)
    g = gpu(hy, prob, W, t_end=0.2)
    o = ref(orc, prob, W, t_end=0.2)
    assert g["t"] == 0.2 and g["n"] == o["n"]
    assert_parity(g["U"], o["U"], label="sod ctu")
    P = g["sim"].primitive()
    assert (P[0] == P[0, :, :1, :]).all() and np.abs(P[2]).max() == 0.0


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, 0), (BC_REFLECT, BC_PERIODIC, 0), (0.0, -0.5, 0.0)),
    ((BC_PERIODIC, BC_REFLECT, 0), (BC_PERIODIC, BC_REFLECT, 0), (0.0, -1.0, 0.0)),
    ((BC_REFLECT, BC_OUTFLOW, 0), (BC_OUTFLOW, BC_REFLECT, 0), (0.3, 0.2, 0.0)),
])
def test_ctu_2d_ragged(hy, orc, bcl, bch, g):
    prob = ctu(Problem(ndim=2, n=(131, 67, 1), hi=(1.3, 0.7, 1.0), bc_lo=bcl, bc_hi=bch, grav=g))
    W = smooth_random(prob, 17)
    gr = gpu(hy, prob, W, steps=40)
    o = ref(orc, prob, W, steps=40)
    assert gr["launches"] == 40
    assert_parity(gr["U"], o["U"], label=f"ctu 2d {bcl} {bch}")
    assert abs(gr["t"] - o["t"]) <= 1e-12 * o["t"]


@pytest.mark.parametrize("shape", [(2, 2, 1), (3, 41, 1), (45, 2, 1), (33, 9, 1)])
def test_ctu_tiny_and_odd_grids(hy, orc, shape):
    prob = ctu(Problem(ndim=2, n=shape, bc_lo=(BC_REFLECT, BC_PERIODIC, 0),
                       bc_hi=(BC_OUTFLOW, BC_PERIODIC, 0), grav=(-0.3, 0.0, 0.0)))
    W = smooth_random(prob, 6, jump=False)
    gr = gpu(hy, prob, W, steps=6)
    o = ref(orc, prob, W, steps=6)
    assert_parity(gr["U"], o["U"], label=str(shape))


def test_ctu_kelvin_helmholtz_dt_sequence_and_fp32(hy, orc):
    prob, W = inputs.kelvin_helmholtz(96, ndim=2, U=1.0, ratio=2.0, precision=inputs.FP64)
    prob = ctu(prob)
    sim = hy.Simulation(prob, W)
    dts = [sim.step(want_dt=True) for _ in range(20)]
    o = ref(orc, prob, W, steps=20)
    np.testing.assert_allclose(dts, o["dts"], rtol=1e-12, atol=0)
    assert_parity(sim.conserved(), o["U"], label="kh ctu")
    g32 = gpu(hy, prob.replace(precision=inputs.FP32), W, steps=20)
    assert l1rel(g32["U"][0], o["U"][0]) <= 1e-5


def test_ctu_conserves_on_periodic_grid(hy):
    prob, W = inputs.kelvin_helmholtz(64, ndim=2, U=1.5, ratio=3.0, precision=inputs.FP64)
    sim = hy.Simulation(ctu(prob), W)
    T0, U0 = sim.totals(), sim.conserved()
    sim.run_steps(100)
    T1 = sim.totals()
    dV = np.prod(prob.dx()[:2])
    mom_scale = np.abs(U0[1:3]).sum() * dV
    for q in range(4):
        scale = mom_scale if 1 <= q <= 2 else np.abs(U0[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), (BC_REFLECT, BC_PERIODIC, BC_REFLECT), (0.0, 0.0, -1.0)),
    ((BC_PERIODIC, BC_REFLECT, BC_OUTFLOW), (BC_PERIODIC, BC_OUTFLOW, BC_OUTFLOW), (0.2, -0.3, 0.5)),
    ((BC_PERIODIC,) * 3, (BC_PERIODIC,) * 3, (0.0, 0.0, 0.0)),
])
def test_ctu_3d_ragged(hy, orc, bcl, bch, g):
    prob = ctu(Problem(ndim=3, n=(37, 29, 23), hi=(1.0, 0.8, 0.6), bc_lo=bcl, bc_hi=bch, grav=g))
    W = smooth_random(prob, 23)
    gr = gpu(hy, prob, W, steps=15)
    o = ref(orc, prob, W, steps=15)
    assert gr["launches"] == 15
    assert_parity(gr["U"], o["U"], label=f"ctu 3d {bcl} {bch}")


@pytest.mark.parametrize("shape", [(2, 2, 2), (5, 3, 7), (33, 9, 3), (9, 17, 5)])
def test_ctu_3d_tiny_and_odd_grids(hy, orc, shape):
    prob = ctu(Problem(ndim=3, n=shape, bc_lo=(BC_REFLECT, BC_PERIODIC, BC_OUTFLOW),
                       bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.1, -0.4)))
    W = smooth_random(prob, 5, jump=False)
    gr = gpu(hy, prob, W, steps=6)
    o = ref(orc, prob, W, steps=6)
    assert_parity(gr["U"], o["U"], label=str(shape))


def test_ctu_3d_rayleigh_taylor_and_fp32(hy, orc):
    prob, W = inputs.rayleigh_taylor(24, nz=40, amplitude=0.05)
    prob = ctu(prob)
    gr = gpu(hy, prob, W, steps=20)
    o = ref(orc, prob, W, steps=20)
    assert_parity(gr["U"], o["U"], label="ctu rt")
    np.testing.assert_allclose(gr["t"], o["t"], rtol=1e-12)
    g32 = gpu(hy, prob.replace(precision=inputs.FP32), W, steps=20)
    assert l1rel(g32["U"][0], o["U"][0]) <= 1e-5


def test_ctu_3d_conserves_on_periodic_grid(hy):
    prob, W = inputs.kelvin_helmholtz(24, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    sim = hy.Simulation(ctu(prob), W)
    T0, U0 = sim.totals(), sim.conserved()
    sim.run_steps(50)
    T1 = sim.totals()
    dV = np.prod(prob.dx())
    mom_scale = np.abs(U0[1:4]).sum() * dV
    for q in range(5):
        scale = mom_scale if 1 <= q <= 3 else np.abs(U0[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


@pytest.mark.parametrize("n,nz,top", [(24, 40, BC_REFLECT), (37, 45, BC_OUTFLOW), (9, 5, BC_REFLECT)])
def test_ctu_3d_hydrostatic_background(hy, orc, n, nz, top):
    """Perturbation storage: the GPU step against the oracle's CTU step in
    the same mode (ragged tiles, several z-chunks, an open top)."""
    prob, W = inputs.rayleigh_taylor(n, nz=nz, amplitude=0.05, hse_subtract=1)
    prob = ctu(prob).replace(bc_hi=(BC_PERIODIC, BC_PERIODIC, top))
    gr = gpu(hy, prob, W, steps=20)
    o = ref(orc, prob, W, steps=20)
    assert gr["launches"] == 20
    assert_parity(gr["U"], o["U"], label=f"ctu hse {n} {nz}")
    np.testing.assert_allclose(gr["t"], o["t"], rtol=1e-12)


def test_ctu_3d_hydrostatic_background_fp32(hy, orc):
    prob, W = inputs.rayleigh_taylor(32, amplitude=0.05, hse_subtract=1)
    prob = ctu(prob)
    o = ref(orc, prob, W, steps=40)
    g32 = gpu(hy, prob.replace(precision=inputs.FP32), W, steps=40)
    assert l1rel(g32["U"][0], o["U"][0]) <= 1e-5
    # the z momentum is the perturbation's own flow here (no hydrostatic
    # imbalance of the discretised background to hide FP32 rounding in)
    assert l1rel(g32["U"][3], o["U"][3]) <= 3e-5


def test_ctu_rejected_combinations(hy):
    ps, Ws = inputs.sod(16)
    with pytest.raises(hy.HydroError):
        hy.Simulation(ctu(ps).replace(recon=inputs.PPM), Ws)      # PPM
