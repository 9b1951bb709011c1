"""Parity of the SSP-RK2 method-of-lines integrator on the GPU (two stage
kernels per step) with the FP64 CPU oracle's SSP-RK2 mode, through the C ABI.

Same bar as the MUSCL-Hancock path: L1-relative 1e-10 per conserved variable
in FP64; FP32 held against the FP64 oracle at its rounding level.  Both sides
start from the same seeded inputs; nothing the GPU produces reaches the
oracle.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, SSPRK2, Problem

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


def gpu(hy, prob, W, steps=None, t_end=None):
    sim = hy.Simulation(prob, W)
    l0 = sim.launches()
    if t_end is not None:
        n, t = sim.advance_to(t_end)
    else:
        sim.run_steps(steps)
        n = steps
    launches = sim.launches() - l0
    return dict(U=sim.conserved(), t=sim.t, n=n, nstep=sim.nstep, launches=launches, sim=sim)


def ref(orc, prob, W, steps=None, t_end=None):
    o = orc.Oracle(prob)
    kw = dict(max_steps=steps) if t_end is None else dict(t_end=t_end)
    V, t, s, dl, dts = o.run(o.state_from_prim(W), record_dt=True, **kw)
    return dict(U=o.total(V), t=t, n=s, dts=dts)


def test_sod_rk2(hy, orc):
    prob, W = inputs.sod(128)
    prob = prob.replace(scheme=SSPRK2)
    g = gpu(hy, prob, W, t_end=0.2)
    o = ref(orc, prob, W, t_end=0.2)
    assert g["t"] == 0.2 and g["n"] == o["n"]
    assert_parity(g["U"], o["U"], label="sod rk2")
    P = g["sim"].primitive()
    assert (P[0] == P[0, :, :1, :]).all() and np.abs(P[2]).max() == 0.0
    rho_ex, _, _ = orc.exact_cell_average([1, 0, 1], [0.125, 0, 0.1], 1.4, 0.5, 0.2, np.linspace(0, 1, 129))
    assert l1rel(P[0, 0, 0], rho_ex) <= 1.5e-2


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, 0), (BC_REFLECT, BC_PERIODIC, 0), (0.0, -0.5, 0.0)),
    ((BC_REFLECT, BC_OUTFLOW, 0), (BC_OUTFLOW, BC_REFLECT, 0), (0.3, 0.2, 0.0)),
])
def test_rk2_2d_ragged(hy, orc, bcl, bch, g):
    prob = Problem(ndim=2, n=(131, 67, 1), hi=(1.3, 0.7, 1.0), bc_lo=bcl, bc_hi=bch, grav=g, scheme=SSPRK2)
    W = smooth_random(prob, 17)
    gr = gpu(hy, prob, W, steps=30)
    o = ref(orc, prob, W, steps=30)
    assert gr["launches"] == 60
    assert_parity(gr["U"], o["U"], label=f"rk2 2d {bcl} {bch}")
    assert abs(gr["t"] - o["t"]) <= 1e-12 * o["t"]


@pytest.mark.parametrize("bcl,bch,g", [
    ((BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), (BC_REFLECT, BC_PERIODIC, BC_REFLECT), (0.0, 0.0, -1.0)),
    ((BC_PERIODIC, BC_REFLECT, BC_OUTFLOW), (BC_PERIODIC, BC_OUTFLOW, BC_OUTFLOW), (0.2, -0.3, 0.5)),
])
def test_rk2_3d_ragged(hy, orc, bcl, bch, g):
    prob = Problem(ndim=3, n=(37, 29, 23), hi=(1.0, 0.8, 0.6), bc_lo=bcl, bc_hi=bch, grav=g, scheme=SSPRK2)
    W = smooth_random(prob, 23)
    gr = gpu(hy, prob, W, steps=15)
    o = ref(orc, prob, W, steps=15)
    assert_parity(gr["U"], o["U"], label=f"rk2 3d {bcl} {bch}")


@pytest.mark.parametrize("hse", [0, 1])
def test_rk2_rayleigh_taylor(hy, orc, hse):
    prob, W = inputs.rayleigh_taylor(24, nz=36, amplitude=0.05, hse_subtract=hse)
    prob = prob.replace(scheme=SSPRK2)
    gr = gpu(hy, prob, W, steps=20)
    o = ref(orc, prob, W, steps=20)
    assert_parity(gr["U"], o["U"], label=f"rk2 rt hse={hse}")
    np.testing.assert_allclose(gr["t"], o["t"], rtol=1e-12)


def test_rk2_dt_sequence_and_t_end(hy, orc):
    prob, W = inputs.kelvin_helmholtz(24, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    prob = prob.replace(scheme=SSPRK2)
    sim = hy.Simulation(prob, W)
    dts = [sim.step(want_dt=True) for _ in range(12)]
    o = ref(orc, prob, W, steps=12)
    np.testing.assert_allclose(dts, o["dts"], rtol=1e-12, atol=0)
    # advance_to lands on t_end and then carries the state over unchanged
    t_end = sim.t + 2.5 * dts[-1]
    n, t = sim.advance_to(t_end)
    assert t == t_end and n == 3
    before = sim.get_state()
    n2, _ = sim.advance_to(t_end)
    assert n2 == 0 and np.array_equal(sim.get_state(), before)


@pytest.mark.parametrize("variant,zchunk", [(0, 0), (1, 5), (2, 64)])
def test_rk2_tile_and_chunk_invariance(hy, variant, zchunk):
    prob, W = inputs.rayleigh_taylor(40, nz=30, amplitude=0.05, hse_subtract=1)
    prob = prob.replace(scheme=SSPRK2)
    base = hy.Simulation(prob, W)
    base.run_steps(4)
    ref_state = base.get_state()
    base.close()
    sim = hy.Simulation(prob, W)
    sim.configure(variant, zchunk)
    sim.run_steps(4)
    assert np.array_equal(sim.get_state(), ref_state)


@pytest.mark.parametrize("variant,zchunk", [(0, 0), (2, 5), (3, 64)])
def test_rk2_fp32_tile_and_chunk_invariance(hy, variant, zchunk):
    """FP32 stages: tiles whose staged-plane ring has a spare slot (staging
    and half step in one barrier interval) and tiles without it give the
    same bits."""
    prob, W = inputs.rayleigh_taylor(40, nz=30, amplitude=0.05, hse_subtract=1, precision=inputs.FP32)
    prob = prob.replace(scheme=SSPRK2)
    base = hy.Simulation(prob, W)
    base.run_steps(4)
    ref_state = base.get_state()
    base.close()
    sim = hy.Simulation(prob, W)
    sim.configure(variant, zchunk)
    sim.run_steps(4)
    assert np.array_equal(sim.get_state(), ref_state)


def test_rk2_fp32_rayleigh_taylor_against_fp64_oracle(hy, orc):
    prob, W = inputs.rayleigh_taylor(32, amplitude=0.05, hse_subtract=1)
    p32 = prob.replace(scheme=SSPRK2, precision=inputs.FP32)
    gr = gpu(hy, p32, W, steps=20)
    o = ref(orc, prob.replace(scheme=SSPRK2), W, steps=20)
    assert l1rel(gr["U"][0], o["U"][0]) <= 1e-5


def test_rk2_conserves_on_periodic_grid(hy):
    prob, W = inputs.kelvin_helmholtz(32, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    prob = prob.replace(scheme=SSPRK2)
    sim = hy.Simulation(prob, W)
    T0, U0 = sim.totals(), sim.conserved()
    sim.run_steps(50)
    T1 = sim.totals()
    dV = np.prod(prob.dx())
    mom_scale = np.abs(U0[1:4]).sum() * dV
    for q in range(5):
        scale = mom_scale if 1 <= q <= 3 else np.abs(U0[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


def test_rk2_not_offered_in_batches_and_slabs(hy):
    prob, W = inputs.kelvin_helmholtz(16, ndim=3, U=1.0, ratio=2.0, precision=inputs.FP32)
    prob = prob.replace(scheme=SSPRK2)
    with pytest.raises(hy.HydroError):
        hy.Batch([(prob, W)])
    with pytest.raises(hy.HydroError):
        hy.Slabs(prob.replace(precision=inputs.FP64), W, 2)
