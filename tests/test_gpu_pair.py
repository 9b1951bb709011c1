"""The paired-cell FP32 MUSCL-Hancock step (tile variants 8..10: two
x-adjacent cells per thread, packed f32x2 arithmetic).

* every paired tile shape and z-chunk gives the same bits (ragged sizes,
  reflecting walls, background mode, gravity with x and y components);
* it agrees with the scalar FP32 step (variants 0..7) to FP32 rounding;
* against the FP64 oracle it meets the FP32 accuracy bounds, on smooth
  Rayleigh-Taylor data, on a Kelvin-Helmholtz box, and on data that takes
  the positivity fallback (the boosted Toro tube along x and y, the
  near-vacuum filament column);
* it conserves mass and energy between reflecting walls to FP32 rounding.
"""

import json
import os

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_PERIODIC, BC_REFLECT, Problem

pytestmark = pytest.mark.gpu

PAIRS = (8, 9, 10)
HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "toro_riemann_star.json")) as _fh:
    TORO = {t["name"]: t for t in json.load(_fh)["tests"]}


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


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def run(hy, prob, W, variant, steps, zchunk=0):
    sim = hy.Simulation(prob, W)
    sim.configure(variant, zchunk)
    sim.run_steps(steps)
    raw, U, t = sim.get_state(), sim.conserved(), sim.t
    sim.close()
    return raw, U, t


def cases():
    rt, W = inputs.rayleigh_taylor(37, nz=45, amplitude=0.05, hse_subtract=1, precision=inputs.FP32)
    rt = rt.replace(n=(37, 37, 45))
    rt_plain, Wp = inputs.rayleigh_taylor(37, nz=45, amplitude=0.05, precision=inputs.FP32)
    rt_plain = rt_plain.replace(n=(37, 37, 45))
    # gravity with x and y components, outflow in x, reflecting in y
    gen = rt_plain.replace(grav=(0.2, -0.3, -1.0), bc_lo=(0, BC_REFLECT, BC_REFLECT),
                           bc_hi=(0, BC_REFLECT, BC_REFLECT))
    kh, Wk = inputs.kelvin_helmholtz(40, ndim=3, U=1.4, ratio=2.5, precision=inputs.FP32)
    kh = kh.replace(n=(40, 40, 40))
    return [("rt_hse", rt, W), ("rt_plain", rt_plain, Wp), ("general_gravity", gen, Wp), ("kh", kh, Wk)]


CASES = cases()


@pytest.mark.parametrize("name,prob,W", CASES, ids=[c[0] for c in CASES])
def test_paired_tiles_and_chunks_agree_bitwise(hy, name, prob, W):
    ref = None
    for v in PAIRS:
        for z in (0, 7, 64):
            raw, _, t = run(hy, prob, W, v, 5, z)
            if ref is None:
                ref = (raw, t)
            else:
                assert np.array_equal(raw, ref[0]), (v, z)
                assert t == ref[1]


@pytest.mark.parametrize("name,prob,W", CASES, ids=[c[0] for c in CASES])
def test_paired_step_agrees_with_scalar_fp32_step(hy, name, prob, W):
    _, Up, tp = run(hy, prob, W, 8, 10)
    _, Us, ts = run(hy, prob, W, 7, 10)
    assert abs(tp - ts) <= 1e-6 * ts
    for q in range(5):
        den = np.abs(Us[q]).sum()
        if den > 1e-3 * np.abs(Us).sum() / 5:
            # rounding differences, amplified where a momentum is small
            # against its fluctuations (the KH box's v_y noise)
            assert l1rel(Up[q], Us[q]) <= 1e-4, (name, q)


@pytest.mark.parametrize("hse", [0, 1])
def test_paired_step_against_fp64_oracle(hy, orc, hse):
    prob, W = inputs.rayleigh_taylor(32, amplitude=0.05, hse_subtract=hse)
    o = orc.Oracle(prob)
    V, _, _, _ = o.run(o.state_from_prim(W), max_steps=40)
    _, U, _ = run(hy, prob.replace(precision=inputs.FP32), W, 9, 40)
    assert l1rel(U[0], o.total(V)[0]) <= 1e-5


def test_paired_step_rt_linear_phase_against_oracle(hy, orc):
    """RT 64^3 with the background, to t = 0.5: density within 1e-3 of the
    FP64 oracle (the FP32 accuracy bound of the linear-growth phase)."""
    prob, W = inputs.rayleigh_taylor(64, hse_subtract=1)
    o = orc.Oracle(prob, threads=os.cpu_count() or 1)
    V, _, _, _ = o.run(o.state_from_prim(W), t_end=0.5)
    sim = hy.Simulation(prob.replace(precision=inputs.FP32), W)
    sim.configure(8, 0)
    n, t = sim.advance_to(0.5)
    assert t == 0.5
    rho = sim.primitive()[0]
    sim.close()
    assert l1rel(rho, o.prim(V)[0]) <= 1e-3


@pytest.mark.parametrize("axis", [0, 1])
def test_paired_step_on_fallback_data(hy, orc, axis):
    """The boosted Toro test 4 tube (cells take the positivity fallback) in
    FP32 with paired tiles: close to the scalar FP32 step and to the oracle."""
    t = TORO["test4_right_blast"]
    prob, W = inputs.riemann_tube(120, t["left"], t["right"], x0=0.5 - 5.0 * 0.035, boost=5.0, axis=axis, ndim=3)
    orc.fallback_counts(reset=True)
    o = orc.Oracle(prob)
    V, tt, s, _ = o.run(o.state_from_prim(W), t_end=0.035)
    assert orc.fallback_counts(reset=True)[0] > 50
    out = {}
    for v in (8, 7):
        sim = hy.Simulation(prob.replace(precision=inputs.FP32), W)
        sim.configure(v, 0)
        n, tg = sim.advance_to(0.035)
        out[v] = sim.conserved()[0]
        sim.close()
    rho = o.total(V)[0]
    assert l1rel(out[8], rho) <= 1e-4
    assert l1rel(out[8], out[7]) <= 1e-4


@pytest.mark.parametrize("hse", [0, 1])
def test_paired_step_on_the_filament_column(hy, orc, hse):
    prob, W = inputs.filament_column(nz=48, stream=3.0, hse_subtract=hse)
    o = orc.Oracle(prob)
    V, _, _, _ = o.run(o.state_from_prim(W), max_steps=10)
    _, U, _ = run(hy, prob.replace(precision=inputs.FP32), W, 10, 10)
    assert l1rel(U[0], o.total(V)[0]) <= 1e-4


def test_paired_step_conserves_between_walls(hy):
    prob = Problem(ndim=3, n=(34, 30, 26), bc_lo=(BC_REFLECT,) * 3, bc_hi=(BC_REFLECT,) * 3,
                   precision=inputs.FP32)
    rng = np.random.default_rng(5)
    W = np.zeros(prob.shape)
    W[0] = 1.0 + 0.3 * rng.random(prob.shape[1:])
    W[1:4] = 0.4 * (rng.random((3,) + prob.shape[1:]) - 0.5)
    W[4] = 1.0 + 0.3 * rng.random(prob.shape[1:])
    sim = hy.Simulation(prob, W)
    sim.configure(8, 0)
    T0 = sim.totals()
    sim.run_steps(20)
    T1 = sim.totals()
    sim.close()
    for q in (0, 4):
        assert abs(T1[q] - T0[q]) <= 1e-5 * abs(T0[q]), q
