"""Row-vector staging of the step kernels.

A tile whose x halo lies inside the grid (and whose state is aligned, nx a
multiple of the vector width) stages its rows as aligned vectors of 2 or 4
cells; the other tiles load one cell at a time with boundary index mapping.
The two must give the same bits:

* translation: on a grid periodic in x, the solution of the initial state
  rolled by s cells along x is the rolled solution, bit for bit, although
  the roll moves cells between vector tiles and mapped tiles (nx = 72: with
  32-wide tiles the tiles at x0 = 0 and 64 are mapped, the one at 32 takes
  vectors; with 16-wide tiles those at 16, 32 and 48).  3D in both
  precisions for every tile variant (walls in y and z, so that mirrored
  rows take the vector path too), with and without the hydrostatic
  background; 2D in both precisions;
* every 3D tile variant and z-chunk gives the same bits on that grid;
* FP64 on that grid agrees with the oracle to 1e-10.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_PERIODIC, BC_REFLECT

pytestmark = pytest.mark.gpu

SHIFTS = (4, 36)


@pytest.fixture(scope="module")
def hy():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_05061_gb300 import build, hydro

    build.build()
    hydro.load()
    return hydro


def rt_walls(precision, hse):
    prob, W = inputs.rayleigh_taylor(72, nz=24, amplitude=0.05, hse_subtract=hse, precision=precision)
    prob = prob.replace(bc_lo=(BC_PERIODIC, BC_REFLECT, BC_REFLECT), bc_hi=(BC_PERIODIC, BC_REFLECT, BC_REFLECT))
    # a y-dependent shear so that the y rows differ
    y = prob.centres(1)
    W[1] = W[1] + 0.2 * np.sin(2 * np.pi * y)[None, :, None]
    return prob, W


def run(hy, prob, W, steps, variant=None, zchunk=0):
    sim = hy.Simulation(prob, W)
    if variant is not None:
        sim.configure(variant, zchunk)
    sim.run_steps(steps)
    U, t = sim.conserved(), sim.t
    sim.close()
    return U, t


def variants_for(hy, precision):
    # FP64: the 32x8, 32x4 and 16x16 tiles, synchronous and asynchronous
    # staging; FP32 also the 32x16 tiles and the paired-cell kernels
    if precision == inputs.FP64:
        return [0, 1, 2, 4, 5, 6]
    return [v for v, _ in hy.sim_variants()]


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("hse", [0, 1])
def test_roll_in_x_commutes_with_the_step_3d(hy, precision, hse):
    prob, W = rt_walls(precision, hse)
    for v in variants_for(hy, precision):
        U0, t0 = run(hy, prob, W, 6, v)
        for s in SHIFTS:
            Us, ts = run(hy, prob, np.roll(W, s, axis=-1), 6, v)
            assert ts == t0, (v, s)
            assert np.array_equal(Us, np.roll(U0, s, axis=-1)), (v, s)


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.FP32], ids=["fp64", "fp32"])
def test_roll_in_x_commutes_with_the_step_2d(hy, precision):
    prob, W = inputs.kelvin_helmholtz(72, ndim=2, U=1.2, precision=precision)
    U0, t0 = run(hy, prob, W, 8)
    for s in SHIFTS:
        Us, ts = run(hy, prob, np.roll(W, s, axis=-1), 8)
        assert ts == t0, s
        assert np.array_equal(Us, np.roll(U0, s, axis=-1)), s


@pytest.mark.parametrize("precision", [inputs.FP64, inputs.FP32], ids=["fp64", "fp32"])
def test_all_tiles_agree_on_a_vector_grid(hy, precision):
    prob, W = rt_walls(precision, 1)
    ref = None
    for v in variants_for(hy, precision):
        if v in hy.PAIR_VARIANTS:
            continue   # rounding of the packed arithmetic differs (own tests)
        for z in (0, 5):
            U, t = run(hy, prob, W, 5, v, z)
            if ref is None:
                ref = (U, t)
            else:
                assert t == ref[1], (v, z)
                assert np.array_equal(U, ref[0]), (v, z)


def test_vector_grid_against_the_oracle(hy):
    import oracle

    oracle.build()
    prob, W = rt_walls(inputs.FP64, 0)
    o = oracle.Oracle(prob)
    V, _, _, _ = o.run(o.state_from_prim(W), max_steps=6)
    Uo = o.total(V)
    U, _ = run(hy, prob, W, 6)
    # L1-relative per conserved variable (a variable with a vanishing total
    # against the scale of the others)
    scale = np.abs(Uo).sum() / Uo.shape[0]
    for q in range(5):
        den = np.abs(Uo[q]).sum()
        err = np.abs(U[q] - Uo[q]).sum() / (den if den > 1e-3 * scale else scale)
        assert err <= 1e-10, (q, err)
