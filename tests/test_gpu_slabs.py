"""The z-slab decomposition on the GPU (virtual ranks on one device).

Given the same state and dt every slab computes exactly the cells the
undivided solve computes, so the decomposed run must be bitwise identical
to ``Simulation`` on the whole grid for any number of slabs, even and
uneven splits, every z boundary kind, the hydrostatic-background mode and
both precisions.  The FP64 runs are also held against the oracle.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT

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


def rt(n=24, nz=26, **kw):
    return inputs.rayleigh_taylor(n=n, nz=nz, amplitude=0.05, **kw)


def whole(hy, prob, W, steps):
    sim = hy.Simulation(prob, W)
    sim.run_steps(steps)
    out = (sim.get_state(), sim.t, sim.nstep, sim.dt, sim.totals())
    sim.close()
    return out


def sliced(hy, prob, W, R, steps, variant=None, zchunk=0):
    s = hy.Slabs(prob, W, R)
    if variant is not None:
        s.configure(variant, zchunk)
    l0 = s.launches()
    s.step(steps)
    launches = s.launches() - l0
    out = (s.get_state(), s.t, s.nstep, s.dt, s.totals())
    s.close()
    assert launches == steps * (R + 1)
    return out


def assert_parity(U, V, tol=1e-10, label=""):
    """L1-relative difference per conserved variable (FP64 parity bar)."""
    scale = np.abs(V).sum() / V.shape[0]
    for q in range(V.shape[0]):
        den = np.abs(V[q]).sum()
        err = np.abs(U[q] - V[q]).sum() / (den if den > 1e-3 * scale else scale)
        assert err <= tol, f"{label} var {q}: L1-rel {err:.3e}"


def assert_same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2] and a[3] == b[3]
    np.testing.assert_allclose(a[4], b[4], rtol=1e-12, atol=1e-12 * np.abs(b[4]).max())


CASES = {
    "rt-reflect": lambda: rt(),
    "rt-reflect-hse": lambda: rt(hse_subtract=1),
    "rt-reflect-fp32": lambda: rt(precision=inputs.FP32),
    "rt-reflect-fp32-hse": lambda: rt(precision=inputs.FP32, hse_subtract=1),
    "rt-outflow": lambda: (lambda p, W: (p.replace(bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_OUTFLOW),
                                                   bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_OUTFLOW)), W))(*rt()),
    "pulse-periodic": lambda: inputs.smooth_pulse(24, ndim=3),
    "kh-periodic-ragged": lambda: inputs.kelvin_helmholtz(19, ndim=3, precision=inputs.FP64),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_slabs_match_undivided(hy, name, R):
    prob, W = CASES[name]()
    steps = 6
    ref = whole(hy, prob, W, steps)
    got = sliced(hy, prob, W, R, steps)
    assert_same(got, ref)


@pytest.mark.parametrize("variant,zchunk", [(1, 3), (2, 0), (0, 1), (6, -1), (0, -1), (2, -4)])
def test_slabs_tile_and_chunk_invariance(hy, variant, zchunk):
    prob, W = rt(n=40, nz=30)
    ref = whole(hy, prob, W, 5)
    assert_same(sliced(hy, prob, W, 3, 5, variant, zchunk), ref)


def test_slabs_against_oracle(hy):
    import oracle
    oracle.build()
    prob, W = rt(n=16, nz=22, hse_subtract=1)
    steps = 5
    s = hy.Slabs(prob, W, 4)
    s.step(steps)
    G, t = s.conserved(), s.t
    s.close()
    o = oracle.Oracle(prob)
    V, t_o, n_o, _, _ = o.run(o.state_from_prim(W), max_steps=steps, record_dt=True)
    assert n_o == steps
    assert_parity(G, o.total(V), label="slabs vs oracle")
    assert abs(t - t_o) <= 1e-12 * t_o


def test_slabs_reject_bad_splits(hy):
    prob, W = rt(n=8, nz=6)
    with pytest.raises(hy.HydroError):
        hy.Slabs(prob, W, 4)          # fewer than two planes per slab
    p2, W2 = inputs.sod(n=16, ndim=2)
    with pytest.raises(hy.HydroError):
        hy.Slabs(p2, W2, 2)
