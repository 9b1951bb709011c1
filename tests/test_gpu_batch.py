"""Batched solves: one persistent launch per step over a work list of
uneven instances.  Each instance's per-cell arithmetic is the single-solve
arithmetic, so every instance must equal its solo run bit for bit, for every
tile shape and z-chunk the autotuner may pick, and match the oracle."""

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


def mixed_fp64():
    return [
        inputs.rayleigh_taylor(20, nz=36, amplitude=0.05),
        inputs.kelvin_helmholtz(24, ndim=3, U=1.3, ratio=2.0, precision=inputs.FP64, instance=1),
        inputs.kelvin_helmholtz(17, ndim=3, U=0.7, ratio=3.5, precision=inputs.FP64, instance=2),
        inputs.kelvin_helmholtz(40, ndim=2, U=1.0, ratio=1.5, precision=inputs.FP64, instance=3),
        inputs.kelvin_helmholtz(70, ndim=2, U=1.9, ratio=2.5, precision=inputs.FP64, instance=4),
    ]


def solo_states(hy, items, steps):
    out = []
    for p, W in items:
        s = hy.Simulation(p, W)
        s.run_steps(steps)
        out.append((s.get_state(), s.t, s.nstep))
        s.close()
    return out


def batch_state(hy, b, i):
    return b.get_state(i)


@pytest.mark.parametrize("variant", [0, 1, 2, 4, 6])
def test_mixed_batch_equals_solo_bitwise(hy, variant):
    items = mixed_fp64()
    steps = 9
    solo = solo_states(hy, items, steps)
    b = hy.Batch(items)
    b.configure(variant, 0)
    b.step(steps)
    for i, (ref, t, n) in enumerate(solo):
        assert np.array_equal(batch_state(hy, b, i), ref), (variant, i)
        assert b.t(i) == t and b.nstep(i) == n
    b.close()


@pytest.mark.parametrize("zchunk", [1, 5, 64])
def test_batch_zchunk_invariance(hy, zchunk):
    items = mixed_fp64()[:3]
    b0 = hy.Batch(items)
    b0.step(6)
    ref = [batch_state(hy, b0, i) for i in range(3)]
    b1 = hy.Batch(items)
    b1.configure(2, zchunk)
    b1.step(6)
    for i in range(3):
        assert np.array_equal(batch_state(hy, b1, i), ref[i])
    b0.close()
    b1.close()


def test_batch_matches_oracle(hy):
    import oracle

    items = mixed_fp64()
    b = hy.Batch(items)
    b.step(5)
    for i, (p, W) in enumerate(items):
        o = oracle.Oracle(p)
        V, _, _, _ = o.run(o.state_from_prim(W), max_steps=5)
        U = b.conserved(i)
        for q in range(p.nvar):
            den = np.abs(V[q]).sum()
            if den > 1e-3 * np.abs(V).sum() / p.nvar:
                assert np.abs(U[q] - V[q]).sum() / den <= 1e-10, (i, q)
    b.close()


def test_kh_batch_fp32_graph_and_per_instance_dt(hy):
    sizes = inputs.kh_batch_sizes(count=8, nmin=32, nmax=64)
    items = [inputs.kelvin_helmholtz(s["n"], ndim=3, U=s["U"], ratio=s["ratio"], instance=s["instance"])
             for s in sizes]
    solo = solo_states(hy, items, 7)
    b = hy.Batch(items)
    n0 = b.launches()
    b.step(7)                       # graph replays plus one direct launch
    assert b.launches() - n0 == 7
    dts = set()
    for i, (ref, t, n) in enumerate(solo):
        assert np.array_equal(batch_state(hy, b, i), ref), i
        assert b.t(i) == t
        dts.add(t)
    assert len(dts) > 1             # each instance advanced with its own CFL dt
    b.close()


def test_batch_with_hse_instances(hy):
    items = [inputs.rayleigh_taylor(16, nz=32, amplitude=0.05, hse_subtract=1),
             inputs.rayleigh_taylor(24, nz=20, amplitude=0.02, hse_subtract=1, seed=7)]
    solo = solo_states(hy, items, 5)
    b = hy.Batch(items)
    b.step(5)
    for i, (ref, t, n) in enumerate(solo):
        assert np.array_equal(batch_state(hy, b, i), ref), i
    b.close()


def test_fp32_batch_all_tiles_equal_solo(hy):
    items = [inputs.kelvin_helmholtz(n, ndim=3, U=1.1, ratio=2.0, instance=i) for i, n in enumerate((21, 34, 40))]
    items.append(inputs.kelvin_helmholtz(90, ndim=2, U=1.4, ratio=3.0, instance=9))
    solo = solo_states(hy, items, 6)
    for v in (0, 1, 2, 3):
        b = hy.Batch(items)
        b.configure(v, 9)
        b.step(6)
        for i, (ref, t, n) in enumerate(solo):
            assert np.array_equal(b.get_state(i), ref), (v, i)
        b.close()
