"""The headline workload run in full against the oracle, and the FP32
batched path against the oracle.

* 3D single-fluid Rayleigh-Taylor, 256^3 FP64, 200 steps (the bench's
  default workload), whole grid, with and without hydrostatic-background
  subtraction: every conserved variable within L1-relative 1e-10 of the
  FP64 oracle run on all host cores (about 3.4e9 zone-updates per mode,
  1.5-2 minutes of oracle time each on a 16-core host).  The GPU uses the
  tile variant and z-chunk that the autotuner picks for the bench.
* A batch of Kelvin-Helmholtz boxes in FP32 (one persistent launch per
  step): density within the FP32 accuracy bound against the oracle.
"""

import os

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.headline]

TOL = 1e-10


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


def l1rel_per_var(U, V):
    scale = np.abs(V).sum() / V.shape[0]
    out = []
    for q in range(V.shape[0]):
        den = np.abs(V[q]).sum()
        out.append(float(np.abs(U[q] - V[q]).sum() / (den if den > 1e-3 * scale else scale)))
    return out


@pytest.mark.parametrize("hse", [0, 1], ids=["plain", "background"])
def test_rt256_fp64_200_steps_whole_grid(hy, orc, hse):
    from paper_1510_05061_gb300 import autotune

    steps = 200
    prob, W = inputs.rayleigh_taylor(256, hse_subtract=hse)
    sim = hy.Simulation(prob, W)
    choice = autotune.tune_simulation(sim)            # the bench's tile and z-chunk
    sim.close()
    sim = hy.Simulation(prob, W)
    sim.configure(choice["variant"], choice["zchunk"])
    sim.run_steps(steps)
    t_gpu = sim.t
    U = sim.conserved()
    sim.close()

    o = orc.Oracle(prob, threads=os.cpu_count() or 1)
    V, t, s, _ = o.run(o.state_from_prim(W), max_steps=steps)
    assert s == steps
    assert abs(t_gpu - t) <= 1e-12 * t
    errs = l1rel_per_var(U, o.total(V))
    assert max(errs) <= TOL, errs


def test_kh_batch_fp32_against_oracle(hy, orc):
    """Eight KH boxes of the batch workload's size law (32^3..64^3), FP32
    bulk with FP64 dt: after 20 steps each box's density is within 1e-4
    (L1-relative) of the FP64 oracle's."""
    sizes = inputs.kh_batch_sizes(count=8, nmin=32, nmax=64)
    items = [inputs.kelvin_helmholtz(s["n"], ndim=3, U=s["U"], ratio=s["ratio"], instance=s["instance"])
             for s in sizes]
    b = hy.Batch(items)
    b.step(20)
    for i, (p, W) in enumerate(items):
        o = orc.Oracle(p.replace(precision=inputs.FP64), threads=os.cpu_count() or 1)
        V, t, s, _ = o.run(o.state_from_prim(W), max_steps=20)
        assert abs(b.t(i) - t) <= 1e-5 * t
        rho_gpu = b.conserved(i)[0]
        rho = o.total(V)[0]
        err = float(np.abs(rho_gpu - rho).sum() / np.abs(rho).sum())
        assert err <= 1e-4, (i, err)
    b.close()
