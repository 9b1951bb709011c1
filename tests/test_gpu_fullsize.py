"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (the autotuned tile shape, staging depth and z-chunk), on sampled
outputs the oracle can compute on its own.

One step of Rayleigh-Taylor 256^3 (FP64) and 512^3 (FP32 with background
subtraction) is run on the GPU over the whole grid.  The oracle takes the
time step from the whole initial state (its own CFL reduction) and advances
z-slabs of the initial state, each 3 planes wider than the planes compared on
every side that is not a physical wall: a cell's update reads cells at most 2
planes away, so the compared planes are exact.  The slabs sample the bottom
wall, the interface and the top wall.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT

pytestmark = pytest.mark.gpu

MARGIN = 3


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


def slab_problem(prob, z0, z1):
    """The planes [z0, z1) as a problem of their own (x-y as the whole; a cut
    z side gets outflow, a physical wall keeps its condition)."""
    nz, dz = prob.n[2], prob.dx()[2]
    lo = list(prob.lo)
    hi = list(prob.hi)
    lo[2] = prob.lo[2] + z0 * dz
    hi[2] = prob.lo[2] + z1 * dz
    bcl, bch = list(prob.bc_lo), list(prob.bc_hi)
    if z0 > 0:
        bcl[2] = BC_OUTFLOW
    if z1 < nz:
        bch[2] = BC_OUTFLOW
    kw = dict(n=(prob.n[0], prob.n[1], z1 - z0), lo=tuple(lo), hi=tuple(hi), bc_lo=tuple(bcl), bc_hi=tuple(bch))
    if prob.hse_subtract:
        # background at the slab's planes -2 .. and faces -2 .. (global index + 2)
        kw.update(bg_rho_c=prob.bg_rho_c[z0:z1 + 4], bg_p_c=prob.bg_p_c[z0:z1 + 4],
                  bg_rho_f=prob.bg_rho_f[z0:z1 + 5], bg_p_f=prob.bg_p_f[z0:z1 + 5])
    return prob.replace(precision=inputs.FP64, **kw)


def compare(G, V, tol, label):
    scale = np.abs(V).sum() / V.shape[0]
    for q in range(V.shape[0]):
        den = np.abs(V[q]).sum()
        err = np.abs(G[q] - V[q]).sum() / (den if den > 1e-3 * scale else scale)
        assert err <= tol, f"{label} var {q}: {err:.3e}"


def run_case(hy, orc, prob, W, tol):
    from paper_1510_05061_gb300 import autotune

    nz = prob.n[2]
    sim = hy.Simulation(prob, W)
    tune = autotune.tune_simulation(sim)          # the configuration bench.py times
    sim.close()
    sim = hy.Simulation(prob, W)
    sim.configure(tune["variant"], tune["zchunk"])
    sim.step()
    G = sim.conserved()
    sim.close()
    # the oracle's own dt from the whole initial state
    o_full = orc.Oracle(prob.replace(precision=inputs.FP64), threads=0)
    dt = o_full.cfl_dt(o_full.state_from_prim(W))
    del o_full
    for a, b in ((0, 16), (nz // 2 - 8, nz // 2 + 8), (nz - 16, nz)):
        z0, z1 = max(0, a - MARGIN), min(nz, b + MARGIN)
        sp = slab_problem(prob, z0, z1)
        o = orc.Oracle(sp, threads=0)
        U = o.step(o.state_from_prim(np.ascontiguousarray(W[:, z0:z1])), dt)
        V = o.total(U)[:, a - z0:b - z0]
        compare(G[:, a:b], V, tol, f"{prob.name} planes {a}..{b}")
    return tune


def test_rt256_fp64_full_size_sampled(hy, orc):
    prob, W = inputs.rayleigh_taylor(256)
    run_case(hy, orc, prob, W, 1e-10)


def test_rt512_fp32_full_size_sampled(hy, orc):
    prob, W = inputs.rayleigh_taylor(512, precision=inputs.FP32, hse_subtract=1)
    run_case(hy, orc, prob, W, 1e-5)
