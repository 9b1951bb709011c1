"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance: L1-relative difference sum|a - b| / sum|b| <= 1e-10 per conserved
variable for FP64 (a variable whose oracle total is exactly zero is compared
against the scale of the other variables).  Both sides start from the same
seeded primitive fields built by paper_1510_05061_gb300.inputs; the oracle
never sees a value produced by the GPU.
"""

import math

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, Problem

pytestmark = pytest.mark.gpu

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


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def assert_parity(U, V, tol=TOL, label=""):
    """U from the GPU, V from the oracle, both FP64 total conserved."""
    scale = np.abs(V).sum() / V.shape[0]
    for q in range(V.shape[0]):
        den = np.abs(V[q]).sum()
        err = np.abs(U[q] - V[q]).sum() / (den if den > 1e-3 * scale else scale)
        assert err <= tol, f"{label} var {q}: L1-rel {err:.3e}"


def gpu_run(hy, prob, W, steps=None, t_end=None):
    sim = hy.Simulation(prob, W)
    if t_end is not None:
        n, t = sim.advance_to(t_end)
    else:
        sim.run_steps(steps)
        n, t = steps, sim.t
    U = sim.conserved()
    out = dict(U=U, n=n, t=t, nstep=sim.nstep, sim=sim)
    return out


def oracle_run(orc, prob, W, steps=None, t_end=None):
    o = orc.Oracle(prob)
    kw = dict(max_steps=steps) if t_end is None else dict(t_end=t_end)
    V, t, s, dl, dts = o.run(o.state_from_prim(W), record_dt=True, **kw)
    return dict(U=o.total(V), t=t, n=s, dts=dts, o=o)


def smooth_random(prob, seed, amp=0.2, jump=True):
    rng = np.random.default_rng(seed)
    nd = prob.ndim
    axes = [prob.centres(d) for d in range(nd)]
    W = np.zeros(prob.shape)
    for q in range(prob.nvar):
        f = np.zeros(prob.shape[1:])
        for _ in range(4):
            k = rng.integers(1, 3, nd)
            ph = rng.uniform(0, 2 * math.pi)
            arg = ph
            for d in range(nd):
                shape = [1, 1, 1]
                shape[2 - d] = -1
                arg = arg + 2 * math.pi * k[d] * axes[d].reshape(shape)
            f = f + rng.normal() * np.cos(arg)
        W[q] = f
    W[0] = 1.0 + amp * W[0] / np.abs(W[0]).max()
    W[-1] = 1.0 + amp * W[-1] / np.abs(W[-1]).max()
    for d in range(nd):
        W[1 + d] = 0.5 * W[1 + d] / np.abs(W[1 + d]).max()
    if jump:
        W[0, ..., : prob.n[0] // 2] *= 1.6
        W[-1, ..., : prob.n[0] // 3] *= 2.0
    return W


# --------------------------------------------------------------------- 2D
def test_sod_128_parity_and_exact(hy, orc):
    prob, W = inputs.sod(128)
    g = gpu_run(hy, prob, W, t_end=0.2)
    o = oracle_run(orc, prob, W, t_end=0.2)
    assert g["t"] == 0.2 and o["t"] == 0.2
    assert g["n"] == o["n"] == g["nstep"]
    assert_parity(g["U"], o["U"], label="sod")
    P = g["sim"].primitive()
    rho_ex, _, _ = orc.exact_cell_average([1, 0, 1], [0.125, 0, 0.1], 1.4, 0.5, 0.2,
                                          np.linspace(0, 1, 129))
    assert l1rel(P[0, 0, 0], rho_ex) <= 1.5e-2
    assert (P[0] == P[0, :, :1, :]).all()       # rows identical on the GPU too
    assert np.abs(P[2]).max() == 0.0


BC2D = [
    ((BC_OUTFLOW, BC_PERIODIC, 0), (BC_REFLECT, BC_PERIODIC, 0), (0.0, -0.5, 0.0)),
    ((BC_PERIODIC, BC_REFLECT, 0), (BC_PERIODIC, BC_REFLECT, 0), (0.0, -1.0, 0.0)),
    ((BC_REFLECT, BC_OUTFLOW, 0), (BC_OUTFLOW, BC_OUTFLOW, 0), (0.3, 0.2, 0.0)),
]


@pytest.mark.parametrize("bcl,bch,g", BC2D)
def test_parity_2d_ragged(hy, orc, bcl, bch, g):
    prob = Problem(ndim=2, n=(131, 67, 1), hi=(1.3, 0.7, 1.0), bc_lo=bcl, bc_hi=bch, grav=g)
    W = smooth_random(prob, 17)
    gr = gpu_run(hy, prob, W, steps=40)
    o = oracle_run(orc, prob, W, steps=40)
    assert_parity(gr["U"], o["U"], label=f"2d {bcl} {bch}")
    assert abs(gr["t"] - o["t"]) <= 1e-12 * o["t"]


# --------------------------------------------------------------------- 3D
BC3D = [
    ((BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), (BC_REFLECT, BC_PERIODIC, BC_REFLECT), (0.0, 0.0, -1.0)),
    ((BC_PERIODIC, BC_REFLECT, BC_OUTFLOW), (BC_PERIODIC, BC_OUTFLOW, BC_OUTFLOW), (0.2, -0.3, 0.5)),
    ((BC_PERIODIC,) * 3, (BC_PERIODIC,) * 3, (0.0, 0.0, 0.0)),
]


@pytest.mark.parametrize("bcl,bch,g", BC3D)
def test_parity_3d_ragged(hy, orc, bcl, bch, g):
    prob = Problem(ndim=3, n=(37, 29, 23), hi=(1.0, 0.8, 0.6), bc_lo=bcl, bc_hi=bch, grav=g)
    W = smooth_random(prob, 23)
    gr = gpu_run(hy, prob, W, steps=20)
    o = oracle_run(orc, prob, W, steps=20)
    assert_parity(gr["U"], o["U"], label=f"3d {bcl} {bch}")


@pytest.mark.parametrize("hse", [0, 1])
def test_parity_rayleigh_taylor_small(hy, orc, hse):
    prob, W = inputs.rayleigh_taylor(32, amplitude=0.05, hse_subtract=hse)
    gr = gpu_run(hy, prob, W, steps=30)
    o = oracle_run(orc, prob, W, steps=30)
    assert_parity(gr["U"], o["U"], label=f"rt hse={hse}")


def test_parity_hse_ragged_chunks(hy, orc):
    prob, W = inputs.rayleigh_taylor(20, nz=45, amplitude=0.05, hse_subtract=1)
    prob = prob.replace(n=(20, 20, 45))
    gr = gpu_run(hy, prob, W, steps=15)
    o = oracle_run(orc, prob, W, steps=15)
    assert_parity(gr["U"], o["U"], label="rt hse ragged")


def test_dt_sequence_matches_oracle(hy, orc):
    prob, W = inputs.kelvin_helmholtz(24, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    sim = hy.Simulation(prob, W)
    dts = [sim.step(want_dt=True) for _ in range(25)]
    o = oracle_run(orc, prob, W, steps=25)
    np.testing.assert_allclose(dts, o["dts"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("shape", [(2, 2, 2), (5, 3, 7), (33, 9, 3)])
def test_tiny_and_odd_grids_3d(hy, orc, shape):
    prob = Problem(ndim=3, n=shape, bc_lo=(BC_REFLECT, BC_PERIODIC, BC_OUTFLOW),
                   bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.1, -0.4))
    W = smooth_random(prob, 5, jump=False)
    gr = gpu_run(hy, prob, W, steps=6)
    o = oracle_run(orc, prob, W, steps=6)
    assert_parity(gr["U"], o["U"], label=str(shape))


@pytest.mark.parametrize("shape", [(2, 2, 1), (3, 41, 1), (45, 2, 1)])
def test_tiny_and_odd_grids_2d(hy, orc, shape):
    prob = Problem(ndim=2, n=shape, bc_lo=(BC_REFLECT, BC_PERIODIC, 0),
                   bc_hi=(BC_OUTFLOW, BC_PERIODIC, 0), grav=(-0.3, 0.0, 0.0))
    W = smooth_random(prob, 6, jump=False)
    gr = gpu_run(hy, prob, W, steps=6)
    o = oracle_run(orc, prob, W, steps=6)
    assert_parity(gr["U"], o["U"], label=str(shape))


# -------------------------------------------------------- time control
def test_advance_to_lands_on_t_end(hy, orc):
    prob, W = inputs.kelvin_helmholtz(64, ndim=2, U=1.0, ratio=2.0, precision=inputs.FP64)
    sim = hy.Simulation(prob, W)
    n, t = sim.advance_to(0.05)
    assert t == 0.05 and sim.t == 0.05
    o = oracle_run(orc, prob, W, t_end=0.05)
    assert n == o["n"]
    assert_parity(sim.conserved(), o["U"], label="advance_to")
    # already there: no further steps
    n2, t2 = sim.advance_to(0.05)
    assert n2 == 0 and t2 == 0.05
    # bounded by max_steps
    n3, t3 = sim.advance_to(1.0, max_steps=3)
    assert n3 == 3 and t3 < 1.0


def test_zchunk_invariance_bitwise(hy):
    prob, W = inputs.rayleigh_taylor(24, nz=40, amplitude=0.05)
    outs = []
    for z in (0, 1, 7, 40):
        sim = hy.Simulation(prob, W)
        sim.set_zchunk(z)
        sim.run_steps(5)
        outs.append(sim.get_state())
        sim.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_determinism_and_totals(hy, orc):
    prob, W = inputs.kelvin_helmholtz(32, ndim=3, U=1.2, ratio=2.5, precision=inputs.FP64)
    a = hy.Simulation(prob, W)
    b = hy.Simulation(prob, W)
    a.run_steps(10)
    b.run_steps(10)
    assert np.array_equal(a.get_state(), b.get_state())
    ta, tb = a.totals(), b.totals()
    assert np.array_equal(ta, tb)
    o = oracle_run(orc, prob, W, steps=10)
    T = o["U"].sum(axis=(1, 2, 3)) * np.prod(prob.dx())
    scale = np.abs(T).max()
    np.testing.assert_allclose(ta, T, rtol=0, atol=1e-12 * scale)


def test_periodic_conservation_gpu(hy):
    prob, W = inputs.kelvin_helmholtz(32, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    sim = hy.Simulation(prob, W)
    T0 = sim.totals()
    U0 = sim.conserved()
    sim.run_steps(100)
    T1 = sim.totals()
    dV = np.prod(prob.dx())
    mom_scale = np.abs(U0[1:4]).sum() * dV
    for q in range(5):
        scale = mom_scale if 1 <= q <= 3 else np.abs(U0[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


def test_reflecting_walls_conserve_mass_and_energy_gpu(hy):
    for hse in (0, 1):
        prob, W = inputs.rayleigh_taylor(16, nz=32, amplitude=0.05, hse_subtract=hse)
        sim = hy.Simulation(prob, W)
        U0 = sim.conserved()
        sim.run_steps(60)
        U1 = sim.conserved()
        phi = -prob.grav[2] * prob.centres(2)[:, None, None]
        m0, m1 = U0[0].sum(), U1[0].sum()
        e0 = (U0[4] + U0[0] * phi).sum()
        e1 = (U1[4] + U1[0] * phi).sum()
        assert abs(m1 - m0) <= 1e-13 * m0
        assert abs(e1 - e0) <= 1e-12 * abs(e0)


# ------------------------------------------------- checkpoint and faults
def test_checkpoint_restart_bitwise(hy):
    prob, W = inputs.rayleigh_taylor(16, nz=32, amplitude=0.05, hse_subtract=1)
    a = hy.Simulation(prob, W)
    a.run_steps(12)
    ref = a.get_state()
    b = hy.Simulation(prob, W)
    b.run_steps(5)
    snap, t5, s5 = b.get_state(), b.t, b.nstep
    c = hy.Simulation(prob, W)
    c.set_state(snap, t5, s5)
    c.run_steps(7)
    assert np.array_equal(c.get_state(), ref)
    assert c.nstep == 12 and c.t == a.t


def test_checkpoint_file_restart_bitwise(hy, tmp_path):
    prob, W = inputs.rayleigh_taylor(16, nz=32, amplitude=0.05, hse_subtract=1)
    a = hy.Simulation(prob, W)
    a.run_steps(12)
    ref = a.get_state()
    b = hy.Simulation(prob, W)
    b.run_steps(5)
    path = str(tmp_path / "rt.ck")
    b.save_checkpoint(path)
    c = hy.Simulation(prob, W)
    c.load_checkpoint(path)
    assert c.nstep == 5 and c.t == b.t
    c.run_steps(7)
    assert np.array_equal(c.get_state(), ref) and c.t == a.t
    # a handle of another problem, a truncated file and a flipped byte are refused
    other = hy.Simulation(prob.replace(cfl=0.7), W)
    with pytest.raises(hy.HydroError):
        other.load_checkpoint(path)
    raw = open(path, "rb").read()
    open(path + ".short", "wb").write(raw[:-8])
    bad = bytearray(raw)
    bad[-3] ^= 0x40
    open(path + ".bad", "wb").write(bytes(bad))
    for p in (path + ".short", path + ".bad", str(tmp_path / "missing.ck")):
        with pytest.raises(hy.HydroError):
            c.load_checkpoint(p)
    assert np.array_equal(c.get_state(), ref)      # unchanged by the refused loads


def test_nonphysical_state_reported(hy):
    prob, W = inputs.sod(32)
    sim = hy.Simulation(prob, W)
    sim.step()
    snap, t, s = sim.get_state(), sim.t, sim.nstep
    sim.h  # handle alive
    hy.hydro_debug_poke(sim.h, 0, 5 * 32 + 7, -1.0)     # negative density
    with pytest.raises(hy.HydroError) as ei:
        sim.step(want_dt=True)
    assert ei.value.status == hy.HYDRO_ERR_NONPHYSICAL
    with pytest.raises(hy.HydroError):
        sim.step()
    # restoring a good state clears the error
    sim.set_state(snap, t, s)
    sim.step(want_dt=True)


def test_nonphysical_initial_state_rejected(hy):
    prob, W = inputs.sod(16)
    W = W.copy()
    W[-1, 0, 3, 3] = -0.5
    with pytest.raises(hy.HydroError) as ei:
        hy.Simulation(prob, W)
    assert ei.value.status == hy.HYDRO_ERR_NONPHYSICAL


# ----------------------------------------------------------------- FP32
def test_fp32_sod_density_error(hy, orc):
    prob, W = inputs.sod(128)
    o = oracle_run(orc, prob, W, t_end=0.2)
    g = gpu_run(hy, prob.replace(precision=inputs.FP32), W, t_end=0.2)
    assert g["t"] == 0.2
    err = l1rel(g["U"][0], o["U"][0])
    assert err <= 1e-4, err


@pytest.mark.parametrize("hse", [0, 1])
def test_fp32_rayleigh_taylor_against_fp64_oracle(hy, orc, hse):
    prob, W = inputs.rayleigh_taylor(32, amplitude=0.05, hse_subtract=hse)
    o = oracle_run(orc, prob, W, steps=40)
    g = gpu_run(hy, prob.replace(precision=inputs.FP32), W, steps=40)
    err = l1rel(g["U"][0], o["U"][0])
    assert err <= 1e-5, err


def test_fp32_rt_linear_phase_density_error(hy):
    """FP32 bulk (FP64 dt, totals, background) against the FP64 run in the
    same hydrostatic mode: density L1-relative difference <= 1e-3 at t = 0.5
    (Rayleigh-Taylor 128^3, linear-growth phase)."""
    rho = {}
    for prec in (inputs.FP32, inputs.FP64):
        prob, W = inputs.rayleigh_taylor(128, precision=prec, hse_subtract=1)
        sim = hy.Simulation(prob, W)
        n, t = sim.advance_to(0.5)
        assert t == 0.5
        rho[prec] = sim.primitive()[0]
        sim.close()
    err = l1rel(rho[inputs.FP32], rho[inputs.FP64])
    assert err <= 1e-3, err


@pytest.mark.parametrize("prec,variants", [(inputs.FP64, (0, 1, 2, 4, 5, 6)), (inputs.FP32, (0, 1, 2, 3, 4, 5, 6, 7))])
def test_tile_shape_invariance_bitwise(hy, prec, variants):
    """Every tile shape the autotuner may pick gives the same bits (ragged
    sizes, reflecting walls, hydrostatic mode)."""
    prob, W = inputs.rayleigh_taylor(37, nz=45, amplitude=0.05, hse_subtract=1, precision=prec)
    prob = prob.replace(n=(37, 37, 45))
    outs = []
    for v in variants:
        sim = hy.Simulation(prob, W)
        sim.configure(v, 7)
        sim.run_steps(4)
        outs.append(sim.get_state())
        sim.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    if prec == inputs.FP64:
        sim = hy.Simulation(prob, W)
        with pytest.raises(hy.HydroError):
            sim.set_tile(3)          # the 512-thread tile is FP32 only
        sim.close()


@pytest.mark.parametrize("prec,variants", [(inputs.FP64, (0, 1, 2, 6)), (inputs.FP32, (0, 3, 5, 7))])
@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.SSPRK2], ids=["hancock", "rk2"])
def test_balanced_grid_equals_chunked_grid_bitwise(hy, prec, variants, scheme):
    """The balanced grid (negative z-chunk: whole waves of chunks, then the
    last wave's planes split evenly over every resident CTA) gives the bits of
    the chunked grid: over whole columns (-1, -45), 5-plane chunks (45 = 9 x 5)
    and 7-plane chunks (a 3-plane last row).  On 37 x 37 x 45 cells the split
    pieces are a few planes long and begin and end inside chunks."""
    prob, W = inputs.rayleigh_taylor(37, nz=45, amplitude=0.05, hse_subtract=1, precision=prec)
    prob = prob.replace(n=(37, 37, 45), scheme=scheme)
    for v in variants:
        outs = []
        for z in (7, hy.ZCHUNK_BALANCED, -5, -7, -45):
            sim = hy.Simulation(prob, W)
            sim.configure(v, z)
            sim.run_steps(4)
            outs.append((sim.get_state(), sim.t, sim.dt))
            sim.close()
        for z, o in zip((hy.ZCHUNK_BALANCED, -5, -7, -45), outs[1:]):
            assert np.array_equal(outs[0][0], o[0]), (v, z)
            assert outs[0][1] == o[1] and outs[0][2] == o[2], (v, z)


@pytest.mark.parametrize("prec,variant", [(inputs.FP64, 6), (inputs.FP64, 2), (inputs.FP32, 0), (inputs.FP32, 3)])
def test_balanced_grid_whole_waves_bitwise(hy, prec, variant):
    """A grid with more chunks than resident CTAs, so that the balanced grid
    takes whole waves of chunks before splitting the last one (128 x 128 x 64
    cells; 4- and 8-plane chunks give 16 and 8 chunks per column), gives the
    bits of the chunked grid."""
    prob, W = inputs.rayleigh_taylor(128, nz=64, amplitude=0.05, hse_subtract=1, precision=prec)
    outs = []
    # (-10**6: chunks longer than the column are whole columns)
    for z in (16, -4, -8, hy.ZCHUNK_BALANCED, -10**6):
        sim = hy.Simulation(prob, W)
        sim.configure(variant, z)
        sim.run_steps(3)
        outs.append((sim.get_state(), sim.t, sim.dt))
        sim.close()
    for z, o in zip((-4, -8, hy.ZCHUNK_BALANCED, -10**6), outs[1:]):
        assert np.array_equal(outs[0][0], o[0]), (variant, z)
        assert outs[0][1] == o[1] and outs[0][2] == o[2], (variant, z)


def test_balanced_grid_rejected_where_unsupported(hy):
    prob, W = inputs.rayleigh_taylor(16, nz=16, amplitude=0.05, precision=inputs.FP32)
    sim = hy.Simulation(prob, W)
    sim.set_tile(8)                       # paired-cell kernel: z-chunks only
    with pytest.raises(hy.HydroError):
        sim.set_zchunk(hy.ZCHUNK_BALANCED)
    sim.close()
    prob2, W2 = inputs.kelvin_helmholtz(32, ndim=2, precision=inputs.FP64)
    sim = hy.Simulation(prob2, W2)
    with pytest.raises(hy.HydroError):
        sim.set_zchunk(hy.ZCHUNK_BALANCED)
    sim.close()


@pytest.mark.parametrize("mode", ["fp64", "fp64_hse", "fp32_hse"])
def test_init_from_conserved_matches_init_from_primitives(hy, orc, mode):
    """hydro_init_conserved with the total conserved variables of an initial
    state gives the stored state hydro_init gives from its primitives (up to
    the rounding of the conversion) and the same run."""
    prec = inputs.FP32 if mode == "fp32" or mode.startswith("fp32") else inputs.FP64
    prob, W = inputs.rayleigh_taylor(20, nz=24, amplitude=0.05, hse_subtract=int("hse" in mode),
                                     precision=prec)
    o = orc.Oracle(prob.replace(precision=inputs.FP64))
    Utot = o.total(o.state_from_prim(W))          # total conserved, FP64, computed on the host
    a = hy.Simulation(prob, W)
    b = hy.Simulation(prob, Utot, conserved=True)
    Sa, Sb = a.get_state(), b.get_state()
    if prec == inputs.FP64:
        np.testing.assert_allclose(Sb, Sa, rtol=1e-13, atol=1e-13 * np.abs(Sa).max())
    else:
        # the two FP64 values round to the same float or to neighbouring floats
        np.testing.assert_allclose(Sb, Sa, rtol=2.5e-7, atol=1e-7 * np.abs(Sa).max())
    assert abs(a.dt - b.dt) <= 1e-12 * a.dt
    a.run_steps(3)
    b.run_steps(3)
    tol = TOL if prec == inputs.FP64 else 1e-5
    assert_parity(b.conserved(), a.conserved(), tol=tol, label=mode)
    a.close()
    b.close()
