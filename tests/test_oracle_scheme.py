"""Pins of the whole oracle step against closed forms and invariants.

Each test fixes a property that the scheme must have whatever its rounding,
so that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them:

* Sod tube: density L1 error against the cell-averaged exact Riemann solution,
  its decrease under refinement, bitwise-identical rows and v = 0 exactly.
* conservation of mass, momentum and energy on periodic grids;
* mirror (x -> -x, u -> -u) and axis-rotation symmetry;
* second-order convergence on an advected smooth pulse (exact translate);
* free fall of a uniform gas and the exact growth of total momentum g M t;
* conservation of mass and of E + rho phi between reflecting walls (the
  energy source's summation-by-parts identity);
* the CFL time step of a uniform state (closed form);
* the hydrostatic-background mode: equal to the plain scheme for a constant
  background, exactly at rest for a discretely balanced one, second-order
  small motion in a smooth isothermal atmosphere.
"""

import math

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, Problem

THREADS = 8


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def run(orc, prob, W, **kw):
    o = orc.Oracle(prob, threads=THREADS)
    U = o.state_from_prim(W)
    V, t, s, dl = o.run(U, **kw)
    return o, U, V, t, s


# ------------------------------------------------------------------- Sod
SOD_L, SOD_R = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1]


def sod_strip(n):
    """Sod along x on n x 4 cells with square cells: each row evolves exactly
    as a row of the n x n tube (same dt, no y coupling)."""
    prob, W = inputs.sod(n)
    prob = prob.replace(n=(n, 4, 1), hi=(1.0, 4.0 / n, 1.0))
    return prob, np.ascontiguousarray(W[:, :, :4, :])


def test_sod_128_against_exact(orc):
    prob, W = inputs.sod(128)
    o, U, V, t, s = run(orc, prob, W, t_end=0.2)
    assert t == 0.2 and 80 <= s <= 140
    P = o.prim(V)
    # every row bitwise identical, transverse velocity exactly zero
    assert (P == P[:, :, :1, :]).all()
    assert (P[2] == 0.0).all()
    edges = np.linspace(0.0, 1.0, 129)
    rho_ex, u_ex, p_ex = orc.exact_cell_average(SOD_L, SOD_R, 1.4, 0.5, 0.2, edges)
    assert l1rel(P[0, 0, 0], rho_ex) <= 1.5e-2
    assert l1rel(P[-1, 0, 0], p_ex) <= 1.5e-2
    # the strip reproduces the full tube row bit for bit
    ps, Ws = sod_strip(128)
    _, _, Vs, _, _ = run(orc, ps, Ws, t_end=0.2)
    assert (Vs[:, 0, 0, :] == V[:, 0, 0, :]).all()


def test_sod_refinement(orc):
    errs = []
    for n in (128, 256, 512, 1024):
        prob, W = sod_strip(n)
        o, U, V, t, s = run(orc, prob, W, t_end=0.2)
        rho_ex, _, _ = orc.exact_cell_average(SOD_L, SOD_R, 1.4, 0.5, 0.2,
                                              np.linspace(0.0, 1.0, n + 1))
        errs.append(l1rel(o.prim(V)[0, 0, 0], rho_ex))
    errs = np.array(errs)
    assert (np.diff(errs) < 0).all()
    order = np.log2(errs[:-1] / errs[1:])
    assert order[-2:].min() >= 0.6, order


# ------------------------------------------------------- conservation
def smooth_random_prim(prob, seed, amp=0.2):
    """A smooth random primitive field built from a few periodic modes."""
    rng = np.random.default_rng(seed)
    nd = prob.ndim
    grids = np.meshgrid(*[prob.centres(d) for d in range(nd)][::-1], indexing="ij")
    grids = grids[::-1]  # grids[d] varies along axis d; arrays are [z][y][x]
    W = np.zeros(prob.shape)
    for q in range(prob.nvar):
        f = np.zeros(grids[0].shape)
        for _ in range(4):
            k = rng.integers(1, 3, nd)
            ph = rng.uniform(0, 2 * math.pi)
            f += rng.normal() * np.cos(2 * math.pi * sum(k[d] * grids[d] for d in range(nd)) + ph)
        W[q] = f.reshape(W[q].shape)
    W[0] = 1.0 + amp * W[0] / np.abs(W[0]).max()
    W[-1] = 1.0 + amp * W[-1] / np.abs(W[-1]).max()
    for d in range(nd):
        W[1 + d] = 0.5 * W[1 + d] / np.abs(W[1 + d]).max()
    return W


@pytest.mark.parametrize("nd,n,steps", [(2, 64, 200), (3, 16, 200)])
def test_periodic_conservation(orc, nd, n, steps):
    prob, W = inputs.kelvin_helmholtz(n, ndim=nd, U=1.5, ratio=3.0, precision=inputs.FP64)
    o, U, V, t, s = run(orc, prob, W, max_steps=steps)
    assert s == steps
    dV = np.prod(prob.dx()[:nd])
    T0, T1 = o.totals(U), o.totals(V)
    mom_scale = np.abs(U[1:1 + nd]).sum() * dV    # a momentum total may start at 0
    for q in range(prob.nvar):
        scale = mom_scale if 1 <= q <= nd else np.abs(U[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, (q, T1[q] - T0[q], scale)


# ------------------------------------------------------------ symmetry
def test_mirror_symmetry(orc):
    prob = Problem(ndim=2, n=(37, 29, 1), bc_lo=(BC_OUTFLOW, BC_PERIODIC, 0),
                   bc_hi=(BC_REFLECT, BC_PERIODIC, 0), grav=(0.0, -0.5, 0.0))
    W = smooth_random_prim(prob, 11)
    W[0, :, :, :18] *= 1.5          # add a jump so limiters are active
    mprob = prob.replace(bc_lo=(BC_REFLECT, BC_PERIODIC, 0), bc_hi=(BC_OUTFLOW, BC_PERIODIC, 0))
    Wm = W[:, :, :, ::-1].copy()
    Wm[1] *= -1
    _, _, V, _, _ = run(orc, prob, W, max_steps=40)
    _, _, Vm, _, _ = run(orc, mprob, Wm, max_steps=40)
    back = Vm[:, :, :, ::-1].copy()
    back[1] *= -1
    for q in range(prob.nvar):
        assert l1rel(back[q], V[q]) <= 1e-12


def test_axis_rotation_symmetry(orc):
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=3, n=(12, 12, 12), bc_lo=per, bc_hi=per)
    W = smooth_random_prim(prob, 5)
    W[0, :6] *= 1.3
    # rotate axes: new x = old y, new y = old z, new z = old x
    Wr = np.empty_like(W)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        Wr[q] = np.transpose(W[src], (2, 0, 1))
    _, _, V, _, _ = run(orc, prob, W, max_steps=30)
    _, _, Vr, _, _ = run(orc, prob, Wr, max_steps=30)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        assert l1rel(Vr[q], np.transpose(V[src], (2, 0, 1))) <= 1e-12


# --------------------------------------------------------- convergence
def test_smooth_pulse_second_order(orc):
    errs = []
    for n in (32, 64, 128, 256):
        prob, W = inputs.smooth_pulse(n, 2)
        o, U, V, t, s = run(orc, prob, W, t_end=0.25)
        errs.append(l1rel(V[0, 0], inputs.pulse_density(prob, 0.25)[0]))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-2:].min() >= 1.7, order


def test_smooth_pulse_second_order_3d(orc):
    errs = []
    for n in (16, 32, 48):
        prob, W = inputs.smooth_pulse(n, 3)
        o, U, V, t, s = run(orc, prob, W, t_end=0.1)
        errs.append(l1rel(V[0], inputs.pulse_density(prob, 0.1)))
    order = math.log(errs[1] / errs[2]) / math.log(48 / 32)
    assert order >= 1.7, (errs, order)


# -------------------------------------------------------------- gravity
def test_uniform_free_fall_exact(orc):
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=3, n=(6, 5, 7), bc_lo=per, bc_hi=per, grav=(0.0, 0.0, -0.7))
    W = np.zeros(prob.shape)
    W[0], W[1], W[2], W[3], W[4] = 1.3, 0.1, -0.2, 0.05, 0.9
    o, U, V, t, s = run(orc, prob, W, max_steps=25)
    P = o.prim(V)
    np.testing.assert_allclose(P[3], 0.05 - 0.7 * t, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P[0], 1.3, rtol=1e-14)
    np.testing.assert_allclose(P[4], 0.9, rtol=1e-12)
    np.testing.assert_allclose(P[1], 0.1, rtol=1e-13)


def test_periodic_momentum_growth_g_M_t(orc):
    prob, W = inputs.kelvin_helmholtz(48, ndim=2, U=1.0, ratio=2.5, precision=inputs.FP64)
    prob = prob.replace(grav=(0.0, -0.8, 0.0))
    o, U, V, t, s = run(orc, prob, W, max_steps=100)
    T0, T1 = o.totals(U), o.totals(V)
    assert abs(T1[0] - T0[0]) <= 1e-14 * T0[0]
    want = T0[2] + (-0.8) * T0[0] * t
    assert abs(T1[2] - want) <= 1e-13 * (abs(T0[0] * t) + 1), (T1[2], want)
    assert abs(T1[1] - T0[1]) <= 1e-13 * np.abs(U[1]).sum() * np.prod(prob.dx()[:2])


def potential_totals(o, prob, V):
    """(mass, E + rho phi) with phi = -g.x at cell centres."""
    T = o.total(V)
    dV = np.prod(prob.dx()[:prob.ndim])
    z = prob.centres(2)
    phi = -prob.grav[2] * z
    return T[0].sum() * dV, (T[4] + T[0] * phi[:, None, None]).sum() * dV


@pytest.mark.parametrize("hse", [0, 1])
def test_reflecting_walls_mass_and_energy_with_potential(orc, hse):
    prob, W = inputs.rayleigh_taylor(12, nz=24, amplitude=0.05, hse_subtract=hse)
    o, U, V, t, s = run(orc, prob, W, max_steps=60)
    m0, e0 = potential_totals(o, prob, U)
    m1, e1 = potential_totals(o, prob, V)
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(e1 - e0) <= 1e-12 * abs(e0), (e1 - e0)


def test_cfl_dt_uniform_closed_form(orc):
    prob = Problem(ndim=3, n=(8, 4, 6), hi=(1.0, 2.0, 0.5))
    W = np.zeros(prob.shape)
    W[0], W[1], W[2], W[3], W[4] = 2.0, 0.3, -0.4, 0.1, 1.5
    o = orc.Oracle(prob)
    c = math.sqrt(1.4 * 1.5 / 2.0)
    dx = prob.dx()
    s = sum((abs(u) + c) / h for u, h in zip((0.3, -0.4, 0.1), dx))
    assert abs(o.cfl_dt(o.state_from_prim(W)) - 0.8 / s) <= 1e-15 * (0.8 / s)


# ------------------------------------------------ hydrostatic background
def with_background(prob, rho_c, p_c, rho_f, p_f):
    return prob.replace(hse_subtract=1, bg_rho_c=np.asarray(rho_c, float),
                        bg_p_c=np.asarray(p_c, float), bg_rho_f=np.asarray(rho_f, float),
                        bg_p_f=np.asarray(p_f, float))


def test_hse_constant_background_equals_plain(orc):
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=3, n=(10, 9, 11), bc_lo=(BC_PERIODIC, BC_OUTFLOW, BC_REFLECT),
                   bc_hi=(BC_PERIODIC, BC_REFLECT, BC_REFLECT))
    W = smooth_random_prim(prob, 3)
    nz = prob.n[2]
    hp = with_background(prob, np.full(nz + 4, 0.7), np.full(nz + 4, 0.9),
                         np.full(nz + 5, 0.7), np.full(nz + 5, 0.9))
    o, U, V, t, s = run(orc, prob, W, max_steps=30)
    oh, Uh, Vh, th, sh = run(orc, hp, W, max_steps=30)
    T, Th = o.total(V), oh.total(Vh)
    for q in range(prob.nvar):
        assert l1rel(Th[q], T[q]) <= 1e-12


def test_hse_balanced_background_stays_at_rest(orc):
    prob, _ = inputs.rayleigh_taylor(8, nz=16, perturb=False)
    nz, dz, g = prob.n[2], prob.dx()[2], -1.0
    zc = (np.arange(-2, nz + 2) + 0.5) * dz
    zf = np.arange(-2, nz + 3) * dz
    # constant density with linear pressure: dp/dz = rho g holds exactly on
    # the discrete faces, so the discrete imbalance B_k vanishes
    hp = with_background(prob, np.ones(nz + 4), 3.0 + g * zc, np.ones(nz + 5), 3.0 + g * zf)
    W = np.zeros(prob.shape)
    W[0] = 1.0
    W[4] = (3.0 + g * prob.centres(2))[:, None, None]
    oh, Uh, Vh, _, _ = run(orc, hp, W, max_steps=40)
    assert np.abs(Vh[1:4]).max() <= 1e-13
    # the plain scheme moves at the walls on the same data (sanity of the test)
    o, U, V, _, _ = run(orc, prob, W, max_steps=40)
    assert np.abs(V[3]).max() > 1e-6


def test_hse_isothermal_atmosphere_second_order(orc):
    """rho0 = p0 = exp(-z) under g = -1: motion stays at the truncation level
    and falls at second order with resolution."""
    amax = []
    for nz in (16, 32, 64):
        prob = Problem(ndim=3, n=(4, 4, nz), hi=(1.0, 1.0, 2.0),
                       bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                       bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -1.0))
        dz = prob.dx()[2]
        zc = (np.arange(-2, nz + 2) + 0.5) * dz
        zf = np.arange(-2, nz + 3) * dz
        hp = with_background(prob, np.exp(-zc), np.exp(-zc), np.exp(-zf), np.exp(-zf))
        W = np.zeros(prob.shape)
        W[0] = np.exp(-prob.centres(2))[:, None, None]
        W[4] = W[0]
        oh, Uh, Vh, t, s = run(orc, hp, W, t_end=0.2)
        amax.append(np.abs(Vh[3]).max())
    order = np.log2(np.array(amax[:-1]) / np.array(amax[1:]))
    assert amax[-1] < 1e-4 and order.min() >= 1.8, (amax, order)


# ------------------------------------------- pins aimed at the predictor
def test_isentropic_vortex_second_order(orc):
    """Exact translate of the isentropic vortex: velocity and pressure vary,
    so every term of the half-step predictor (including the transverse
    advection terms) enters."""
    errs = []
    for n in (48, 96, 192):
        prob, W = inputs.isentropic_vortex(n)
        o, U, V, t, s = run(orc, prob, W, t_end=0.5)
        P, ex = o.prim(V), inputs.vortex_prim(prob, 0.5)
        errs.append([l1rel(P[q], ex[q]) for q in range(4)])
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() >= 1.8, order


def restrict2(a):
    """Average 2x2 blocks of a [.., ny, nx] array."""
    return 0.25 * (a[..., ::2, ::2] + a[..., 1::2, ::2] + a[..., ::2, 1::2] + a[..., 1::2, 1::2])


def test_self_convergence_with_gravity(orc):
    """Smooth compressive periodic flow under constant gravity: successive
    resolutions approach each other at second order (time-centred gravity
    source, the rho div u term of the predictor)."""
    sols = []
    for n in (32, 64, 128, 256):
        per = (BC_PERIODIC,) * 3
        prob = Problem(ndim=2, n=(n, n, 1), bc_lo=per, bc_hi=per, grav=(0.3, -1.0, 0.0))
        x, y = prob.centres(0), prob.centres(1)
        X, Y = np.meshgrid(x, y)
        W = np.zeros(prob.shape)
        W[0, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        W[1, 0] = 0.2 * np.cos(2 * np.pi * X) + 0.1 * np.cos(2 * np.pi * Y)
        W[2, 0] = 0.1 * np.sin(2 * np.pi * Y) - 0.1 * np.sin(2 * np.pi * X)
        W[3, 0] = 2.0 + 0.2 * np.cos(2 * np.pi * (X + Y))
        o, U, V, t, s = run(orc, prob, W, t_end=0.15)
        sols.append(o.total(V)[:, 0])
    d = np.array([[np.abs(restrict2(sols[i + 1][q]) - sols[i][q]).sum() / np.abs(sols[i][q]).sum()
                   for q in range(4)] for i in range(3)])
    order = np.log2(d[:-1] / d[1:])          # per pair of resolutions, per variable
    assert order.min() >= 1.8, (d, order)


def test_reflecting_wall_equals_mirrored_periodic(orc):
    """A reflecting wall is a symmetry plane: [0, 1] between walls evolves as
    the right half of mirror-symmetric data on the periodic [-1, 1]."""
    n = 24
    walls = Problem(ndim=2, n=(n, 20, 1), bc_lo=(BC_REFLECT, BC_PERIODIC, 0),
                    bc_hi=(BC_REFLECT, BC_PERIODIC, 0), grav=(0.0, -0.6, 0.0))
    W = smooth_random_prim(walls, 21)
    W[0, :, 5:9, :10] *= 1.4
    doubled = walls.replace(n=(2 * n, 20, 1), lo=(-1.0, 0.0, 0.0),
                            bc_lo=(BC_PERIODIC,) * 3, bc_hi=(BC_PERIODIC,) * 3)
    Wd = np.concatenate([W[:, :, :, ::-1], W], axis=3)
    Wd[1, :, :, :n] *= -1
    _, _, V, _, _ = run(orc, walls, W, max_steps=40)
    _, _, Vd, _, _ = run(orc, doubled, Wd, max_steps=40)
    for q in range(walls.nvar):
        assert l1rel(Vd[q, :, :, n:], V[q]) <= 1e-12


def test_hse_constant_background_with_gravity_equals_plain(orc):
    """A constant background out of balance under gravity: its imbalance B_k
    = -rho0 g must reproduce the full gravity force exactly."""
    prob = Problem(ndim=3, n=(9, 8, 12), hi=(1.0, 1.0, 2.0),
                   bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                   bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -0.9))
    W = smooth_random_prim(prob, 8)
    nz = prob.n[2]
    hp = with_background(prob, np.full(nz + 4, 0.8), np.full(nz + 4, 0.6),
                         np.full(nz + 5, 0.8), np.full(nz + 5, 0.6))
    o, U, V, t, s = run(orc, prob, W, max_steps=30)
    oh, Uh, Vh, th, sh = run(orc, hp, W, max_steps=30)
    T, Th = o.total(V), oh.total(Vh)
    for q in range(prob.nvar):
        assert l1rel(Th[q], T[q]) <= 1e-12


def test_hse_one_step_equals_plain_on_linear_data(orc):
    """For data linear in z with uniform velocity the MC slopes are central
    differences, so reconstructing perturbations from a linear background and
    adding the background back at faces is algebraically the plain scheme:
    one step agrees to rounding in every cell whose stencil avoids the walls.
    This fixes the background face values, the background terms of the
    predictor and the imbalance source B_k."""
    nz = 16
    prob = Problem(ndim=3, n=(5, 4, nz), hi=(1.0, 1.0, 2.0),
                   bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                   bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -0.7))
    dz = prob.dx()[2]
    zc = (np.arange(-2, nz + 2) + 0.5) * dz
    zf = np.arange(-2, nz + 3) * dz
    hp = with_background(prob, 1.0 + 0.3 * zc, 2.0 - 0.5 * zc, 1.0 + 0.3 * zf, 2.0 - 0.5 * zf)
    z = prob.centres(2)
    W = np.zeros(prob.shape)
    W[0] = (1.2 + 0.1 * z)[:, None, None]
    W[1], W[2], W[3] = 0.1, -0.2, 0.15
    W[4] = (2.1 - 0.4 * z)[:, None, None]
    o, oh = orc.Oracle(prob), orc.Oracle(hp)
    U, Uh = o.state_from_prim(W), oh.state_from_prim(W)
    dt = 0.5 * o.cfl_dt(U)
    T = o.total(o.step(U, dt))
    Th = oh.total(oh.step(Uh, dt))
    inner = slice(2, nz - 2)
    for q in range(prob.nvar):
        a, b = Th[q, inner], T[q, inner]
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max()), q
    # the wall cells differ (ghost data are not linear), so the test has teeth
    assert np.abs(Th[4] - T[4]).max() > 1e-10


def test_hse_and_plain_converge_together(orc):
    """Both forms are second-order schemes for the same equations: their
    difference on a smooth stratified flow falls at second order."""
    diffs = []
    for n in (16, 32, 64):
        prob = Problem(ndim=3, n=(n, 4, n), hi=(1.0, 4.0 / n, 2.0),
                       bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                       bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -1.0))
        dz = prob.dx()[2]
        zc = (np.arange(-2, n + 2) + 0.5) * dz
        zf = np.arange(-2, n + 3) * dz
        hp = with_background(prob, np.exp(-zc), np.exp(-zc), np.exp(-zf), np.exp(-zf))
        x, z = prob.centres(0), prob.centres(2)
        W = np.zeros(prob.shape)
        W[0] = np.exp(-z)[:, None, None] * (1.0 + 0.05 * np.cos(2 * np.pi * x))[None, None, :]
        W[3] = (0.05 * np.sin(np.pi * z / 2.0))[:, None, None] * np.sin(2 * np.pi * x)[None, None, :]
        W[4] = np.exp(-z)[:, None, None]
        o, U, V, t, s = run(orc, prob, W, t_end=0.3)
        oh, Uh, Vh, th, sh = run(orc, hp, W, t_end=0.3)
        T, Th = o.total(V), oh.total(Vh)
        diffs.append(max(l1rel(Th[q], T[q]) for q in (0, 4)) + np.abs(Th[3] - T[3]).mean())
    order = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    assert order.min() >= 1.7, (diffs, order)
