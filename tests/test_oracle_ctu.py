"""Pins of the oracle's corner transport upwind integrator (Colella 1990):
one-dimensional predictors per axis, first-pass fluxes, transverse
corrections of the face states, final fluxes.

* Scalar advection: with uniform velocity and pressure the density follows
  the textbook linear CTU scheme written here from scratch (upwind
  one-dimensional face values a + (1 - nu_d) s_d / 2, corrected by
  -nu_e/2 times the upwind face-value difference across every other axis
  e), in 2D and 3D with every sign pattern of the velocity; the transverse
  terms make it differ from both other integrators.
* Sod against the exact solution and under refinement; conservation;
  mirror and axis-rotation symmetry; second order on the pulse, the
  isentropic vortex and a self-convergence study with gravity; uniform free
  fall exact; total momentum grows as g M t; mass and E + rho phi conserved
  between reflecting walls.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, CTU, Problem

from test_oracle_rk2 import mc_slopes
from test_oracle_scheme import (SOD_L, SOD_R, l1rel, potential_totals, restrict2, smooth_random_prim,
                                with_background)

THREADS = 8


def ctu(prob):
    return prob.replace(scheme=CTU)


def run(orc, prob, W, **kw):
    o = orc.Oracle(prob, threads=THREADS)
    U = o.state_from_prim(W)
    V, t, s, dl = o.run(U, **kw)
    return o, U, V, t, s


# ------------------------------------------------------ scalar advection
def mc_slopes_axis(a, ax):
    return np.moveaxis(mc_slopes_nd(np.moveaxis(a, ax, -1)), -1, ax)


def mc_slopes_nd(a):
    dl = a - np.roll(a, 1, axis=-1)
    dr = np.roll(a, -1, axis=-1) - a
    lim = np.minimum(np.minimum(2 * np.abs(dl), 2 * np.abs(dr)), 0.5 * np.abs(dl + dr))
    return np.where(dl * dr > 0, np.sign(dr) * lim, 0.0)


def advect_ctu(a, nus):
    """One step of the linear CTU scheme for a_t + sum_d v_d a_{x_d} = 0 with
    every v_d > 0 on a periodic array; nus[d] = v_d dt / dx_d for array axis d."""
    nd = a.ndim
    # upwind one-dimensional face value at the high face of each cell
    face = [a + 0.5 * (1.0 - nus[d]) * mc_slopes_axis(a, d) for d in range(nd)]
    flux = []
    for d in range(nd):
        corr = face[d].copy()
        for e in range(nd):
            if e != d:
                corr -= 0.5 * nus[e] * (face[e] - np.roll(face[e], 1, axis=e))
        flux.append(corr)
    out = a.copy()
    for d in range(nd):
        out -= nus[d] * (flux[d] - np.roll(flux[d], 1, axis=d))
    return out


CASES = [((1, 1), 2), ((1, -1), 2), ((-1, 1), 2), ((1, 1, 1), 3), ((-1, 1, -1), 3), ((1, -1, 1), 3)]


@pytest.mark.parametrize("signs,ndim", CASES)
def test_ctu_contact_advection_equals_textbook_scheme(orc, signs, ndim):
    n = (24, 20, 1) if ndim == 2 else (14, 12, 10)
    per = (BC_PERIODIC,) * 3
    prob = ctu(Problem(ndim=ndim, n=n, hi=(1.0, 1.0, 1.0), bc_lo=per, bc_hi=per))
    speeds = [0.6, 0.45, 0.5][:ndim]
    W = np.zeros(prob.shape)
    grids = np.meshgrid(*[prob.centres(d) for d in range(ndim)][::-1], indexing="ij")[::-1]
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * grids[0]) * np.cos(2 * np.pi * grids[1])
    rho = rho + 0.2 * ((grids[0] > 0.3) & (grids[0] < 0.6) & (grids[1] > 0.2) & (grids[1] < 0.5))
    if ndim == 3:
        rho = rho * (1.0 + 0.2 * np.sin(2 * np.pi * grids[2]))
    W[0] = rho.reshape(prob.shape[1:])
    for d in range(ndim):
        W[1 + d] = signs[d] * speeds[d]
    W[-1] = 1.0
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    dx = prob.dx()
    dt = 0.8 / sum(speeds[d] / dx[d] for d in range(ndim)) * 0.5
    nus_axis = [speeds[d] * dt / dx[d] for d in range(ndim)]
    # numpy array axes run (z, y, x): array axis k is physical axis ndim-1-k
    a = W[0].reshape(prob.shape[1:][3 - ndim:]).copy()
    flip = tuple(k for k in range(ndim) if signs[ndim - 1 - k] < 0)
    nus = [nus_axis[ndim - 1 - k] for k in range(ndim)]
    b = np.flip(a, axis=flip) if flip else a
    for _ in range(10):
        U = o.step(U, dt)
        b = advect_ctu(b, nus)
    a = np.flip(b, axis=flip) if flip else b
    got = o.prim(U)[0].reshape(a.shape)
    assert np.abs(got - a).max() <= 1e-13
    # the transverse terms matter: dropping them changes the answer
    c = np.flip(W[0].reshape(a.shape), axis=flip) if flip else W[0].reshape(a.shape).copy()
    for _ in range(10):
        faces = [c + 0.5 * (1.0 - nus[d]) * mc_slopes_axis(c, d) for d in range(ndim)]
        c = c - sum(nus[d] * (faces[d] - np.roll(faces[d], 1, axis=d)) for d in range(ndim))
    assert np.abs(c - b).max() > 1e-4


# ------------------------------------------------------------------ Sod
def test_ctu_sod_against_exact_and_refinement(orc):
    errs = []
    for n in (128, 256, 512, 1024):
        prob, W = inputs.sod(n)
        prob = ctu(prob.replace(n=(n, 4, 1), hi=(1.0, 4.0 / n, 1.0)))
        W = np.ascontiguousarray(W[:, :, :4, :])
        o, U, V, t, s = run(orc, prob, W, t_end=0.2)
        P = o.prim(V)
        assert t == 0.2 and (P == P[:, :, :1, :]).all() and (P[2] == 0.0).all()
        rho_ex, _, p_ex = orc.exact_cell_average(SOD_L, SOD_R, 1.4, 0.5, 0.2, np.linspace(0, 1, n + 1))
        errs.append(l1rel(P[0, 0, 0], rho_ex))
        if n == 128:
            assert errs[0] <= 1.5e-2 and l1rel(P[-1, 0, 0], p_ex) <= 1.5e-2
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (np.diff(errs) < 0).all() and order[-2:].min() >= 0.6, (errs, order)


# --------------------------------------------------- invariants, symmetry
@pytest.mark.parametrize("nd,n,steps", [(2, 64, 150), (3, 16, 100)])
def test_ctu_periodic_conservation(orc, nd, n, steps):
    prob, W = inputs.kelvin_helmholtz(n, ndim=nd, U=1.5, ratio=3.0, precision=inputs.FP64)
    o, U, V, t, s = run(orc, ctu(prob), W, max_steps=steps)
    assert s == steps
    dV = np.prod(prob.dx()[:nd])
    T0, T1 = o.totals(U), o.totals(V)
    mom_scale = np.abs(U[1:1 + nd]).sum() * dV
    for q in range(prob.nvar):
        scale = mom_scale if 1 <= q <= nd else np.abs(U[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


def test_ctu_mirror_and_rotation_symmetry(orc):
    prob = ctu(Problem(ndim=2, n=(37, 29, 1), bc_lo=(BC_OUTFLOW, BC_PERIODIC, 0),
                       bc_hi=(BC_REFLECT, BC_PERIODIC, 0), grav=(0.0, -0.5, 0.0)))
    W = smooth_random_prim(prob, 11)
    W[0, :, :, :18] *= 1.5
    mprob = prob.replace(bc_lo=(BC_REFLECT, BC_PERIODIC, 0), bc_hi=(BC_OUTFLOW, BC_PERIODIC, 0))
    Wm = W[:, :, :, ::-1].copy()
    Wm[1] *= -1
    _, _, V, _, _ = run(orc, prob, W, max_steps=40)
    _, _, Vm, _, _ = run(orc, mprob, Wm, max_steps=40)
    back = Vm[:, :, :, ::-1].copy()
    back[1] *= -1
    for q in range(prob.nvar):
        assert l1rel(back[q], V[q]) <= 1e-12
    per = (BC_PERIODIC,) * 3
    p3 = ctu(Problem(ndim=3, n=(12, 12, 12), bc_lo=per, bc_hi=per))
    W3 = smooth_random_prim(p3, 5)
    W3[0, :6] *= 1.3
    Wr = np.empty_like(W3)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        Wr[q] = np.transpose(W3[src], (2, 0, 1))
    _, _, V3, _, _ = run(orc, p3, W3, max_steps=30)
    _, _, Vr, _, _ = run(orc, p3, Wr, max_steps=30)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        assert l1rel(Vr[q], np.transpose(V3[src], (2, 0, 1))) <= 1e-12


# ---------------------------------------------------------- convergence
def test_ctu_smooth_pulse_second_order(orc):
    errs = []
    for n in (32, 64, 128, 256):
        prob, W = inputs.smooth_pulse(n, 2)
        o, U, V, t, s = run(orc, ctu(prob), W, t_end=0.25)
        errs.append(l1rel(V[0, 0], inputs.pulse_density(prob, 0.25)[0]))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-2:].min() >= 1.7, order


def test_ctu_isentropic_vortex_second_order(orc):
    errs = []
    for n in (48, 96, 192):
        prob, W = inputs.isentropic_vortex(n)
        o, U, V, t, s = run(orc, ctu(prob), W, t_end=0.5)
        P, ex = o.prim(V), inputs.vortex_prim(prob, 0.5)
        errs.append([l1rel(P[q], ex[q]) for q in range(4)])
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() >= 1.8, order


def test_ctu_self_convergence_with_gravity(orc):
    sols = []
    for n in (32, 64, 128, 256):
        per = (BC_PERIODIC,) * 3
        prob = ctu(Problem(ndim=2, n=(n, n, 1), bc_lo=per, bc_hi=per, grav=(0.3, -1.0, 0.0)))
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
    order = np.log2(d[:-1] / d[1:])
    assert order.min() >= 1.8, (d, order)


# -------------------------------------------------------------- gravity
def test_ctu_uniform_free_fall_exact(orc):
    per = (BC_PERIODIC,) * 3
    prob = ctu(Problem(ndim=3, n=(6, 5, 7), bc_lo=per, bc_hi=per, grav=(0.0, 0.0, -0.7)))
    W = np.zeros(prob.shape)
    W[0], W[1], W[2], W[3], W[4] = 1.3, 0.1, -0.2, 0.05, 0.9
    o, U, V, t, s = run(orc, prob, W, max_steps=25)
    P = o.prim(V)
    np.testing.assert_allclose(P[3], 0.05 - 0.7 * t, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P[0], 1.3, rtol=1e-14)
    np.testing.assert_allclose(P[4], 0.9, rtol=1e-12)


def test_ctu_periodic_momentum_growth_g_M_t(orc):
    prob, W = inputs.kelvin_helmholtz(48, ndim=2, U=1.0, ratio=2.5, precision=inputs.FP64)
    prob = ctu(prob.replace(grav=(0.0, -0.8, 0.0)))
    o, U, V, t, s = run(orc, prob, W, max_steps=100)
    T0, T1 = o.totals(U), o.totals(V)
    assert abs(T1[0] - T0[0]) <= 1e-14 * T0[0]
    want = T0[2] + (-0.8) * T0[0] * t
    assert abs(T1[2] - want) <= 1e-13 * (abs(T0[0] * t) + 1), (T1[2], want)


def test_ctu_reflecting_walls_mass_and_energy_with_potential(orc):
    prob, W = inputs.rayleigh_taylor(12, nz=24, amplitude=0.05)
    o, U, V, t, s = run(orc, ctu(prob), W, max_steps=60)
    m0, e0 = potential_totals(o, prob, U)
    m1, e1 = potential_totals(o, prob, V)
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(e1 - e0) <= 1e-12 * abs(e0), (e1 - e0)


# ------------------------------------------------ hydrostatic background
def test_ctu_hse_constant_background_with_gravity_equals_plain(orc):
    """A constant background out of balance: its imbalance B_k = -rho0 g
    must reproduce the full gravity force in the predictors, the transverse
    corrections and the update."""
    prob = ctu(Problem(ndim=3, n=(9, 8, 12), hi=(1.0, 1.0, 2.0),
                       bc_lo=(BC_PERIODIC, BC_OUTFLOW, BC_REFLECT),
                       bc_hi=(BC_PERIODIC, BC_REFLECT, BC_REFLECT), grav=(0.0, 0.0, -0.9)))
    W = smooth_random_prim(prob, 8)
    nz = prob.n[2]
    hp = with_background(prob, np.full(nz + 4, 0.8), np.full(nz + 4, 0.6),
                         np.full(nz + 5, 0.8), np.full(nz + 5, 0.6))
    o, U, V, t, s = run(orc, prob, W, max_steps=30)
    oh, Uh, Vh, th, sh = run(orc, hp, W, max_steps=30)
    T, Th = o.total(V), oh.total(Vh)
    for q in range(prob.nvar):
        assert l1rel(Th[q], T[q]) <= 1e-12


def test_ctu_hse_balanced_background_stays_at_rest(orc):
    prob, _ = inputs.rayleigh_taylor(8, nz=16, perturb=False)
    prob = ctu(prob)
    nz, dz, g = prob.n[2], prob.dx()[2], -1.0
    zc = (np.arange(-2, nz + 2) + 0.5) * dz
    zf = np.arange(-2, nz + 3) * dz
    hp = with_background(prob, np.ones(nz + 4), 3.0 + g * zc, np.ones(nz + 5), 3.0 + g * zf)
    W = np.zeros(prob.shape)
    W[0] = 1.0
    W[4] = (3.0 + g * prob.centres(2))[:, None, None]
    oh, Uh, Vh, _, _ = run(orc, hp, W, max_steps=40)
    assert np.abs(Vh[1:4]).max() <= 1e-13
    o, U, V, _, _ = run(orc, prob, W, max_steps=40)
    assert np.abs(V[3]).max() > 1e-6


def test_ctu_hse_one_step_equals_plain_on_linear_data(orc):
    nz = 16
    prob = ctu(Problem(ndim=3, n=(5, 4, nz), hi=(1.0, 1.0, 2.0),
                       bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                       bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -0.7)))
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
    inner = slice(3, nz - 3)
    for q in range(prob.nvar):
        a, b = Th[q, inner], T[q, inner]
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max()), q
    assert np.abs(Th[4] - T[4]).max() > 1e-10


def test_ctu_hse_one_step_equals_plain_with_shear(orc):
    """Density and pressure linear in z, velocities varying across x and y:
    the transverse corrections of z-face states then change velocities, and
    their conversions see the background at the face."""
    nz = 16
    prob = ctu(Problem(ndim=3, n=(12, 10, nz), hi=(1.0, 1.0, 2.0),
                       bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                       bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -0.7)))
    dz = prob.dx()[2]
    zc = (np.arange(-2, nz + 2) + 0.5) * dz
    zf = np.arange(-2, nz + 3) * dz
    hp = with_background(prob, 1.0 + 0.3 * zc, 2.0 - 0.5 * zc, 1.0 + 0.3 * zf, 2.0 - 0.5 * zf)
    x, y, z = prob.centres(0), prob.centres(1), prob.centres(2)
    W = np.zeros(prob.shape)
    W[0] = (1.2 + 0.1 * z)[:, None, None]
    W[1] = (0.1 + 0.2 * np.sin(2 * np.pi * y))[None, :, None]
    W[2] = (-0.2 + 0.2 * np.cos(2 * np.pi * x))[None, None, :]
    W[3] = 0.15 + 0.1 * np.sin(2 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * y)[None, :, None]
    W[4] = (2.1 - 0.4 * z)[:, None, None]
    o, oh = orc.Oracle(prob), orc.Oracle(hp)
    U, Uh = o.state_from_prim(W), oh.state_from_prim(W)
    dt = 0.5 * o.cfl_dt(U)
    T = o.total(o.step(U, dt))
    Th = oh.total(oh.step(Uh, dt))
    inner = slice(3, nz - 3)
    for q in range(prob.nvar):
        a, b = Th[q, inner], T[q, inner]
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max()), q


def test_ctu_hse_reflecting_walls_mass_and_energy_with_potential(orc):
    prob, W = inputs.rayleigh_taylor(12, nz=24, amplitude=0.05, hse_subtract=1)
    o, U, V, t, s = run(orc, ctu(prob), W, max_steps=60)
    m0, e0 = potential_totals(o, prob, U)
    m1, e1 = potential_totals(o, prob, V)
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(e1 - e0) <= 1e-12 * abs(e0), (e1 - e0)


def test_ctu_rejected_combinations(orc):
    ps, Ws = inputs.sod(16)
    with pytest.raises(ValueError):
        orc.Oracle(ctu(ps).replace(recon=inputs.PPM)).state_from_prim(Ws)
