"""Pins of the oracle's two integrators against textbook schemes, closed
forms and invariants, aimed at what the method-of-lines integrator (SSP-RK2,
Shu and Osher 1988) changes: no half-step predictor, the stage-wise gravity
source and the two-stage average.

* Scalar advection: with uniform velocity and pressure the Euler equations
  carry density as a passive scalar, and HLLC's flux through such a contact
  is exactly upwind.  One step of either integrator must then equal the
  textbook linear scheme written here from scratch (MC-limited piecewise
  linear reconstruction; LeVeque, "Finite Volume Methods for Hyperbolic
  Problems", ch. 6): the MUSCL-Hancock face value a_i + (1 - nu) s_i / 2,
  or two forward-Euler stages with face value a_i + s_i / 2 averaged
  Shu-Osher style.  Run along every axis, both signs of velocity.
* Sod against the exact Riemann solution and under refinement.
* Conservation; mirror and axis-rotation symmetry.
* Second order on the advected pulse, the isentropic vortex and a
  self-convergence study with gravity.
* Uniform free fall exact; total momentum grows as g M t; mass and
  E + rho phi conserved between reflecting walls.
* Hydrostatic-background mode: equal to the plain scheme for a constant
  background and on linear data, at rest for a balanced background.
"""

import math

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, SSPRK2, Problem

from test_oracle_scheme import (SOD_L, SOD_R, l1rel, potential_totals, restrict2, smooth_random_prim,
                                with_background)

THREADS = 8


def run(orc, prob, W, **kw):
    o = orc.Oracle(prob, threads=THREADS)
    U = o.state_from_prim(W)
    V, t, s, dl = o.run(U, **kw)
    return o, U, V, t, s


def rk2(prob):
    return prob.replace(scheme=SSPRK2)


# ------------------------------------------------------ scalar advection
def mc_slopes(a):
    """MC-limited cell slopes of a periodic 1D array (van Leer 1977)."""
    dl = a - np.roll(a, 1)
    dr = np.roll(a, -1) - a
    lim = np.minimum(np.minimum(2 * np.abs(dl), 2 * np.abs(dr)), 0.5 * np.abs(dl + dr))
    return np.where(dl * dr > 0, np.sign(dr) * lim, 0.0)


def advect_hancock(a, nu):
    """One step of the MUSCL-Hancock linear scheme for a_t + u a_x = 0,
    Courant number nu = u dt / dx > 0, periodic."""
    face = a + 0.5 * (1.0 - nu) * mc_slopes(a)          # value at i + 1/2
    return a - nu * (face - np.roll(face, 1))


def advect_rk2(a, nu):
    """One SSP-RK2 step of the semi-discrete upwind PLM scheme."""
    def L(b):
        face = b + 0.5 * mc_slopes(b)
        return -nu * (face - np.roll(face, 1))
    a1 = a + L(a)
    return 0.5 * (a + a1 + L(a1))


def advection_case(axis, ndim, sign, n=48):
    shape = [4, 4, 1] if ndim == 2 else [4, 4, 4]
    shape[axis] = n
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=ndim, n=tuple(shape), bc_lo=per, bc_hi=per)
    s = prob.centres(axis)
    profile = 1.0 + 0.3 * np.sin(2 * np.pi * s) + 0.25 * ((s > 0.2) & (s < 0.45))
    bshape = [1, 1, 1]
    bshape[2 - axis] = -1
    W = np.zeros(prob.shape)
    W[0] = profile.reshape(bshape)
    u = 0.7 * sign
    W[1 + axis] = u
    W[-1] = 1.0
    return prob, W, profile, abs(u)


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, SSPRK2])
@pytest.mark.parametrize("axis,ndim,sign", [(0, 2, 1), (1, 2, -1), (0, 3, -1), (1, 3, 1), (2, 3, -1)])
def test_contact_advection_equals_textbook_scheme(orc, scheme, axis, ndim, sign):
    prob, W, a, speed = advection_case(axis, ndim, sign)
    prob = prob.replace(scheme=scheme)
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    dx = prob.dx()[axis]
    nu = 0.4
    dt = nu * dx / speed
    step = advect_hancock if scheme == inputs.HANCOCK else advect_rk2
    for _ in range(12):
        U = o.step(U, dt)
        # u < 0 is the mirror image of u > 0
        a = step(a, nu) if sign > 0 else step(a[::-1], nu)[::-1]
    rho = np.moveaxis(o.prim(U)[0], 2 - axis, -1).reshape(-1, a.size)
    assert np.abs(rho - a[None, :]).max() <= 1e-13
    # the two integrators differ on this data (the pin separates them)
    b = c = advection_case(axis, ndim, 1)[2]
    for _ in range(12):
        b, c = advect_hancock(b, nu), advect_rk2(c, nu)
    assert np.abs(b - c).max() > 1e-4


# ---------------------------------------------------------------- Sod
def sod_strip(n):
    prob, W = inputs.sod(n)
    prob = prob.replace(n=(n, 4, 1), hi=(1.0, 4.0 / n, 1.0), scheme=SSPRK2)
    return prob, np.ascontiguousarray(W[:, :, :4, :])


def test_sod_rk2_against_exact_and_refinement(orc):
    errs = []
    for n in (128, 256, 512, 1024):
        prob, W = sod_strip(n)
        o, U, V, t, s = run(orc, prob, W, t_end=0.2)
        assert t == 0.2
        P = o.prim(V)
        assert (P == P[:, :, :1, :]).all() and (P[2] == 0.0).all()
        edges = np.linspace(0.0, 1.0, n + 1)
        rho_ex, _, p_ex = orc.exact_cell_average(SOD_L, SOD_R, 1.4, 0.5, 0.2, edges)
        errs.append(l1rel(P[0, 0, 0], rho_ex))
        if n == 128:
            assert errs[0] <= 1.5e-2 and l1rel(P[-1, 0, 0], p_ex) <= 1.5e-2
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (np.diff(errs) < 0).all() and order[-2:].min() >= 0.6, (errs, order)


# ------------------------------------------------ invariants, symmetry
@pytest.mark.parametrize("nd,n,steps", [(2, 64, 150), (3, 16, 100)])
def test_rk2_periodic_conservation(orc, nd, n, steps):
    prob, W = inputs.kelvin_helmholtz(n, ndim=nd, U=1.5, ratio=3.0, precision=inputs.FP64)
    o, U, V, t, s = run(orc, rk2(prob), W, max_steps=steps)
    assert s == steps
    dV = np.prod(prob.dx()[:nd])
    T0, T1 = o.totals(U), o.totals(V)
    mom_scale = np.abs(U[1:1 + nd]).sum() * dV
    for q in range(prob.nvar):
        scale = mom_scale if 1 <= q <= nd else np.abs(U[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, (q, T1[q] - T0[q], scale)


def test_rk2_mirror_symmetry(orc):
    prob = rk2(Problem(ndim=2, n=(37, 29, 1), bc_lo=(BC_OUTFLOW, BC_PERIODIC, 0),
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


def test_rk2_axis_rotation_symmetry(orc):
    per = (BC_PERIODIC,) * 3
    prob = rk2(Problem(ndim=3, n=(12, 12, 12), bc_lo=per, bc_hi=per))
    W = smooth_random_prim(prob, 5)
    W[0, :6] *= 1.3
    Wr = np.empty_like(W)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        Wr[q] = np.transpose(W[src], (2, 0, 1))
    _, _, V, _, _ = run(orc, prob, W, max_steps=30)
    _, _, Vr, _, _ = run(orc, prob, Wr, max_steps=30)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        assert l1rel(Vr[q], np.transpose(V[src], (2, 0, 1))) <= 1e-12


# ---------------------------------------------------------- convergence
def test_rk2_smooth_pulse_second_order(orc):
    errs = []
    for n in (32, 64, 128, 256):
        prob, W = inputs.smooth_pulse(n, 2)
        o, U, V, t, s = run(orc, rk2(prob), W, t_end=0.25)
        errs.append(l1rel(V[0, 0], inputs.pulse_density(prob, 0.25)[0]))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-2:].min() >= 1.7, order


def test_rk2_isentropic_vortex_second_order(orc):
    errs = []
    for n in (48, 96, 192):
        prob, W = inputs.isentropic_vortex(n)
        o, U, V, t, s = run(orc, rk2(prob), W, t_end=0.5)
        P, ex = o.prim(V), inputs.vortex_prim(prob, 0.5)
        errs.append([l1rel(P[q], ex[q]) for q in range(4)])
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() >= 1.8, order


def test_rk2_self_convergence_with_gravity(orc):
    sols = []
    for n in (32, 64, 128, 256):
        per = (BC_PERIODIC,) * 3
        prob = rk2(Problem(ndim=2, n=(n, n, 1), bc_lo=per, bc_hi=per, grav=(0.3, -1.0, 0.0)))
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
def test_rk2_uniform_free_fall_exact(orc):
    per = (BC_PERIODIC,) * 3
    prob = rk2(Problem(ndim=3, n=(6, 5, 7), bc_lo=per, bc_hi=per, grav=(0.0, 0.0, -0.7)))
    W = np.zeros(prob.shape)
    W[0], W[1], W[2], W[3], W[4] = 1.3, 0.1, -0.2, 0.05, 0.9
    o, U, V, t, s = run(orc, prob, W, max_steps=25)
    P = o.prim(V)
    np.testing.assert_allclose(P[3], 0.05 - 0.7 * t, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P[0], 1.3, rtol=1e-14)
    np.testing.assert_allclose(P[4], 0.9, rtol=1e-12)
    np.testing.assert_allclose(P[1], 0.1, rtol=1e-13)


def test_rk2_periodic_momentum_growth_g_M_t(orc):
    prob, W = inputs.kelvin_helmholtz(48, ndim=2, U=1.0, ratio=2.5, precision=inputs.FP64)
    prob = rk2(prob.replace(grav=(0.0, -0.8, 0.0)))
    o, U, V, t, s = run(orc, prob, W, max_steps=100)
    T0, T1 = o.totals(U), o.totals(V)
    assert abs(T1[0] - T0[0]) <= 1e-14 * T0[0]
    want = T0[2] + (-0.8) * T0[0] * t
    assert abs(T1[2] - want) <= 1e-13 * (abs(T0[0] * t) + 1), (T1[2], want)


@pytest.mark.parametrize("hse", [0, 1])
def test_rk2_reflecting_walls_mass_and_energy_with_potential(orc, hse):
    prob, W = inputs.rayleigh_taylor(12, nz=24, amplitude=0.05, hse_subtract=hse)
    o, U, V, t, s = run(orc, rk2(prob), W, max_steps=60)
    m0, e0 = potential_totals(o, prob, U)
    m1, e1 = potential_totals(o, prob, V)
    assert abs(m1 - m0) <= 1e-13 * m0
    assert abs(e1 - e0) <= 1e-12 * abs(e0), (e1 - e0)


# ------------------------------------------------ hydrostatic background
def test_rk2_hse_constant_background_with_gravity_equals_plain(orc):
    prob = rk2(Problem(ndim=3, n=(9, 8, 12), hi=(1.0, 1.0, 2.0),
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


def test_rk2_hse_balanced_background_stays_at_rest(orc):
    prob, _ = inputs.rayleigh_taylor(8, nz=16, perturb=False)
    prob = rk2(prob)
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


def test_rk2_hse_one_step_equals_plain_on_linear_data(orc):
    nz = 16
    prob = rk2(Problem(ndim=3, n=(5, 4, nz), hi=(1.0, 1.0, 2.0),
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
    # two stages widen the wall-influenced band to four planes
    inner = slice(4, nz - 4)
    for q in range(prob.nvar):
        a, b = Th[q, inner], T[q, inner]
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max()), q
    assert np.abs(Th[4] - T[4]).max() > 1e-10
