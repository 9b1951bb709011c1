"""Pins of the oracle's piecewise parabolic reconstruction (Colella and
Woodward 1984) used as the method of lines' face states.

* The interface value equals the fourth-order formula
  7/12 (a_i + a_{i+1}) - 1/12 (a_{i-1} + a_{i+2}) where the MC slopes are the
  unlimited central differences, and reproduces linear data exactly.
* The limited parabola has the properties the method guarantees, checked on
  random stencils: its mean is the cell value, it is monotone between its
  face values, a cell at a local extremum is flat, and every face value lies
  between the cell and its face neighbour.
* Scalar advection: the Euler oracle carries density like a textbook
  PPM/SSP-RK2 linear scheme written here from scratch (every axis, both
  signs), and a step profile keeps its bounds (no new extrema).
* Sod against the exact solution; conservation; mirror and rotation
  symmetry; second order on the pulse with a smaller error than PLM.
"""

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT, PPM, SSPRK2, Problem

from test_oracle_rk2 import advection_case, mc_slopes
from test_oracle_scheme import SOD_L, SOD_R, l1rel, smooth_random_prim

THREADS = 8


def ppm(prob):
    return prob.replace(scheme=SSPRK2, recon=PPM)


def run(orc, prob, W, **kw):
    o = orc.Oracle(prob, threads=THREADS)
    U = o.state_from_prim(W)
    V, t, s, dl = o.run(U, **kw)
    return o, U, V, t, s


# ------------------------------------------------------------ one cell
def faces_of(orc, a5):
    """PPM faces of the middle cell of five values (slopes from MC)."""
    s = [orc.mc_slope(a5[k] - a5[k - 1], a5[k + 1] - a5[k]) for k in (1, 2, 3)]
    return orc.ppm_faces(a5[1], a5[2], a5[3], s[0], s[1], s[2])


def test_ppm_fourth_order_interface_and_linear_data(orc):
    # smooth monotone data whose MC slopes are the central differences
    x = np.arange(-2, 3, dtype=float)
    a5 = 1.0 + 0.1 * x + 0.01 * x ** 2 + 0.001 * x ** 3
    for k in (1, 2, 3):
        dl, dr = a5[k] - a5[k - 1], a5[k + 1] - a5[k]
        assert orc.mc_slope(dl, dr) == pytest.approx(0.5 * (dl + dr), rel=1e-15)
    lo, hi = faces_of(orc, a5)
    want_lo = 7 / 12 * (a5[1] + a5[2]) - 1 / 12 * (a5[0] + a5[3])
    want_hi = 7 / 12 * (a5[2] + a5[3]) - 1 / 12 * (a5[1] + a5[4])
    assert lo == pytest.approx(want_lo, abs=1e-15) and hi == pytest.approx(want_hi, abs=1e-15)
    lo, hi = faces_of(orc, np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    assert (lo, hi) == (2.5, 3.5)


def test_ppm_limited_parabola_properties(orc):
    rng = np.random.default_rng(1984)
    n_flat = n_limited = 0
    for _ in range(3000):
        a5 = rng.normal(size=5) * rng.choice([1.0, 0.01])
        if rng.random() < 0.3:
            a5 = np.sort(a5) * rng.choice([-1, 1])
        lo, hi = faces_of(orc, a5)
        a = a5[2]
        # faces between the cell and its face neighbour
        assert min(a5[1], a) - 1e-14 <= lo <= max(a5[1], a) + 1e-14
        assert min(a, a5[3]) - 1e-14 <= hi <= max(a, a5[3]) + 1e-14
        if (a5[3] - a) * (a - a5[1]) <= 0:
            n_flat += 1
            assert lo == hi == a
            continue
        # parabola a(xi) = lo + xi (da + a6 (1 - xi)) on [0, 1]
        da, a6 = hi - lo, 6.0 * (a - 0.5 * (lo + hi))
        xi = np.linspace(0.0, 1.0, 201)
        par = lo + xi * (da + a6 * (1.0 - xi))
        # mean equals the cell value (Simpson is exact for a parabola)
        mean = (lo + 4 * (lo + 0.5 * (da + 0.5 * a6)) + hi) / 6.0
        assert mean == pytest.approx(a, abs=1e-13 * (1 + abs(a)))
        # monotone between its face values
        tol = 1e-12 * (1 + np.abs(a5).max())
        assert par.min() >= min(lo, hi) - tol and par.max() <= max(lo, hi) + tol
        n_limited += abs(da * a6) >= da * da - 1e-15
    assert n_flat > 100 and n_limited > 100


# ----------------------------------------------------- scalar advection
def ppm_faces_np(a):
    """Limited PPM face values (lo, hi) of a periodic array (numpy)."""
    s = mc_slopes(a)
    face = 0.5 * (a + np.roll(a, -1)) - (np.roll(s, -1) - s) / 6.0    # a_{i+1/2}
    lo, hi = np.roll(face, 1).copy(), face.copy()
    flat = (hi - a) * (a - lo) <= 0
    lo[flat] = a[flat]
    hi[flat] = a[flat]
    da = hi - lo
    a6 = 6.0 * (a - 0.5 * (lo + hi))
    over_l = ~flat & (da * a6 > da * da)
    over_r = ~flat & ~over_l & (-(da * da) > da * a6)
    lo = np.where(over_l, 3 * a - 2 * hi, lo)
    hi = np.where(over_r, 3 * a - 2 * lo, hi)
    return lo, hi


def advect_ppm_rk2(a, nu):
    def L(b):
        _, hi = ppm_faces_np(b)
        return -nu * (hi - np.roll(hi, 1))      # upwind: the left cell's high face
    a1 = a + L(a)
    return 0.5 * (a + a1 + L(a1))


@pytest.mark.parametrize("axis,ndim,sign", [(0, 2, 1), (1, 2, -1), (0, 3, -1), (1, 3, 1), (2, 3, 1)])
def test_ppm_contact_advection_equals_textbook_scheme(orc, axis, ndim, sign):
    prob, W, a, speed = advection_case(axis, ndim, sign)
    prob = ppm(prob)
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    nu = 0.4
    dt = nu * prob.dx()[axis] / speed
    lo0, hi0 = a.min(), a.max()
    for _ in range(12):
        U = o.step(U, dt)
        a = advect_ppm_rk2(a, nu) if sign > 0 else advect_ppm_rk2(a[::-1], nu)[::-1]
    rho = np.moveaxis(o.prim(U)[0], 2 - axis, -1).reshape(-1, a.size)
    assert np.abs(rho - a[None, :]).max() <= 1e-13
    assert rho.min() >= lo0 - 1e-12 and rho.max() <= hi0 + 1e-12


# ------------------------------------------------------------ whole step
def test_ppm_sod_against_exact(orc):
    errs = []
    for n in (128, 256, 512):
        prob, W = inputs.sod(n)
        prob = ppm(prob.replace(n=(n, 4, 1), hi=(1.0, 4.0 / n, 1.0)))
        W = np.ascontiguousarray(W[:, :, :4, :])
        o, U, V, t, s = run(orc, prob, W, t_end=0.2)
        P = o.prim(V)
        assert t == 0.2 and (P == P[:, :, :1, :]).all() and (P[2] == 0.0).all()
        rho_ex, _, p_ex = orc.exact_cell_average(SOD_L, SOD_R, 1.4, 0.5, 0.2, np.linspace(0, 1, n + 1))
        errs.append(l1rel(P[0, 0, 0], rho_ex))
        if n == 128:
            assert errs[0] <= 1.5e-2 and l1rel(P[-1, 0, 0], p_ex) <= 1.5e-2
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (np.diff(errs) < 0).all() and order.min() >= 0.6, (errs, order)


@pytest.mark.parametrize("nd,n,steps", [(2, 48, 100), (3, 12, 60)])
def test_ppm_periodic_conservation(orc, nd, n, steps):
    prob, W = inputs.kelvin_helmholtz(n, ndim=nd, U=1.5, ratio=3.0, precision=inputs.FP64)
    o, U, V, t, s = run(orc, ppm(prob), W, max_steps=steps)
    dV = np.prod(prob.dx()[:nd])
    T0, T1 = o.totals(U), o.totals(V)
    mom_scale = np.abs(U[1:1 + nd]).sum() * dV
    for q in range(prob.nvar):
        scale = mom_scale if 1 <= q <= nd else np.abs(U[q]).sum() * dV
        assert abs(T1[q] - T0[q]) <= 1e-13 * scale, q


def test_ppm_mirror_and_rotation_symmetry(orc):
    prob = ppm(Problem(ndim=2, n=(37, 29, 1), bc_lo=(BC_OUTFLOW, BC_PERIODIC, 0),
                       bc_hi=(BC_REFLECT, BC_PERIODIC, 0), grav=(0.0, -0.5, 0.0)))
    W = smooth_random_prim(prob, 11)
    W[0, :, :, :18] *= 1.5
    mprob = prob.replace(bc_lo=(BC_REFLECT, BC_PERIODIC, 0), bc_hi=(BC_OUTFLOW, BC_PERIODIC, 0))
    Wm = W[:, :, :, ::-1].copy()
    Wm[1] *= -1
    _, _, V, _, _ = run(orc, prob, W, max_steps=30)
    _, _, Vm, _, _ = run(orc, mprob, Wm, max_steps=30)
    back = Vm[:, :, :, ::-1].copy()
    back[1] *= -1
    for q in range(prob.nvar):
        assert l1rel(back[q], V[q]) <= 1e-12
    per = (BC_PERIODIC,) * 3
    p3 = ppm(Problem(ndim=3, n=(10, 10, 10), bc_lo=per, bc_hi=per))
    W3 = smooth_random_prim(p3, 5)
    W3[0, :5] *= 1.3
    Wr = np.empty_like(W3)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        Wr[q] = np.transpose(W3[src], (2, 0, 1))
    _, _, V3, _, _ = run(orc, p3, W3, max_steps=20)
    _, _, Vr, _, _ = run(orc, p3, Wr, max_steps=20)
    for q, src in enumerate([0, 2, 3, 1, 4]):
        assert l1rel(Vr[q], np.transpose(V3[src], (2, 0, 1))) <= 1e-12


def test_ppm_pulse_second_order_and_more_accurate_than_plm(orc):
    errs, errs_plm = [], []
    for n in (32, 64, 128, 256):
        prob, W = inputs.smooth_pulse(n, 2)
        o, U, V, t, s = run(orc, ppm(prob), W, t_end=0.25)
        errs.append(l1rel(V[0, 0], inputs.pulse_density(prob, 0.25)[0]))
        o, U, V, t, s = run(orc, prob.replace(scheme=SSPRK2), W, t_end=0.25)
        errs_plm.append(l1rel(V[0, 0], inputs.pulse_density(prob, 0.25)[0]))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order[-2:].min() >= 1.8, (errs, order)
    # the pulse's extremum is flattened by both limiters, so the gain is modest
    assert all(e < 0.95 * ep for e, ep in zip(errs, errs_plm)), (errs, errs_plm)


def test_ppm_rejected_combinations(orc):
    prob, W = inputs.sod(16)
    for bad in (prob.replace(recon=PPM),                              # MUSCL-Hancock
                ppm(prob.replace(n=(16, 2, 1))),                      # fewer than 3 cells
                ppm(inputs.rayleigh_taylor(8, nz=8, hse_subtract=1)[0])):   # background mode
        with pytest.raises(ValueError):
            orc.Oracle(bad).state_from_prim(np.ones(bad.shape))
