"""Pins of the oracle's positivity fallback and of its strong-shock behaviour.

A cell whose predicted face density or pressure is not positive uses zero
slopes along every axis; its face states are then its own primitive state
advanced half a step by its own gravity source (MUSCL-Hancock and the corner
transport upwind predictors), or the state itself (method of lines).  The
fallback is pinned by:

* a hand-built cell that must take it, whose six face states must equal that
  definition exactly (plain and hydrostatic-background modes, both
  predictors), while the method of lines, whose MC-limited faces lie between
  neighbouring values, must never take it;
* Toro's standard tubes 2-5 against the exact Riemann solution (L1 bound and
  refinement order), and a Galilean-boosted test 4 that takes the fallback in
  hundreds of cells, against the translated exact solution;
* that boosted tube run along y and z equalling the x run (a fallback that
  zeroes some axes only breaks this);
* exact free fall across the tube under transverse gravity, v = g t in every
  cell (a fallback without the gravity term breaks this);
* the hydrostatic-background mode with a constant background equalling the
  plain scheme on the boosted tube (the background's imbalance term of the
  fallback enters there).

Toro's tests: E. F. Toro, Riemann Solvers and Numerical Methods for Fluid
Dynamics, 3rd ed., ch. 4 (data in tests/golden/toro_riemann_star.json).
"""

import json
import math
import os

import numpy as np
import pytest

from paper_1510_05061_gb300 import inputs
from paper_1510_05061_gb300.inputs import BC_PERIODIC, BC_REFLECT, Problem

THREADS = 8
HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "toro_riemann_star.json")) as _fh:
    TORO = {t["name"]: t for t in json.load(_fh)["tests"]}
# output times of the five tests (the times Toro's figures show)
T_END = {"test2_123": 0.15, "test3_left_blast": 0.012, "test4_right_blast": 0.035,
         "test5_shock_collision": 0.035}
BOOST = 5.0   # Galilean boost of test 4 that drives cells into the fallback


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def run(orc, prob, W, **kw):
    o = orc.Oracle(prob, threads=THREADS)
    orc.fallback_counts(reset=True)
    V, t, s, dl = o.run(o.state_from_prim(W), **kw)
    return o, V, t, s, orc.fallback_counts(reset=True)


def tube_error(orc, name, n, scheme, boost=0.0):
    """Density L1-rel error of the x tube of Toro's test `name` at its output
    time, against the cell-averaged exact solution; and the fallback count."""
    t = TORO[name]
    x0 = 0.5 - boost * T_END[name]
    prob, W = inputs.riemann_tube(n, t["left"], t["right"], x0=x0, boost=boost, scheme=scheme)
    o, V, tt, s, fb = run(orc, prob, W, t_end=T_END[name])
    assert tt == T_END[name]
    P = o.prim(V)
    wl = [t["left"][0], t["left"][1] + boost, t["left"][2]]
    wr = [t["right"][0], t["right"][1] + boost, t["right"][2]]
    rho, _, _ = orc.exact_cell_average(wl, wr, 1.4, x0, T_END[name], np.linspace(0.0, 1.0, n + 1))
    # every row of the strip is the same row
    assert (P == P[:, :, :1, :]).all()
    return l1rel(P[0, 0, 0], rho), fb


# ------------------------------------------------ Toro tubes at rest
# density L1-rel bounds at n = 200 (about 1.3-1.6x the measured errors)
BOUND_200 = {
    (inputs.HANCOCK, "test2_123"): 1.0e-2, (inputs.HANCOCK, "test3_left_blast"): 8.0e-2,
    (inputs.HANCOCK, "test4_right_blast"): 7.0e-2, (inputs.HANCOCK, "test5_shock_collision"): 2.2e-2,
    (inputs.SSPRK2, "test2_123"): 1.6e-2, (inputs.SSPRK2, "test3_left_blast"): 9.0e-2,
    (inputs.SSPRK2, "test4_right_blast"): 8.0e-2, (inputs.SSPRK2, "test5_shock_collision"): 3.0e-2,
}


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.SSPRK2], ids=["hancock", "ssprk2"])
@pytest.mark.parametrize("name", sorted(T_END))
def test_toro_tubes_against_exact(orc, name, scheme):
    errs = [tube_error(orc, name, n, scheme)[0] for n in (100, 200, 400)]
    assert errs[1] <= BOUND_200[(scheme, name)], errs
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() >= 0.5, (errs, order)


@pytest.mark.parametrize("name", sorted(T_END))
def test_ctu_reduces_to_hancock_in_a_tube(orc, name):
    """With every transverse flux difference zero the corner transport
    upwind step is the MUSCL-Hancock step (up to the rounding of its
    conserved-variable round trip)."""
    t = TORO[name]
    out = []
    for scheme in (inputs.HANCOCK, inputs.CTU):
        prob, W = inputs.riemann_tube(100, t["left"], t["right"], scheme=scheme)
        o, V, _, _, _ = run(orc, prob, W, t_end=T_END[name])
        out.append(o.total(V))
    for q in range(4):
        if np.abs(out[0][q]).sum() > 0:
            assert l1rel(out[1][q], out[0][q]) <= 1e-10, q


# ------------------------------------------------ boosted test 4: fallback
@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
def test_boosted_tube_takes_fallback_and_matches_translate(orc, scheme):
    errs, fbs = [], []
    for n in (100, 200, 400):
        e, fb = tube_error(orc, "test4_right_blast", n, scheme, boost=BOOST)
        errs.append(e)
        fbs.append(fb[0])
    assert min(fbs) > 50, fbs                     # hundreds of cell-steps take the fallback
    assert errs[1] <= 4.5e-2, errs                # measured 3.2e-2
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() >= 0.5, (errs, order)


def test_method_of_lines_never_takes_the_fallback_on_the_boosted_tube(orc):
    """MC-limited faces W -/+ dW/2 lie between neighbouring values, so a
    positive state has positive faces."""
    t = TORO["test4_right_blast"]
    prob, W = inputs.riemann_tube(200, t["left"], t["right"], x0=0.5 - BOOST * 0.035, boost=BOOST,
                                  scheme=inputs.SSPRK2)
    _, _, _, s, fb = run(orc, prob, W, t_end=0.035)
    assert s > 100 and fb == (0, 0)


def _transpose_state(V, axis, ndim):
    """State of a tube along x rearranged as the same tube along `axis`."""
    nv = ndim + 2
    perm_q = list(range(nv))
    perm_q[1], perm_q[1 + axis] = perm_q[1 + axis], perm_q[1]
    # a variable's array is [z][y][x]: swap its x axis (2) with the axis's one
    return np.stack([np.swapaxes(V[perm_q[q]], 2, 2 - axis) for q in range(nv)])


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
@pytest.mark.parametrize("ndim,axis", [(2, 1), (3, 1), (3, 2)])
def test_boosted_tube_is_the_same_along_every_axis(orc, scheme, ndim, axis):
    t = TORO["test4_right_blast"]
    kw = dict(x0=0.5 - BOOST * 0.035, boost=BOOST, ndim=ndim, scheme=scheme)
    px, Wx = inputs.riemann_tube(100, t["left"], t["right"], axis=0, **kw)
    pa, Wa = inputs.riemann_tube(100, t["left"], t["right"], axis=axis, **kw)
    ox, Vx, _, sx, fbx = run(orc, px, Wx, t_end=0.035)
    oa, Va, _, sa, fba = run(orc, pa, Wa, t_end=0.035)
    assert sx == sa and fbx[0] == fba[0] > 0
    want = _transpose_state(Vx, axis, ndim)
    assert want.shape == Va.shape
    for q in range(ndim + 2):
        if np.abs(want[q]).sum() > 0:
            assert l1rel(Va[q], want[q]) <= 1e-12, q
        else:
            assert np.abs(Va[q]).max() == 0.0, q


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
@pytest.mark.parametrize("ndim", [2, 3])
def test_free_fall_across_the_boosted_tube(orc, scheme, ndim):
    """Uniform transverse gravity g on a tube periodic across: every cell
    falls freely, v = g t exactly (up to rounding), fallback cells included."""
    g = -1.0
    grav = (0.0, g, 0.0) if ndim == 2 else (0.0, 0.0, g)
    t = TORO["test4_right_blast"]
    prob, W = inputs.riemann_tube(200, t["left"], t["right"], x0=0.5 - BOOST * 0.035, boost=BOOST,
                                  ndim=ndim, grav=grav, scheme=scheme)
    o, V, tt, s, fb = run(orc, prob, W, t_end=0.035)
    assert fb[0] > 50
    P = o.prim(V)
    v = P[1 + (ndim - 1)]
    assert np.abs(v - g * tt).max() <= 1e-12 * abs(g * tt), np.abs(v - g * tt).max()


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
@pytest.mark.parametrize("axis", [0, 2])
def test_constant_background_equals_plain_on_the_boosted_tube(orc, scheme, axis):
    """With a constant background (rho0, p0) the perturbation form is the plain
    scheme rewritten, its imbalance B = -rho0 g included: the boosted tube
    under gravity along z, with fallback cells, must give the same state."""
    t = TORO["test4_right_blast"]
    prob, W = inputs.riemann_tube(120, t["left"], t["right"], x0=0.5 - BOOST * 0.035, boost=BOOST,
                                  axis=axis, ndim=3, grav=(0.0, 0.0, -1.0), scheme=scheme)
    nz = prob.n[2]
    hp = prob.replace(hse_subtract=1, bg_rho_c=np.full(nz + 4, 0.5), bg_p_c=np.full(nz + 4, 0.005),
                      bg_rho_f=np.full(nz + 5, 0.5), bg_p_f=np.full(nz + 5, 0.005))
    o, V, _, s, fb = run(orc, prob, W, t_end=0.035)
    oh, Vh, _, sh, fbh = run(orc, hp, W, t_end=0.035)
    assert s == sh and fb[0] == fbh[0] > 0
    T, Th = o.total(V), oh.total(Vh)
    scale = np.abs(T).sum() / T.shape[0]
    for q in range(5):
        den = max(np.abs(T[q]).sum(), 1e-3 * scale)
        assert np.abs(Th[q] - T[q]).sum() / den <= 1e-12, q


# ------------------------------------------------ hand-built fallback cell
C = (3, 3, 3)   # (x, y, z) of the designed cell


def designed_state(prob):
    """rho = 1 + 0.1 j, v_x = 10, v_y = 0, v_z = 0.05 k, and along x a
    pressure pattern in which cell x = 3 sits between p = 0.001 and p = 4:
    its MC slope is min(2 * 0.999, 2 * 3, 3.999 / 2) = 1.998, so its low-x
    face pressure W - dW/2 is already 0.001 before the predictor, and the
    predictor's advection term -dt/2 v_x dp/dx (here the only change of p
    along x: v_x is uniform) pushes it below zero for every dt > 0.  The
    cell also has nonzero slopes along y (density) and z (v_z)."""
    n = prob.n
    W = np.zeros(prob.shape)
    j = np.arange(n[1], dtype=float)
    k = np.arange(n[2], dtype=float)
    W[0] = (1.0 + 0.1 * j)[None, :, None] * np.ones((n[2], 1, n[0]))
    W[1] = 10.0
    if prob.ndim == 3:
        W[3] = (0.05 * k)[:, None, None] * np.ones((1, n[1], n[0]))
    p_x = np.array([1.0, 1.0, 0.001, 1.0, 4.0, 4.0, 4.0, 1.0])
    W[-1] = p_x[None, None, :] * np.ones((n[2], n[1], 1))
    return W


def designed_problem(ndim, scheme, hse=False):
    n = (8, 8, 8) if ndim == 3 else (8, 8, 1)
    per = BC_PERIODIC
    if hse:
        prob = Problem(ndim=3, n=n, hi=(1.0, 1.0, 1.0), bc_lo=(per, per, BC_REFLECT),
                       bc_hi=(per, per, BC_REFLECT), grav=(0.0, 0.0, -1.1), scheme=scheme)
        dz = prob.dx()[2]
        zc = (np.arange(-2, 10) + 0.5) * dz
        zf = np.arange(-2, 11) * dz
        # isothermal background rho0 = p0 = 0.5 exp(-z): not discretely balanced, B != 0
        prob = prob.replace(hse_subtract=1, bg_rho_c=0.5 * np.exp(-zc), bg_p_c=0.5 * np.exp(-zc),
                            bg_rho_f=0.5 * np.exp(-zf), bg_p_f=0.5 * np.exp(-zf))
        return prob
    grav = (0.3, -0.7, -1.1) if ndim == 3 else (0.3, -0.7, 0.0)
    return Problem(ndim=ndim, n=n, bc_lo=(per,) * 3, bc_hi=(per,) * 3, grav=grav, scheme=scheme)


def cell_index(ndim):
    return (C[2], C[1], C[0]) if ndim == 3 else (0, C[1], C[0])


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
@pytest.mark.parametrize("ndim", [2, 3])
def test_designed_cell_faces_are_its_state_plus_half_a_step_of_gravity(orc, ndim, scheme):
    prob = designed_problem(ndim, scheme)
    W = designed_state(prob)
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    dt = o.cfl_dt(U)
    Wf, mask = o.face_states(U, dt)
    ci = cell_index(ndim)
    assert mask[ci]
    assert mask.sum() <= mask.size // 4        # the smooth cells keep their slopes
    w = o.prim(U)[(slice(None),) + ci]         # the cell's primitive state
    expect = w.copy()
    for d in range(ndim):
        expect[1 + d] = w[1 + d] + 0.5 * dt * prob.grav[d]
    for d in range(ndim):
        for s in range(2):
            got = Wf[(d, s, slice(None)) + ci]
            np.testing.assert_array_equal(got, expect, err_msg=f"axis {d} side {s}")
    # an unflagged neighbour along y has faces that differ across y (nonzero slope)
    cn = ci[:-2] + (ci[-2] + 1, ci[-1] + 1)
    assert not mask[cn]
    assert Wf[(1, 0, 0) + cn] != Wf[(1, 1, 0) + cn]


@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
def test_designed_cell_faces_in_background_mode(orc, scheme):
    """Perturbation form: the half step of gravity on v_z is
    g rho'/rho - B/rho (B the background's discrete imbalance) for the
    MUSCL-Hancock predictor and the corner transport upwind z predictor; the
    corner transport upwind x and y predictors take plain g."""
    prob = designed_problem(3, scheme, hse=True)
    W = designed_state(prob)
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    dt = o.cfl_dt(U)
    Wf, mask = o.face_states(U, dt)
    ci = cell_index(3)
    assert mask[ci]
    k = C[2]
    g = prob.grav[2]
    dz = prob.dx()[2]
    rho0 = prob.bg_rho_c[k + 2]
    B = (prob.bg_p_f[k + 3] - prob.bg_p_f[k + 2]) / dz - rho0 * g
    wp = U[(slice(None),) + ci].copy()              # stored perturbation
    rho = rho0 + wp[0]
    w = np.array([wp[0], wp[1] / rho, wp[2] / rho, wp[3] / rho, 0.0])
    w[4] = (prob.gamma - 1.0) * (wp[4] - 0.5 * (wp[1] ** 2 + wp[2] ** 2 + wp[3] ** 2) / rho)
    hdt = 0.5 * dt
    vz_src = w[3] + hdt * g * (w[0] / rho) - hdt * B / rho
    vz_plain = w[3] + hdt * g
    for d in range(3):
        expect = w.copy()
        expect[3] = vz_plain if (scheme == inputs.CTU and d < 2) else vz_src
        for s in range(2):
            got = Wf[(d, s, slice(None)) + ci]
            np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-15,
                                       err_msg=f"axis {d} side {s}")
    # the two gravity forms differ here, so the test tells them apart
    assert abs(vz_src - vz_plain) > 1e-3 * abs(hdt * g)


@pytest.mark.parametrize("ndim", [2, 3])
def test_method_of_lines_faces_of_the_designed_cell(orc, ndim):
    """The method of lines' faces are W -/+ dW/2 with the MC slope: the low-x
    face pressure of the designed cell is exactly 0.001 (positive), so no
    cell takes the fallback."""
    prob = designed_problem(ndim, inputs.SSPRK2)
    W = designed_state(prob)
    o = orc.Oracle(prob)
    U = o.state_from_prim(W)
    Wf, mask = o.face_states(U, o.cfl_dt(U))
    assert not mask.any()
    ci = cell_index(ndim)
    np.testing.assert_allclose(Wf[(0, 0, prob.nvar - 1) + ci], 0.001, rtol=1e-12)
    np.testing.assert_allclose(Wf[(0, 1, prob.nvar - 1) + ci], 1.999, rtol=1e-12)


# ------------------------------------------------ a column with a near-vacuum top
@pytest.mark.parametrize("scheme", [inputs.HANCOCK, inputs.CTU], ids=["hancock", "ctu"])
@pytest.mark.parametrize("hse", [0, 1])
def test_filament_column_takes_the_fallback_and_conserves_mass(orc, scheme, hse):
    """Heavy filaments streaming through a near-vacuum top: many cells take
    the fallback, the run stays physical, and mass is conserved between the
    reflecting ends (periodic across) to rounding."""
    prob, W = inputs.filament_column(nz=48, stream=3.0, hse_subtract=hse, scheme=scheme)
    o = orc.Oracle(prob, threads=THREADS)
    U = o.state_from_prim(W)
    orc.fallback_counts(reset=True)
    V, t, s, _ = o.run(U, max_steps=10)
    fb = orc.fallback_counts(reset=True)
    assert s == 10 and fb[0] > 100
    m0, m1 = o.totals(U)[0], o.totals(V)[0]
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
