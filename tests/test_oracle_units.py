"""Pins of the oracle's pointwise pieces against definitions and closed forms.

* MC limiter (van Leer 1977): hand-evaluated truth table, symmetry, oddness.
* HLLC (Toro, 3rd ed., sec. 10.4-10.6): consistency F(W, W) = F(W) with the
  Euler flux written out here; exact upwinding for supersonic data; exact
  resolution of stationary and moving isolated contacts; mirror and axis
  symmetry.
* Exact Riemann solver (Toro, ch. 4): the printed star values of the five
  standard tests (tests/golden), the root condition, the Rankine-Hugoniot
  jump conditions across the computed shock, and the Riemann invariants in the
  computed rarefaction fan.
"""

import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def euler_flux(w, d, gamma):
    """Euler flux along axis d of a primitive state (rho, u_0..u_{n-1}, p)."""
    w = np.asarray(w, dtype=np.float64)
    nd = w.size - 2
    rho, p = w[0], w[-1]
    vel = w[1:1 + nd]
    E = p / (gamma - 1.0) + 0.5 * rho * float(vel @ vel)
    f = np.empty_like(w)
    f[0] = rho * vel[d]
    f[1:1 + nd] = rho * vel[d] * vel
    f[1 + d] += p
    f[-1] = vel[d] * (E + p)
    return f


# --------------------------------------------------------------------- MC
MC_TABLE = [
    # (dl, dr, slope) evaluated by hand from sign(dr) min(2|dl|, 2|dr|, |dl+dr|/2)
    (1.0, 2.0, 1.5), (2.0, 1.0, 1.5), (1.0, 1.0, 1.0), (1.0, 0.1, 0.2), (0.1, 1.0, 0.2),
    (-1.0, -2.0, -1.5), (-3.0, -1.0, -2.0), (3.0, 1.0, 2.0), (1.0, 3.0, 2.0),
    (4.0, 1.0, 2.0), (1.0, 4.0, 2.0), (5.0, 4.0, 4.5), (1.0, -1.0, 0.0), (-2.0, 5.0, 0.0),
    (0.0, 1.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, -3.0, 0.0),
]


@pytest.mark.parametrize("dl,dr,want", MC_TABLE)
def test_mc_truth_table(orc, dl, dr, want):
    assert orc.mc_slope(dl, dr) == want


def test_mc_symmetry_and_oddness(orc):
    rng = np.random.default_rng(1)
    for dl, dr in rng.normal(size=(200, 2)):
        s = orc.mc_slope(dl, dr)
        assert s == orc.mc_slope(dr, dl)
        assert -s == orc.mc_slope(-dl, -dr)
        # never steeper than twice either one-sided difference (TVD bound)
        assert abs(s) <= 2 * min(abs(dl), abs(dr)) + 0.0


# ------------------------------------------------------------------- HLLC
def random_state(rng, nd):
    w = np.empty(nd + 2)
    w[0] = rng.uniform(0.2, 3.0)
    w[1:1 + nd] = rng.uniform(-1.5, 1.5, nd)
    w[-1] = rng.uniform(0.2, 3.0)
    return w


@pytest.mark.parametrize("nd", [2, 3])
def test_hllc_consistency(orc, nd):
    rng = np.random.default_rng(2 + nd)
    for _ in range(50):
        w = random_state(rng, nd)
        for d in range(nd):
            f = orc.hllc(nd, 1.4, d, w, w)
            np.testing.assert_allclose(f, euler_flux(w, d, 1.4), rtol=1e-14, atol=1e-14)
            np.testing.assert_allclose(orc.phys_flux(nd, 1.4, d, w), euler_flux(w, d, 1.4),
                                       rtol=1e-15, atol=1e-15)


def test_hllc_supersonic_upwind_bitexact(orc):
    g = 1.4
    wl = np.array([1.0, 5.0, 0.3, 0.1, 1.0])
    wr = np.array([0.5, 4.0, -0.2, 0.4, 0.4])
    assert (orc.hllc(3, g, 0, wl, wr) == orc.phys_flux(3, g, 0, wl)).all()
    wl2 = np.array([1.0, -5.0, 0.3, 0.1, 1.0])
    wr2 = np.array([0.5, -4.0, -0.2, 0.4, 0.4])
    assert (orc.hllc(3, g, 0, wl2, wr2) == orc.phys_flux(3, g, 0, wr2)).all()


def test_hllc_stationary_contact(orc):
    g = 1.4
    wl = np.array([1.0, 0.0, 0.7, 1.3])
    wr = np.array([0.125, 0.0, -0.2, 1.3])
    f = orc.hllc(2, g, 0, wl, wr)
    assert abs(f[0]) < 1e-15 and abs(f[3]) < 1e-15
    assert abs(f[2]) < 1e-15
    assert abs(f[1] - 1.3) < 1e-15


@pytest.mark.parametrize("u", [0.3, -0.4])
def test_hllc_moving_contact_exact(orc, u):
    """HLLC resolves an isolated contact exactly: the flux is the upwind
    side's Euler flux."""
    g = 1.4
    wl = np.array([1.0, u, 0.2, -0.1, 1.0])
    wr = np.array([0.25, u, 0.2, -0.1, 1.0])
    f = orc.hllc(3, g, 0, wl, wr)
    up = wl if u > 0 else wr
    np.testing.assert_allclose(f, euler_flux(up, 0, g), rtol=1e-14, atol=1e-14)


def test_hllc_mirror_and_rotation(orc):
    rng = np.random.default_rng(7)
    g = 1.4
    for _ in range(50):
        wl, wr = random_state(rng, 3), random_state(rng, 3)
        f = orc.hllc(3, g, 0, wl, wr)
        # mirror x -> -x: swap sides, negate u; mass, transverse momenta and
        # energy fluxes change sign, the normal momentum flux does not
        ml, mr = wr.copy(), wl.copy()
        ml[1] *= -1
        mr[1] *= -1
        fm = orc.hllc(3, g, 0, ml, mr)
        np.testing.assert_allclose(fm, f * np.array([-1, 1, -1, -1, -1]), rtol=1e-13, atol=1e-14)
        # rotate axes (x, y, z) -> (y, z, x): the y-flux of the rotated states
        perm = [0, 3, 1, 2, 4]
        fy = orc.hllc(3, g, 1, wl[perm], wr[perm])
        np.testing.assert_allclose(fy, f[perm], rtol=1e-13, atol=1e-14)


# ------------------------------------------------------- exact Riemann solver
def _golden():
    with open(os.path.join(GOLDEN, "toro_riemann_star.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("case", _golden()["tests"], ids=lambda c: c["name"])
def test_exact_riemann_printed_values(orc, case):
    g = _golden()["gamma"]
    wl, wr = case["left"], case["right"]
    ps, us, _ = orc.exact_star(wl, wr, g)
    # agreement to the digits printed (5-6 significant)
    assert abs(ps - case["pstar"]) <= 2e-5 * abs(case["pstar"]) + 6e-6
    assert abs(us - case["ustar"]) <= 2e-5 * abs(case["ustar"]) + 6e-6
    eps = 1e-9
    rl, _, _ = orc.exact_profile(wl, wr, g, 0.0, 1.0, np.array([us - eps]))
    rr, _, _ = orc.exact_profile(wl, wr, g, 0.0, 1.0, np.array([us + eps]))
    assert abs(rl[0] - case["rho_star_l"]) <= 2e-5 * case["rho_star_l"] + 6e-6
    assert abs(rr[0] - case["rho_star_r"]) <= 2e-5 * case["rho_star_r"] + 6e-6
    # the root condition itself
    assert abs(orc.exact_residual(wl, wr, g, ps)) < 1e-13 * max(1.0, abs(wr[1] - wl[1]),
                                                                 math.sqrt(max(wl[2], wr[2])))


def test_exact_riemann_sod_jump_conditions(orc):
    """Rankine-Hugoniot across the right shock and Riemann invariants in the
    left fan of the Sod solution, from sampled states only."""
    g = 1.4
    wl, wr = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1]
    ps, us, _ = orc.exact_star(wl, wr, g)
    rr_star, _, _ = orc.exact_profile(wl, wr, g, 0.0, 1.0, np.array([us + 1e-9]))
    rs = rr_star[0]
    S = (rs * us - wr[0] * wr[1]) / (rs - wr[0])      # mass jump gives the speed
    mom_l = rs * us * (us - S) + ps
    mom_r = wr[0] * wr[1] * (wr[1] - S) + wr[2]
    assert abs(mom_l - mom_r) < 1e-13
    E_star = ps / (g - 1) + 0.5 * rs * us * us
    E_r = wr[2] / (g - 1) + 0.5 * wr[0] * wr[1] ** 2
    en_l = (E_star + ps) * us - S * E_star
    en_r = (E_r + wr[2]) * wr[1] - S * E_r
    assert abs(en_l - en_r) < 1e-13
    # the sampled solution jumps exactly at S
    r_before, _, _ = orc.exact_profile(wl, wr, g, 0.0, 1.0, np.array([S - 1e-9]))
    r_after, _, _ = orc.exact_profile(wl, wr, g, 0.0, 1.0, np.array([S + 1e-9]))
    assert abs(r_before[0] - rs) < 1e-12 and r_after[0] == wr[0]
    # left fan: p / rho^gamma and u + 2c/(gamma-1) are constant
    cl = math.sqrt(g * wl[2] / wl[0])
    xs = np.linspace(-cl + 1e-3, us - 0.5, 9)
    rho, u, p = orc.exact_profile(wl, wr, g, 0.0, 1.0, xs)
    np.testing.assert_allclose(p / rho ** g, wl[2] / wl[0] ** g, rtol=1e-13)
    c = np.sqrt(g * p / rho)
    np.testing.assert_allclose(u + 2 * c / (g - 1), 2 * cl / (g - 1), rtol=1e-13)
