"""The seeded input generators (shared by the oracle and the CUDA path).

* the counter-based generator's mixer reproduces the published first outputs
  of SplitMix64 seeded with 0 (Steele, Lea and Flood, OOPSLA 2014; the
  reference implementation's stream e220a8397b1dcdaf, 6e789e6aa1b965f4,
  06c45d188009454f);
* the Rayleigh-Taylor background is hydrostatic (dp0/dz = rho0 g) and its
  multimode perturbation has unit RMS before the 0.01 amplitude;
* the Kelvin-Helmholtz, batch and served-request recipes stay in their
  stated ranges.
"""

import math

import numpy as np

from paper_1510_05061_gb300 import inputs


def test_splitmix64_published_outputs():
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [inputs._mix64_int(k * g & ((1 << 64) - 1)) for k in (1, 2, 3)]
    assert got == want
    arr = inputs._mix64(np.array([g, 2 * g & ((1 << 64) - 1)], dtype=np.uint64))
    assert [int(v) for v in arr] == want[:2]


def test_uniform_and_normal_draws():
    u = inputs.draw_uniform(7, 3, np.arange(200000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = inputs.draw_normal(7, 4, np.arange(200000, dtype=np.uint64))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    # counter-based: a draw does not depend on which other indices are drawn
    assert inputs.draw_uniform(7, 3, np.array([12345], dtype=np.uint64))[0] == u[12345]


def test_rt_background_hydrostatic_and_perturbation_rms():
    z = np.linspace(0.0, 2.0, 20001)
    rho0, p0 = inputs.rt_background(z)
    dpdz = np.gradient(p0, z)
    assert np.abs(dpdz - (-1.0) * rho0).max() < 2e-3      # centred difference of a 0.01-wide tanh
    assert abs(p0[10000] - 2.5) < 1e-12 and p0[-1] > 0.5
    prob, W = inputs.rayleigh_taylor(64)
    k = int(np.argmin(np.abs(prob.centres(2) - 1.0)))
    env = 0.01 * math.exp(-((prob.centres(2)[k] - 1.0) / 0.1) ** 2)
    rms = math.sqrt(float((W[3, k] ** 2).mean())) / env
    assert abs(rms - 1.0) < 1e-12
    assert np.all(W[1] == 0) and np.all(W[2] == 0)
    # extended background tables cover the ghost planes
    assert prob.bg_rho_c.size == 68 and prob.bg_p_f.size == 69


def test_rt_modes_band():
    ks, amp, ph = inputs.rt_modes(151005061)
    r = np.hypot(ks[:, 0], ks[:, 1])
    assert r.min() >= 4 and r.max() <= 16
    assert len({(a, b) for a, b in ks}) == len(ks)
    assert not any((-a, -b) in {(c, d) for c, d in ks} for a, b in ks)


def test_kh_profile_and_batch_recipe():
    prob, W = inputs.kelvin_helmholtz(64, ndim=3, U=1.5, ratio=3.0, precision=inputs.FP64)
    assert abs(W[1].max() - 0.75) < 1e-6 and abs(W[1].min() + 0.75) < 1e-6
    assert abs(W[0].max() - 3.0) < 1e-6 and abs(W[0].min() - 1.0) < 1e-6
    assert np.abs(W[2]).max() <= 0.01 and np.all(W[-1] == 2.5)
    sizes = inputs.kh_batch_sizes()
    assert len(sizes) == 64
    assert all(32 <= s["n"] <= 192 and 0.5 <= s["U"] <= 2.0 and 1.0 <= s["ratio"] <= 4.0 for s in sizes)


def test_served_requests_recipe():
    reqs = inputs.served_requests(count=2000, rate=50.0)
    t = np.array([r["arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(2000 / t[-1] - 50.0) < 5.0
    fam = [r["family"] for r in reqs]
    assert 0.45 < fam.count("kh2d") / 2000 < 0.55
    for r in reqs:
        lo, hi = (64, 2048) if r["family"] == "kh2d" else (32, 256)
        assert lo <= r["n"] <= hi and 100 <= r["steps"] <= 1000
