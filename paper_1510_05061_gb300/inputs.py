"""Seeded synthetic inputs for the compressible-Euler update.

This module is the one piece of code that both the CUDA path and the CPU
oracle consume.  It describes a problem (grid, boundaries, gas, gravity) and
builds the initial primitive fields W0 = (rho, u, v[, w], p) in float64 on the
host.  It holds none of the update's arithmetic: no equation of state, no
reconstruction, no flux; converting W0 to conserved variables is left to each
consumer.

Random draws use one counter-based generator, the SplitMix64 output mixer
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), keyed by (seed, stream, index) so that any cell's draw is
independent of the order in which cells are generated.

Workloads (stellar-flow motivation: the paper's introduction describes a star
modelled as a fluid on a domain-decomposed grid, and its "Increasing computing
power" section names instabilities and turbulence as the flows of interest):

* ``sod``               2D shock tube along x, checked against the exact
                        Riemann solution.
* ``rayleigh_taylor``   3D single-fluid RT in hydrostatic balance under g=-1
                        with a seeded multimode vz perturbation.
* ``kelvin_helmholtz``  periodic double shear layer with white-noise vy.
* ``smooth_pulse``      advected Gaussian density pulse (exact translate).
* ``kh_batch_sizes``    the 64 seeded box sizes of the batched KH workload.
* ``served_requests``   Poisson arrivals of the served workload.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

BC_OUTFLOW = 0
BC_PERIODIC = 1
BC_REFLECT = 2

FP64 = 0
FP32 = 1

HANCOCK = 0   # single-stage unsplit MUSCL-Hancock
SSPRK2 = 1    # two-stage SSP Runge-Kutta method of lines
CTU = 2       # corner transport upwind (Colella 1990), PLM

PLM = 0       # piecewise linear reconstruction, MC limiter
PPM = 1       # piecewise parabolic reconstruction (SSPRK2, no hse)

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


@dataclasses.dataclass
class Problem:
    """Grid, boundary, gas and gravity description of one solve.

    ``n`` holds (nx, ny, nz); nz is 1 for 2D.  ``lo``/``hi`` are the domain
    corners.  ``bc_lo``/``bc_hi`` hold one of BC_OUTFLOW, BC_PERIODIC,
    BC_REFLECT per axis.  ``grav`` is the constant acceleration vector.
    ``precision`` is FP64 or FP32 (FP32 bulk, FP64 reductions).
    ``hse_subtract`` selects storage of perturbations from a hydrostatic
    background (3D, gravity along z only).  The background is given as float64
    tables over the padded z range: ``bg_rho_c`` / ``bg_p_c`` at the centres
    of planes k = -2 .. nz+1 (length nz + 4, entry k + 2) and ``bg_rho_f`` /
    ``bg_p_f`` at the faces z_lo + f dz, f = -2 .. nz+2 (length nz + 5, entry
    f + 2).  Ghost planes need the background outside the domain.
    ``scheme`` selects the time integrator: HANCOCK (single-stage
    MUSCL-Hancock), SSPRK2 (two-stage method of lines) or CTU (corner
    transport upwind); ``recon`` the
    reconstruction: PLM or PPM (PPM with SSPRK2 and no background only).
    """

    ndim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    bc_lo: Tuple[int, int, int] = (BC_OUTFLOW,) * 3
    bc_hi: Tuple[int, int, int] = (BC_OUTFLOW,) * 3
    gamma: float = 1.4
    cfl: float = 0.8
    grav: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    precision: int = FP64
    hse_subtract: int = 0
    name: str = ""
    bg_rho_c: Optional[np.ndarray] = None
    bg_p_c: Optional[np.ndarray] = None
    bg_rho_f: Optional[np.ndarray] = None
    bg_p_f: Optional[np.ndarray] = None
    scheme: int = 0
    recon: int = 0

    @property
    def nvar(self) -> int:
        return self.ndim + 2

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def shape(self) -> Tuple[int, int, int, int]:
        """Array shape of a state: (nvar, nz, ny, nx), x fastest."""
        return (self.nvar, self.n[2], self.n[1], self.n[0])

    def dx(self) -> Tuple[float, float, float]:
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))

    def centres(self, d: int) -> np.ndarray:
        """Cell-centre coordinates along axis d (point sampling at centres)."""
        h = (self.hi[d] - self.lo[d]) / self.n[d]
        return self.lo[d] + (np.arange(self.n[d], dtype=np.float64) + 0.5) * h

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# counter-based random numbers
# ---------------------------------------------------------------------------

def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK
    z ^= z >> 31
    return z


def draw_u64(seed: int, stream: int, index) -> np.ndarray:
    """64 random bits for each counter ``index`` of (seed, stream)."""
    key = _mix64_int(seed ^ _mix64_int(stream))
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = np.uint64(key) + (idx + np.uint64(1)) * np.uint64(_GOLDEN)
    return _mix64(ctr)


def draw_uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of ``draw_u64``."""
    bits = draw_u64(seed, stream, index) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def draw_normal(seed: int, stream: int, index) -> np.ndarray:
    """Standard normals by Box-Muller on two uniforms per index."""
    idx = np.asarray(index, dtype=np.uint64)
    u1 = draw_uniform(seed, stream, idx * np.uint64(2))
    u2 = draw_uniform(seed, stream, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _prim_zeros(p: Problem) -> np.ndarray:
    return np.zeros(p.shape, dtype=np.float64)


def sod(n: int = 128, ndim: int = 2, gamma: float = 1.4, cfl: float = 0.8,
        precision: int = FP64) -> Tuple[Problem, np.ndarray]:
    """Sod shock tube along x on [0,1]^ndim, split at x = 0.5, outflow BCs.

    Left (rho, u, p) = (1, 0, 1); right = (0.125, 0, 0.1).  The split falls
    on a face for even n, so centre sampling is unambiguous.
    """
    ns = (n, n if ndim >= 2 else 1, n if ndim == 3 else 1)
    prob = Problem(ndim=ndim, n=ns, gamma=gamma, cfl=cfl, precision=precision,
                   name=f"sod{ndim}d-{n}")
    W = _prim_zeros(prob)
    x = prob.centres(0)
    left = x < 0.5
    W[0] = np.where(left, 1.0, 0.125)[None, None, :]
    W[-1] = np.where(left, 1.0, 0.1)[None, None, :]
    return prob, W


def _log_cosh(x: np.ndarray) -> np.ndarray:
    """ln cosh x evaluated without overflow: |x| + log1p(exp(-2|x|)) - ln 2."""
    a = np.abs(x)
    return a + np.log1p(np.exp(-2.0 * a)) - math.log(2.0)


RT_Z_INTERFACE = 1.0
RT_WIDTH = 0.01
RT_P_INTERFACE = 2.5


def rt_background(z: np.ndarray, g: float = -1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Hydrostatic RT background (rho0, p0) at heights z.

    rho0 = 1.5 + 0.5 tanh((z - 1)/0.01) goes from 1 below to 2 above; p0 is
    the closed-form integral of dp/dz = rho0 g with p0(1) = 2.5.
    """
    s = (z - RT_Z_INTERFACE) / RT_WIDTH
    rho0 = 1.5 + 0.5 * np.tanh(s)
    p0 = RT_P_INTERFACE + g * (1.5 * (z - RT_Z_INTERFACE) + 0.5 * RT_WIDTH * _log_cosh(s))
    return rho0, p0


def rt_modes(seed: int, kmin: int = 4, kmax: int = 16):
    """Integer horizontal wave vectors with kmin <= |k| <= kmax (one of each
    +-k pair), their N(0,1) amplitudes and U[0, 2 pi) phases."""
    ks = []
    for ky in range(0, kmax + 1):
        for kx in range(-kmax, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            r2 = kx * kx + ky * ky
            if kmin * kmin <= r2 <= kmax * kmax:
                ks.append((kx, ky))
    m = np.arange(len(ks), dtype=np.uint64)
    amp = draw_normal(seed, 1, m)
    phase = 2.0 * math.pi * draw_uniform(seed, 2, m)
    return np.array(ks, dtype=np.float64), amp, phase


def rayleigh_taylor(n: int = 256, seed: int = 151005061, nz: Optional[int] = None,
                    amplitude: float = 0.01, precision: int = FP64,
                    hse_subtract: int = 0, perturb: bool = True,
                    gamma: float = 1.4, cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """3D single-fluid Rayleigh-Taylor on [0,1]x[0,1]x[0,2].

    n cells per axis (dz = 2 dx), periodic in x and y, reflecting in z,
    g = -1 along z.  Heavy fluid (rho = 2) above z = 1, light (rho = 1) below,
    tanh interface of scale 0.01, hydrostatic pressure with p = 2.5 at the
    interface.  vz = A exp(-((z-1)/0.1)^2) sum_k a_k cos(2 pi k.x + phi_k)
    normalised to unit RMS by sqrt(sum a_k^2 / 2), modes 4 <= |k| <= 16.
    """
    nz = n if nz is None else nz
    g = -1.0
    prob = Problem(ndim=3, n=(n, n, nz), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 2.0),
                   bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                   bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                   gamma=gamma, cfl=cfl, grav=(0.0, 0.0, g), precision=precision,
                   hse_subtract=hse_subtract,
                   name=f"rt3d-{n}x{n}x{nz}")
    x, y, z = prob.centres(0), prob.centres(1), prob.centres(2)
    rho0, p0 = rt_background(z, g)
    dz = prob.dx()[2]
    zc = prob.lo[2] + (np.arange(-2, nz + 2, dtype=np.float64) + 0.5) * dz
    zf = prob.lo[2] + np.arange(-2, nz + 3, dtype=np.float64) * dz
    prob.bg_rho_c, prob.bg_p_c = rt_background(zc, g)
    prob.bg_rho_f, prob.bg_p_f = rt_background(zf, g)
    W = _prim_zeros(prob)
    W[0] = rho0[:, None, None]
    W[4] = p0[:, None, None]
    if perturb:
        ks, amp, phase = rt_modes(seed)
        norm = math.sqrt(0.5 * float(np.sum(amp * amp)))
        # sum_k a_k cos(2 pi (kx x + ky y) + phi_k) = Re(Y^T A X) with
        # A[ky, kx] = a_k exp(i phi_k), X[kx, x] = exp(2 pi i kx x),
        # Y[ky, y] = exp(2 pi i ky y): a small complex matrix product
        kmax = int(np.abs(ks).max())
        A = np.zeros((kmax + 1, 2 * kmax + 1), dtype=np.complex128)
        for (kx, ky), a, ph in zip(ks, amp, phase):
            A[int(ky), int(kx) + kmax] += a * np.exp(1j * ph)
        X = np.exp(2j * math.pi * np.outer(np.arange(-kmax, kmax + 1), x))
        Y = np.exp(2j * math.pi * np.outer(np.arange(0, kmax + 1), y))
        plane = np.real(Y.T @ A @ X) / norm
        env = amplitude * np.exp(-((z - RT_Z_INTERFACE) / 0.1) ** 2)
        W[3] = env[:, None, None] * plane[None, :, :]
    return prob, W


def kelvin_helmholtz(n: int, ndim: int = 3, U: float = 1.0, ratio: float = 2.0,
                     seed: int = 151005062, instance: int = 0, a: float = 0.025,
                     amplitude: float = 0.01, precision: int = FP32,
                     gamma: float = 1.4, cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Periodic double shear layer on [0,1]^ndim.

    vx = U/2 (tanh((y-.25)/a) - tanh((y-.75)/a) - 1) jumps by U across each
    layer; rho goes from 1 (outer band) to ``ratio`` (inner band) with the
    same profile; p = 2.5; vy = amplitude (2 u - 1) with u a per-cell draw
    keyed by (seed, instance, cell index).
    """
    ns = (n, n, n if ndim == 3 else 1)
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=ndim, n=ns, bc_lo=per, bc_hi=per, gamma=gamma, cfl=cfl,
                   precision=precision, name=f"kh{ndim}d-{n}")
    y = prob.centres(1)
    prof = 0.5 * (np.tanh((y - 0.25) / a) - np.tanh((y - 0.75) / a))
    W = _prim_zeros(prob)
    W[0] = (1.0 + (ratio - 1.0) * prof)[None, :, None]
    W[1] = (U * (prof - 0.5))[None, :, None]
    cells = np.arange(prob.ncell, dtype=np.uint64).reshape(ns[2], ns[1], ns[0])
    W[2] = amplitude * (2.0 * draw_uniform(seed, 1000 + instance, cells) - 1.0)
    W[-1] = 2.5
    return prob, W


def smooth_pulse(n: int, ndim: int = 2, width: float = 0.1, amp: float = 0.2,
                 vel=(1.0, 0.5, 0.25), p0: float = 1.0,
                 gamma: float = 1.4, cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Gaussian density pulse in uniform flow on the periodic unit box.

    rho = 1 + amp exp(-|x - c|^2 / width^2), velocity ``vel``, p = p0; the
    exact solution at time t is the same pulse translated by vel t.
    """
    ns = (n, n if ndim >= 2 else 1, n if ndim == 3 else 1)
    per = (BC_PERIODIC,) * 3
    prob = Problem(ndim=ndim, n=ns, bc_lo=per, bc_hi=per, gamma=gamma, cfl=cfl,
                   name=f"pulse{ndim}d-{n}")
    W = _prim_zeros(prob)
    W[0] = pulse_density(prob, 0.0, width, amp, vel)
    for d in range(ndim):
        W[1 + d] = vel[d]
    W[-1] = p0
    return prob, W


def pulse_density(prob: Problem, t: float, width: float = 0.1, amp: float = 0.2,
                  vel=(1.0, 0.5, 0.25)) -> np.ndarray:
    """Exact pulse density at time t (nearest periodic image of the centre)."""
    r2 = np.zeros((prob.n[2], prob.n[1], prob.n[0]), dtype=np.float64)
    for d in range(prob.ndim):
        xc = (0.5 + vel[d] * t) % 1.0
        q = prob.centres(d) - xc
        q = q - np.round(q)
        shape = [1, 1, 1]
        shape[2 - d] = -1
        r2 = r2 + (q * q).reshape(shape)
    return 1.0 + amp * np.exp(-r2 / (width * width))


def kh_batch_sizes(count: int = 64, seed: int = 151005062, nmin: int = 32,
                   nmax: int = 192) -> List[dict]:
    """Seeded parameters of the batched KH boxes: cubic size log-uniform in
    [nmin, nmax], velocity jump U ~ U[0.5, 2], density ratio ~ U[1, 4]."""
    i = np.arange(count, dtype=np.uint64)
    u_n = draw_uniform(seed, 10, i)
    u_U = draw_uniform(seed, 11, i)
    u_r = draw_uniform(seed, 12, i)
    out = []
    for k in range(count):
        nn = int(round(math.exp(math.log(nmin) + u_n[k] * math.log(nmax / nmin))))
        out.append(dict(n=nn, U=0.5 + 1.5 * float(u_U[k]), ratio=1.0 + 3.0 * float(u_r[k]),
                        instance=k))
    return out


def served_requests(count: int = 2000, rate: float = 50.0, seed: int = 151005063,
                    kh2d=(64, 2048), rt3d=(32, 256), steps=(100, 1000)) -> List[dict]:
    """Poisson arrivals of solve requests, 50/50 2D KH and 3D RT, sizes
    log-uniform in the given ranges, step counts uniform on ``steps``."""
    i = np.arange(count, dtype=np.uint64)
    gaps = -np.log1p(-draw_uniform(seed, 20, i)) / rate
    arrive = np.cumsum(gaps)
    kind = draw_uniform(seed, 21, i)
    usz = draw_uniform(seed, 22, i)
    ust = draw_uniform(seed, 23, i)
    out = []
    for k in range(count):
        if kind[k] < 0.5:
            lo, hi = kh2d
            fam = "kh2d"
        else:
            lo, hi = rt3d
            fam = "rt3d"
        nn = int(round(math.exp(math.log(lo) + usz[k] * math.log(hi / lo))))
        nst = steps[0] + int(ust[k] * (steps[1] - steps[0] + 1))
        out.append(dict(id=k, arrival=float(arrive[k]), family=fam, n=nn, steps=nst,
                        seed=seed + k))
    return out


def isentropic_vortex(n: int, half_width: float = 6.0, beta: float = 5.0,
                      vel=(1.0, 1.0), gamma: float = 1.4,
                      cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Isentropic vortex (Yee, Sandham and Djomehri, J. Comput. Phys. 150,
    1999) in uniform flow on the periodic square [-L, L]^2, L = half_width.

    T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) exp(1 - r^2), rho = T^(1/(gamma-1)),
    p = rho^gamma, velocity vel + beta/(2 pi) exp((1 - r^2)/2) (-y, x).  An
    exact steady solution in the vortex frame: at time t it is the same field
    translated by vel t.  At r = L = 6 the perturbation is ~1e-8.
    """
    per = (BC_PERIODIC,) * 3
    L = half_width
    prob = Problem(ndim=2, n=(n, n, 1), lo=(-L, -L, 0.0), hi=(L, L, 1.0),
                   bc_lo=per, bc_hi=per, gamma=gamma, cfl=cfl, name=f"vortex2d-{n}")
    return prob, vortex_prim(prob, 0.0, beta, vel)


def vortex_prim(prob: Problem, t: float, beta: float = 5.0, vel=(1.0, 1.0)) -> np.ndarray:
    """Exact isentropic-vortex primitives at time t (nearest periodic image)."""
    gamma = prob.gamma
    span = [prob.hi[d] - prob.lo[d] for d in range(2)]
    x = prob.centres(0) - vel[0] * t
    y = prob.centres(1) - vel[1] * t
    x = x - span[0] * np.round(x / span[0])
    y = y - span[1] * np.round(y / span[1])
    X, Y = np.meshgrid(x, y)                       # [y][x]
    r2 = X * X + Y * Y
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    W = np.zeros(prob.shape)
    W[0, 0] = rho
    W[1, 0] = vel[0] - amp * Y
    W[2, 0] = vel[1] + amp * X
    W[3, 0] = rho ** gamma
    return W


def riemann_tube(n: int, left, right, x0: float = 0.5, axis: int = 0, ndim: int = 2,
                 width: int = 4, boost: float = 0.0, grav=(0.0, 0.0, 0.0),
                 transverse_bc: int = BC_PERIODIC, gamma: float = 1.4, cfl: float = 0.8,
                 precision: int = FP64, scheme: int = HANCOCK) -> Tuple[Problem, np.ndarray]:
    """One-dimensional Riemann problem in a strip of n cells along `axis`
    (length 1, split at x0) and `width` square cells across each other axis.

    left/right hold (rho, u, p) with u along the strip; `boost` is added to
    both velocities (a Galilean boost, whose exact solution is the unboosted
    one translated by boost * t).  Outflow ends along the strip; the
    transverse boundaries are `transverse_bc`.  Every cross-section starts
    equal, so each row along the strip evolves as the same row.
    """
    n_ = [1, 1, 1]
    hi = [1.0, 1.0, 1.0]
    bc_lo = [BC_OUTFLOW] * 3
    bc_hi = [BC_OUTFLOW] * 3
    for d in range(ndim):
        n_[d] = n if d == axis else width
        hi[d] = 1.0 if d == axis else width / n
        if d != axis:
            bc_lo[d] = bc_hi[d] = transverse_bc
    prob = Problem(ndim=ndim, n=tuple(n_), hi=tuple(hi), bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi),
                   gamma=gamma, cfl=cfl, grav=tuple(grav), precision=precision, scheme=scheme,
                   name=f"tube{ndim}d-{n}-axis{axis}")
    x = prob.centres(axis)
    shape = [1, 1, 1]
    shape[2 - axis] = -1
    is_left = (x < x0).reshape(shape)
    W = _prim_zeros(prob)
    W[0] = np.where(is_left, left[0], right[0])
    W[1 + axis] = np.where(is_left, left[1] + boost, right[1] + boost)
    W[-1] = np.where(is_left, left[2], right[2])
    return prob, W


def filament_column(nz: int = 48, nxy: int = 8, height: float = 12.0, stream: float = 3.0,
                    hse_subtract: int = 0, precision: int = FP64, scheme: int = HANCOCK,
                    cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Isothermal atmosphere rho0 = p0 = exp(-z) under g = -1 on
    [0,1]^2 x [0, height] (periodic in x and y, reflecting in z), whose top
    (above z = 2/3 height, where p0 falls to ~1e-4 .. 6e-6: near vacuum)
    carries dense filaments streaming along x: there the density is rho0
    times the periodic x pattern (1, 10, 40, 40, 40, 10, 1, 1) (stretched over
    nxy cells), the pressure stays p0, v_x = stream and v_y = 0.3 sin(2 pi y).
    The heavy filaments above the light gas and the fast stream through
    density jumps of 40 make predicted face states non-positive in many
    cells.  The background tables are the exact exp(-z) at centres and faces.
    """
    prob = Problem(ndim=3, n=(nxy, nxy, nz), hi=(1.0, 1.0, height),
                   bc_lo=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT),
                   bc_hi=(BC_PERIODIC, BC_PERIODIC, BC_REFLECT), grav=(0.0, 0.0, -1.0),
                   precision=precision, hse_subtract=hse_subtract, scheme=scheme, cfl=cfl,
                   name=f"filaments-{nxy}x{nxy}x{nz}")
    dz = prob.dx()[2]
    zc = (np.arange(-2, nz + 2, dtype=np.float64) + 0.5) * dz
    zf = np.arange(-2, nz + 3, dtype=np.float64) * dz
    prob.bg_rho_c, prob.bg_p_c = np.exp(-zc), np.exp(-zc)
    prob.bg_rho_f, prob.bg_p_f = np.exp(-zf), np.exp(-zf)
    z = prob.centres(2)
    y = prob.centres(1)
    top = (z > 2.0 * height / 3.0)[:, None, None]
    base = np.array([1.0, 10.0, 40.0, 40.0, 40.0, 10.0, 1.0, 1.0])
    pattern = base[(np.arange(nxy) * 8) // nxy]
    W = _prim_zeros(prob)
    W[0] = np.exp(-z)[:, None, None] * np.where(top, pattern[None, None, :], 1.0)
    W[4] = np.exp(-z)[:, None, None] * np.ones((1, nxy, nxy))
    W[1] = np.where(top, stream, 0.0) * np.ones((nz, nxy, nxy))
    W[2] = np.where(top, 0.3 * np.sin(2.0 * math.pi * y)[None, :, None], 0.0) * np.ones((nz, nxy, nxy))
    return prob, W
