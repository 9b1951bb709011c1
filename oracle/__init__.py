"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct C statement (``hydro_oracle.c``,
``exact_riemann.c``) of the unsplit MUSCL-Hancock / MC-limited PLM / HLLC
update of the compressible Euler equations with constant gravity, and of the
exact Riemann solver that pins it.  Only the tests, ``__graft_entry__.smoke``
and the benchmark's CPU-baseline leg may import this package; the library
path never touches it.  It shares no code with the CUDA path: the only module
both consume is ``paper_1510_05061_gb300.inputs`` (seeded initial data).

Every function that this wrapper exposes is pinned by ``tests/test_oracle_*``
against closed forms, invariants or textbook special cases; the late-time
nonlinear Rayleigh-Taylor and Kelvin-Helmholtz fields are pinned only through
those same invariants (conservation, symmetry) and carry no closed form.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["hydro_oracle.c", "exact_riemann.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("gamma", C.c_double), ("cfl", C.c_double), ("grav", C.c_double * 3),
        ("hse", C.c_int),
        ("bg_rho_c", C.c_void_p), ("bg_p_c", C.c_void_p),
        ("bg_rho_f", C.c_void_p), ("bg_p_f", C.c_void_p),
        ("scheme", C.c_int), ("recon", C.c_int),
    ]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.POINTER(_Params)
            L.orc_mc_slope.restype = C.c_double
            L.orc_mc_slope.argtypes = [C.c_double, C.c_double]
            L.orc_ppm_faces.restype = None
            L.orc_ppm_faces.argtypes = [C.c_double] * 6 + [_D, _D]
            L.orc_hllc.restype = None
            L.orc_hllc.argtypes = [C.c_int, C.c_double, C.c_int, _D, _D, _D]
            L.orc_phys_flux.restype = None
            L.orc_phys_flux.argtypes = [C.c_int, C.c_double, C.c_int, _D, _D]
            L.orc_prim_to_cons1.restype = None
            L.orc_prim_to_cons1.argtypes = [C.c_int, C.c_double, _D, _D]
            L.orc_max_signal.restype = C.c_double
            L.orc_max_signal.argtypes = [P, _D]
            L.orc_cfl_dt.restype = C.c_double
            L.orc_cfl_dt.argtypes = [P, _D]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [P, _D, C.c_double]
            L.orc_run.restype = C.c_int
            L.orc_run.argtypes = [P, _D, C.c_double, C.c_double, C.c_long, _D,
                                  C.POINTER(C.c_long), _D, _D]
            for fn in ("orc_prim_to_state", "orc_state_to_total", "orc_state_to_prim",
                       "orc_totals"):
                getattr(L, fn).restype = C.c_int
                getattr(L, fn).argtypes = [P, _D, _D]
            L.orc_set_threads.restype = None
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_max_threads.restype = C.c_int
            L.orc_max_threads.argtypes = []
            L.orc_exact_star.restype = C.c_int
            L.orc_exact_star.argtypes = [_D, _D, C.c_double, _D, _D, C.POINTER(C.c_int)]
            L.orc_exact_residual.restype = C.c_double
            L.orc_exact_residual.argtypes = [_D, _D, C.c_double, C.c_double]
            L.orc_exact_sample.restype = None
            L.orc_exact_sample.argtypes = [_D, _D, C.c_double, C.c_double, C.c_double,
                                           C.c_double, _D]
            L.orc_fallback_counts.restype = None
            L.orc_fallback_counts.argtypes = [C.POINTER(C.c_longlong), C.c_int]
            L.orc_face_states.restype = C.c_int
            L.orc_face_states.argtypes = [P, _D, C.c_double, _D, C.POINTER(C.c_ubyte)]
            L.orc_exact_profile.restype = C.c_int
            L.orc_exact_profile.argtypes = [_D, _D, C.c_double, C.c_double, C.c_double, _D,
                                            C.c_long, _D, _D, _D]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Oracle:
    """Binds one ``inputs.Problem`` to the C oracle (keeps the tables alive)."""

    def __init__(self, prob, threads: int = 0):
        self.prob = prob
        self._keep = []
        p = _Params()
        p.ndim = prob.ndim
        for d in range(3):
            p.n[d] = int(prob.n[d])
            p.lo[d] = float(prob.lo[d])
            p.hi[d] = float(prob.hi[d])
            p.bc_lo[d] = int(prob.bc_lo[d])
            p.bc_hi[d] = int(prob.bc_hi[d])
            p.grav[d] = float(prob.grav[d])
        p.gamma = float(prob.gamma)
        p.cfl = float(prob.cfl)
        p.hse = int(prob.hse_subtract)
        p.scheme = int(getattr(prob, "scheme", 0))
        p.recon = int(getattr(prob, "recon", 0))
        if prob.hse_subtract:
            for name in ("bg_rho_c", "bg_p_c", "bg_rho_f", "bg_p_f"):
                arr = np.ascontiguousarray(getattr(prob, name), dtype=np.float64)
                self._keep.append(arr)
                setattr(p, name, arr.ctypes.data)
        self.p = p
        self.L = lib()
        if threads:
            self.L.orc_set_threads(int(threads))

    # conversions -----------------------------------------------------
    def state_from_prim(self, W: np.ndarray) -> np.ndarray:
        """Initial primitive fields -> stored state (perturbation in hse mode)."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        U = np.empty_like(W)
        rc = self.L.orc_prim_to_state(C.byref(self.p), _ptr(W), _ptr(U))
        if rc:
            raise ValueError(f"oracle rejected the problem ({rc})")
        return U

    def total(self, U: np.ndarray) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        T = np.empty_like(U)
        self.L.orc_state_to_total(C.byref(self.p), _ptr(U), _ptr(T))
        return T

    def prim(self, U: np.ndarray) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        W = np.empty_like(U)
        self.L.orc_state_to_prim(C.byref(self.p), _ptr(U), _ptr(W))
        return W

    def totals(self, U: np.ndarray) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(self.prob.nvar, dtype=np.float64)
        self.L.orc_totals(C.byref(self.p), _ptr(U), _ptr(out))
        return out

    # time stepping ---------------------------------------------------
    def cfl_dt(self, U: np.ndarray) -> float:
        return self.L.orc_cfl_dt(C.byref(self.p), _ptr(np.ascontiguousarray(U)))

    def max_signal(self, U: np.ndarray) -> float:
        return self.L.orc_max_signal(C.byref(self.p), _ptr(np.ascontiguousarray(U)))

    def step(self, U: np.ndarray, dt: float) -> np.ndarray:
        """One step with a given dt; returns a new array."""
        V = np.array(U, dtype=np.float64, order="C", copy=True)
        rc = self.L.orc_step(C.byref(self.p), _ptr(V), float(dt))
        if rc:
            raise FloatingPointError(f"oracle step failed ({rc})")
        return V

    def face_states(self, U: np.ndarray, dt: float):
        """(Wf, mask): the face states the integrator predicts from U with
        time step dt, Wf[d, s, q] of shape state-shape[1:] (s = 0 the low
        face; stored form, i.e. perturbations in hse mode), and the cells
        that took the positivity fallback."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        nd, nv = self.prob.ndim, self.prob.nvar
        Wf = np.zeros((nd, 2, nv) + tuple(U.shape[1:]), dtype=np.float64)
        mask = np.zeros(U.shape[1:], dtype=np.uint8)
        rc = self.L.orc_face_states(C.byref(self.p), _ptr(U), float(dt), _ptr(Wf),
                                    mask.ctypes.data_as(C.POINTER(C.c_ubyte)))
        if rc:
            raise ValueError(f"oracle rejected the problem ({rc})")
        return Wf, mask.astype(bool)

    def run(self, U: np.ndarray, t_end: float = float("inf"), max_steps: int = 1 << 40,
            t0: float = 0.0, record_dt: bool = False):
        """Advance a copy of U; returns (U, t, steps, dt_last[, dts])."""
        V = np.array(U, dtype=np.float64, order="C", copy=True)
        t = C.c_double(0.0)
        s = C.c_long(0)
        dl = C.c_double(0.0)
        dts = np.zeros(int(min(max_steps, 1 << 20)) if record_dt else 1, dtype=np.float64)
        rc = self.L.orc_run(C.byref(self.p), _ptr(V), float(t0), float(t_end), int(max_steps),
                            C.byref(t), C.byref(s), C.byref(dl),
                            _ptr(dts) if record_dt else None)
        if rc:
            raise FloatingPointError(f"oracle run failed ({rc}) after {s.value} steps")
        if record_dt:
            return V, t.value, s.value, dl.value, dts[: s.value].copy()
        return V, t.value, s.value, dl.value


def fallback_counts(reset: bool = True):
    """(cells, pairs) since the last reset: interior cells whose face states
    took the positivity fallback, and corner transport upwind cell-axis pairs
    kept uncorrected (test instrumentation; no effect on results)."""
    out = (C.c_longlong * 2)()
    lib().orc_fallback_counts(out, 1 if reset else 0)
    return int(out[0]), int(out[1])


# single-face helpers for unit tests ------------------------------------------

def ppm_faces(am: float, a: float, ap: float, sm: float, s: float, sp: float):
    """Limited PPM values at the low and high faces of a cell."""
    lo, hi = C.c_double(), C.c_double()
    lib().orc_ppm_faces(am, a, ap, sm, s, sp, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def mc_slope(dl: float, dr: float) -> float:
    return lib().orc_mc_slope(float(dl), float(dr))


def hllc(ndim: int, gamma: float, d: int, wl, wr) -> np.ndarray:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(ndim + 2, dtype=np.float64)
    lib().orc_hllc(ndim, float(gamma), d, _ptr(wl), _ptr(wr), _ptr(f))
    return f


def phys_flux(ndim: int, gamma: float, d: int, w) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(ndim + 2, dtype=np.float64)
    lib().orc_phys_flux(ndim, float(gamma), d, _ptr(w), _ptr(f))
    return f


def exact_star(wl, wr, gamma: float = 1.4):
    """(p*, u*, newton iterations) of the exact Riemann problem."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    ps, us, it = C.c_double(), C.c_double(), C.c_int()
    rc = lib().orc_exact_star(_ptr(wl), _ptr(wr), float(gamma), C.byref(ps), C.byref(us),
                              C.byref(it))
    if rc:
        raise ValueError(f"exact Riemann solver failed ({rc})")
    return ps.value, us.value, it.value


def exact_residual(wl, wr, gamma: float, p: float) -> float:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    return lib().orc_exact_residual(_ptr(wl), _ptr(wr), float(gamma), float(p))


def exact_profile(wl, wr, gamma: float, x0: float, t: float, x: np.ndarray):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    rho, u, p = (np.zeros_like(x) for _ in range(3))
    rc = lib().orc_exact_profile(_ptr(wl), _ptr(wr), float(gamma), float(x0), float(t),
                                 _ptr(x), x.size, _ptr(rho), _ptr(u), _ptr(p))
    if rc:
        raise ValueError(f"exact Riemann solver failed ({rc})")
    return rho, u, p


def exact_cell_average(wl, wr, gamma: float, x0: float, t: float, edges: np.ndarray,
                       sub: int = 64):
    """Cell averages of the exact (rho, u, p) over cells with the given edges
    (midpoint rule with ``sub`` points per cell)."""
    edges = np.asarray(edges, dtype=np.float64)
    h = np.diff(edges)
    frac = (np.arange(sub) + 0.5) / sub
    x = (edges[:-1, None] + h[:, None] * frac[None, :]).ravel()
    rho, u, p = exact_profile(wl, wr, gamma, x0, t, x)
    n = edges.size - 1
    return (rho.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1))
