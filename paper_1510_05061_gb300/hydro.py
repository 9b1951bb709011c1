"""Python binding of libhydro (include/hydro.h): argument marshalling only.

Module-level functions carry the C names (hydro_init, hydro_step,
hydro_advance_to, hydro_reduce, ...) and map one to one onto the C ABI; every
step of the update runs in the library's CUDA kernels.  ``Simulation`` wraps a
handle with PyTorch-owned device buffers on the current CUDA stream.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1510_05061_gb300.build``); loading fails loudly otherwise.
There is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhydro.so")

HYDRO_OK = 0
HYDRO_ERR_INVALID_ARG = -1
HYDRO_ERR_OOM = -2
HYDRO_ERR_CUDA = -3
HYDRO_ERR_NONPHYSICAL = -4
HYDRO_ERR_TIMEOUT = -5
HYDRO_ERR_STATE = -6

HYDRO_RED_TOTALS = 1
HYDRO_RED_DT = 2
HYDRO_RED_TIME = 3
HYDRO_RED_MAXSPEED = 4
HYDRO_RED_STEP = 5
HYDRO_RED_DT_LAST = 6

# every symbol include/hydro.h declares
EXPORTS = (
    "hydro_state_bytes", "hydro_workspace_bytes", "hydro_init", "hydro_init_conserved", "hydro_step",
    "hydro_advance_to", "hydro_reduce", "hydro_current", "hydro_get_state",
    "hydro_set_state", "hydro_get_fields", "hydro_debug_poke", "hydro_debug_pieces", "hydro_set_zchunk", "hydro_set_tile",
    "hydro_launch_count", "hydro_tile_shape", "hydro_destroy", "hydro_strerror", "hydro_totals_noalloc",
    "hydro_selftest_math", "hydro_selftest_device_once", "hydro_fma_probe", "hydro_fma_probe_flops", "hydro_batch_workspace_bytes", "hydro_batch_init",
    "hydro_instance_work_bytes", "hydro_problem_max_items", "hydro_batch_create_bytes",
    "hydro_batch_create", "hydro_batch_add", "hydro_batch_add_async", "hydro_batch_remove",
    "hydro_batch_remove_async", "hydro_batch_get_state_async", "hydro_batch_set_graph",
    "hydro_batch_configure", "hydro_batch_variant_shape", "hydro_batch_step", "hydro_batch_reduce",
    "hydro_batch_get_fields", "hydro_batch_get_state", "hydro_batch_current", "hydro_batch_launch_count", "hydro_batch_items",
    "hydro_batch_destroy", "hydro_checkpoint_save", "hydro_checkpoint_load", "hydro_slab_extent", "hydro_slab_state_bytes", "hydro_slab_workspace_bytes",
    "hydro_slabs_exchange_plan", "hydro_slabs_init", "hydro_slabs_configure", "hydro_slabs_step",
    "hydro_slabs_get_state", "hydro_slabs_get_fields", "hydro_slabs_reduce", "hydro_slabs_launch_count", "hydro_slabs_destroy",
)


class hydro_problem(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("gamma", C.c_double), ("cfl", C.c_double), ("grav", C.c_double * 3),
        ("precision", C.c_int), ("hse_subtract", C.c_int), ("scheme", C.c_int), ("recon", C.c_int),
    ]


class HydroError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.hydro_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libhydro.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhydro.so not built at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    P = C.POINTER(hydro_problem)
    vp, D = C.c_void_p, C.POINTER(C.c_double)
    L.hydro_state_bytes.restype = C.c_size_t
    L.hydro_state_bytes.argtypes = [P]
    L.hydro_workspace_bytes.restype = C.c_size_t
    L.hydro_workspace_bytes.argtypes = [P]
    L.hydro_init.restype = C.c_int
    L.hydro_init.argtypes = [P, vp, vp, vp, D, D, vp, C.POINTER(vp)]
    L.hydro_init_conserved.restype = C.c_int
    L.hydro_init_conserved.argtypes = [P, vp, vp, vp, D, D, vp, C.POINTER(vp)]
    L.hydro_step.restype = C.c_int
    L.hydro_step.argtypes = [vp, D]
    L.hydro_advance_to.restype = C.c_int
    L.hydro_advance_to.argtypes = [vp, C.c_double, C.c_long, C.POINTER(C.c_long), D]
    L.hydro_reduce.restype = C.c_int
    L.hydro_reduce.argtypes = [vp, C.c_int, D]
    L.hydro_current.restype = vp
    L.hydro_current.argtypes = [vp]
    L.hydro_get_state.restype = C.c_int
    L.hydro_get_state.argtypes = [vp, vp]
    L.hydro_set_state.restype = C.c_int
    L.hydro_set_state.argtypes = [vp, vp, C.c_double, C.c_long]
    L.hydro_get_fields.restype = C.c_int
    L.hydro_get_fields.argtypes = [vp, C.c_int, D]
    L.hydro_debug_poke.restype = C.c_int
    L.hydro_debug_poke.argtypes = [vp, C.c_int, C.c_long, C.c_double]
    L.hydro_set_zchunk.restype = C.c_int
    L.hydro_set_zchunk.argtypes = [vp, C.c_int]
    L.hydro_set_tile.restype = C.c_int
    L.hydro_set_tile.argtypes = [vp, C.c_int]
    L.hydro_launch_count.restype = C.c_long
    L.hydro_launch_count.argtypes = [vp]
    L.hydro_tile_shape.restype = C.c_int
    L.hydro_tile_shape.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.hydro_destroy.restype = C.c_int
    L.hydro_destroy.argtypes = [vp]
    L.hydro_strerror.restype = C.c_char_p
    L.hydro_strerror.argtypes = [C.c_int]
    L.hydro_debug_pieces.restype = C.c_int
    L.hydro_debug_pieces.argtypes = [C.c_int, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_longlong,
                                     C.c_longlong, vp, C.c_int]
    L.hydro_selftest_math.restype = C.c_int
    L.hydro_selftest_math.argtypes = [C.c_int, vp, vp, vp, C.c_long, vp]
    L.hydro_fma_probe.restype = C.c_int
    L.hydro_fma_probe.argtypes = [C.c_int, C.c_longlong, C.c_int, C.c_int, vp, vp]
    L.hydro_fma_probe_flops.restype = C.c_double
    L.hydro_fma_probe_flops.argtypes = [C.c_longlong, C.c_int, C.c_int]
    L.hydro_selftest_device_once.restype = C.c_int
    L.hydro_selftest_device_once.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    PP = C.POINTER(C.c_void_p)
    L.hydro_batch_workspace_bytes.restype = C.c_size_t
    L.hydro_batch_workspace_bytes.argtypes = [P, C.c_int]
    L.hydro_batch_init.restype = C.c_int
    L.hydro_batch_init.argtypes = [P, C.c_int, PP, PP, vp, PP, PP, vp, C.POINTER(vp)]
    L.hydro_instance_work_bytes.restype = C.c_size_t
    L.hydro_instance_work_bytes.argtypes = [P]
    L.hydro_problem_max_items.restype = C.c_long
    L.hydro_problem_max_items.argtypes = [P]
    L.hydro_batch_create_bytes.restype = C.c_size_t
    L.hydro_batch_create_bytes.argtypes = [C.c_int, C.c_long, C.c_long]
    L.hydro_batch_create.restype = C.c_int
    L.hydro_batch_create.argtypes = [C.c_int, C.c_long, C.c_long, C.c_int, vp, vp, C.POINTER(vp)]
    L.hydro_batch_add.restype = C.c_int
    L.hydro_batch_add.argtypes = [vp, P, vp, vp, vp, D, D, C.c_long, C.POINTER(C.c_int)]
    L.hydro_batch_remove.restype = C.c_int
    L.hydro_batch_remove.argtypes = [vp, C.c_int]
    L.hydro_batch_add_async.restype = C.c_int
    L.hydro_batch_add_async.argtypes = [vp, P, vp, vp, vp, vp, D, C.c_long, C.POINTER(C.c_int)]
    L.hydro_batch_remove_async.restype = C.c_int
    L.hydro_batch_remove_async.argtypes = [vp, C.c_int]
    L.hydro_batch_get_state_async.restype = C.c_int
    L.hydro_batch_get_state_async.argtypes = [vp, C.c_int, vp]
    L.hydro_batch_set_graph.restype = C.c_int
    L.hydro_batch_set_graph.argtypes = [vp, C.c_int]
    L.hydro_batch_configure.restype = C.c_int
    L.hydro_batch_configure.argtypes = [vp, C.c_int, C.c_int]
    L.hydro_batch_variant_shape.restype = C.c_int
    L.hydro_batch_variant_shape.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.hydro_batch_step.restype = C.c_int
    L.hydro_batch_step.argtypes = [vp, C.c_long]
    L.hydro_batch_reduce.restype = C.c_int
    L.hydro_batch_reduce.argtypes = [vp, C.c_int, C.c_int, D]
    L.hydro_batch_get_fields.restype = C.c_int
    L.hydro_batch_get_fields.argtypes = [vp, C.c_int, C.c_int, D]
    L.hydro_batch_get_state.restype = C.c_int
    L.hydro_batch_get_state.argtypes = [vp, C.c_int, vp]
    L.hydro_batch_current.restype = vp
    L.hydro_batch_current.argtypes = [vp, C.c_int]
    L.hydro_batch_launch_count.restype = C.c_long
    L.hydro_batch_launch_count.argtypes = [vp]
    L.hydro_batch_items.restype = C.c_int
    L.hydro_batch_items.argtypes = [vp] + [C.POINTER(C.c_int)] * 4
    L.hydro_batch_destroy.restype = C.c_int
    L.hydro_batch_destroy.argtypes = [vp]
    L.hydro_checkpoint_save.restype = C.c_int
    L.hydro_checkpoint_save.argtypes = [vp, C.c_char_p]
    L.hydro_checkpoint_load.restype = C.c_int
    L.hydro_checkpoint_load.argtypes = [vp, C.c_char_p]
    L.hydro_totals_noalloc.restype = C.c_int
    L.hydro_totals_noalloc.argtypes = [P, vp, D, vp, D]
    IP = C.POINTER(C.c_int)
    L.hydro_slab_extent.restype = C.c_int
    L.hydro_slab_extent.argtypes = [P, C.c_int, C.c_int, IP, IP]
    L.hydro_slab_state_bytes.restype = C.c_size_t
    L.hydro_slab_state_bytes.argtypes = [P, C.c_int, C.c_int]
    L.hydro_slab_workspace_bytes.restype = C.c_size_t
    L.hydro_slab_workspace_bytes.argtypes = [P, C.c_int, C.c_int]
    L.hydro_slabs_exchange_plan.restype = C.c_int
    L.hydro_slabs_exchange_plan.argtypes = [P, C.c_int, IP, C.c_int]
    L.hydro_slabs_init.restype = C.c_int
    L.hydro_slabs_init.argtypes = [P, C.c_int, PP, PP, PP, D, D, vp, C.POINTER(vp)]
    L.hydro_slabs_configure.restype = C.c_int
    L.hydro_slabs_configure.argtypes = [vp, C.c_int, C.c_int]
    L.hydro_slabs_step.restype = C.c_int
    L.hydro_slabs_step.argtypes = [vp, C.c_long]
    L.hydro_slabs_get_state.restype = C.c_int
    L.hydro_slabs_get_state.argtypes = [vp, vp]
    L.hydro_slabs_get_fields.restype = C.c_int
    L.hydro_slabs_get_fields.argtypes = [vp, C.c_int, D]
    L.hydro_slabs_reduce.restype = C.c_int
    L.hydro_slabs_reduce.argtypes = [vp, C.c_int, D]
    L.hydro_slabs_launch_count.restype = C.c_long
    L.hydro_slabs_launch_count.argtypes = [vp]
    L.hydro_slabs_destroy.restype = C.c_int
    L.hydro_slabs_destroy.argtypes = [vp]
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != HYDRO_OK:
        raise HydroError(rc, what)


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_problem(p: "inputs.Problem") -> hydro_problem:
    s = hydro_problem()
    s.ndim = p.ndim
    for d in range(3):
        s.n[d] = int(p.n[d])
        s.lo[d] = float(p.lo[d])
        s.hi[d] = float(p.hi[d])
        s.bc_lo[d] = int(p.bc_lo[d])
        s.bc_hi[d] = int(p.bc_hi[d])
        s.grav[d] = float(p.grav[d])
    s.gamma = float(p.gamma)
    s.cfl = float(p.cfl)
    s.precision = int(p.precision)
    s.hse_subtract = int(p.hse_subtract)
    s.scheme = int(getattr(p, "scheme", 0))
    s.recon = int(getattr(p, "recon", 0))
    return s


def background_tables(p: "inputs.Problem") -> Optional[np.ndarray]:
    """The hse tables in the order hydro_init expects, or None."""
    if not p.hse_subtract:
        return None
    nz = p.n[2]
    parts = [np.asarray(p.bg_rho_c, np.float64), np.asarray(p.bg_p_c, np.float64),
             np.asarray(p.bg_rho_f, np.float64), np.asarray(p.bg_p_f, np.float64)]
    want = (nz + 4, nz + 4, nz + 5, nz + 5)
    if tuple(x.size for x in parts) != want:
        raise ValueError(f"background tables must have lengths {want}")
    return np.ascontiguousarray(np.concatenate(parts))


# ----------------------------------------------------------- C-named calls

def hydro_state_bytes(prob: hydro_problem) -> int:
    return load().hydro_state_bytes(C.byref(prob))


def hydro_workspace_bytes(prob: hydro_problem) -> int:
    return load().hydro_workspace_bytes(C.byref(prob))


def hydro_init(prob: hydro_problem, Ua: int, Ub: int, work: int, W0: np.ndarray,
               bg: Optional[np.ndarray], stream: int) -> C.c_void_p:
    h = C.c_void_p()
    rc = load().hydro_init(C.byref(prob), C.c_void_p(Ua), C.c_void_p(Ub), C.c_void_p(work),
                           _dptr(W0), _dptr(bg), C.c_void_p(stream), C.byref(h))
    if rc != HYDRO_OK and h.value:
        load().hydro_destroy(h)
    _check(rc, "hydro_init")
    return h


def hydro_init_conserved(prob: hydro_problem, Ua: int, Ub: int, work: int, U0: np.ndarray,
                         bg: Optional[np.ndarray], stream: int) -> C.c_void_p:
    h = C.c_void_p()
    rc = load().hydro_init_conserved(C.byref(prob), C.c_void_p(Ua), C.c_void_p(Ub), C.c_void_p(work),
                                     _dptr(U0), _dptr(bg), C.c_void_p(stream), C.byref(h))
    if rc != HYDRO_OK and h.value:
        load().hydro_destroy(h)
    _check(rc, "hydro_init_conserved")
    return h


def hydro_step(h, want_dt: bool = False) -> Optional[float]:
    dt = C.c_double(0.0)
    _check(load().hydro_step(h, C.byref(dt) if want_dt else None), "hydro_step")
    return dt.value if want_dt else None


def hydro_advance_to(h, t_end: float, max_steps: int = 1 << 40):
    n, t = C.c_long(0), C.c_double(0.0)
    _check(load().hydro_advance_to(h, float(t_end), int(max_steps), C.byref(n), C.byref(t)),
           "hydro_advance_to")
    return n.value, t.value


def hydro_reduce(h, what: int, nvar: int = 1) -> np.ndarray:
    out = np.zeros(max(nvar, 1), dtype=np.float64)
    _check(load().hydro_reduce(h, int(what), _dptr(out)), "hydro_reduce")
    return out


def hydro_current(h) -> int:
    return load().hydro_current(h)


def hydro_get_state(h, dst: np.ndarray):
    _check(load().hydro_get_state(h, C.c_void_p(dst.ctypes.data)), "hydro_get_state")


def hydro_set_state(h, src: np.ndarray, t: float, step: int):
    _check(load().hydro_set_state(h, C.c_void_p(src.ctypes.data), float(t), int(step)),
           "hydro_set_state")


def hydro_get_fields(h, what: int, dst: np.ndarray):
    _check(load().hydro_get_fields(h, int(what), _dptr(dst)), "hydro_get_fields")


def hydro_debug_pieces(zchunk: int, tiles: int, nz: int, tile: int = 0, chunk: int = 0, G: int = 1, b: int = 0):
    """Column pieces (tile, z0, z1) one CTA of a 3D step marches, in order
    (test hook; no GPU needed)."""
    L = load()
    buf = (C.c_int * 3 * 64)()
    n = L.hydro_debug_pieces(int(zchunk), int(tiles), int(nz), int(tile), int(chunk), int(G), int(b),
                             C.cast(buf, C.c_void_p), 64)
    if n < 0:
        _check(n, "hydro_debug_pieces")
    if n > 64:
        buf = (C.c_int * 3 * n)()
        n = L.hydro_debug_pieces(int(zchunk), int(tiles), int(nz), int(tile), int(chunk), int(G), int(b),
                                 C.cast(buf, C.c_void_p), n)
    return [tuple(buf[i]) for i in range(n)]


def hydro_debug_poke(h, var: int, cell: int, v: float):
    _check(load().hydro_debug_poke(h, int(var), int(cell), float(v)), "hydro_debug_poke")


def hydro_set_zchunk(h, z: int):
    _check(load().hydro_set_zchunk(h, int(z)), "hydro_set_zchunk")


def hydro_launch_count(h) -> int:
    return load().hydro_launch_count(h)


def hydro_selftest_math(which: int, x: int, y: int, out: int, n: int, stream: int):
    _check(load().hydro_selftest_math(int(which), C.c_void_p(x), C.c_void_p(y), C.c_void_p(out),
                                      int(n), C.c_void_p(stream)), "hydro_selftest_math")


def hydro_selftest_device_once(devs, fail_dev: int = -1, threads: int = 1, ndev: int = 4):
    """(once_calls, value_calls, values) per fake device (see include/hydro.h)."""
    d = np.ascontiguousarray(devs, dtype=np.int32)
    once = np.zeros(ndev, np.int32)
    vcalls = np.zeros(ndev, np.int32)
    vals = np.zeros(ndev, np.int32)
    ip = C.POINTER(C.c_int)
    _check(load().hydro_selftest_device_once(d.ctypes.data_as(ip), d.size, int(fail_dev), int(threads),
                                             int(ndev), once.ctypes.data_as(ip), vcalls.ctypes.data_as(ip),
                                             vals.ctypes.data_as(ip)), "hydro_selftest_device_once")
    return once, vcalls, vals


def hydro_fma_probe(precision: int, iters: int, ctas: int, threads: int, out: int, stream: int):
    _check(load().hydro_fma_probe(int(precision), int(iters), int(ctas), int(threads), C.c_void_p(out),
                                  C.c_void_p(stream)), "hydro_fma_probe")


def hydro_fma_probe_flops(iters: int, ctas: int, threads: int) -> float:
    return load().hydro_fma_probe_flops(int(iters), int(ctas), int(threads))


def hydro_destroy(h):
    _check(load().hydro_destroy(h), "hydro_destroy")


def hydro_totals_noalloc(prob: hydro_problem, U: int, bg: Optional[np.ndarray], stream: int,
                         nvar: int) -> np.ndarray:
    """Totals of the device state U with no allocation (see include/hydro.h)."""
    out = np.zeros(nvar, dtype=np.float64)
    _check(load().hydro_totals_noalloc(C.byref(prob), C.c_void_p(U), _dptr(bg), C.c_void_p(stream),
                                       _dptr(out)), "hydro_totals_noalloc")
    return out


# --------------------------------------------------------------- wrapper

class Simulation:
    """One solve: torch-owned device buffers bound to a libhydro handle.

    W0 is the host FP64 array of total primitive fields (rho, u.., p) of
    shape prob.shape, or with ``conserved=True`` of total conserved fields
    (rho, m.., E) (hydro_init_conserved).  Runs on ``stream`` (a
    torch.cuda.Stream) or on the current stream of the current device.
    """

    def __init__(self, prob: "inputs.Problem", W0: np.ndarray, stream=None, device=None,
                 conserved: bool = False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libhydro needs a CUDA device")
        self.prob = prob
        self.cp = make_problem(prob)
        sb = hydro_state_bytes(self.cp)
        wb = hydro_workspace_bytes(self.cp)
        if sb == 0 or wb == 0:
            raise HydroError(HYDRO_ERR_INVALID_ARG, "problem")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        # 256-byte aligned device buffers owned by torch
        self._bufs = [torch.empty(n + 256, dtype=torch.uint8, device=dev) for n in (sb, sb, wb)]
        ptrs = [(b.data_ptr() + 255) // 256 * 256 for b in self._bufs]
        self.state_bytes, self.work_bytes = sb, wb
        self._W0 = np.ascontiguousarray(W0, dtype=np.float64)
        if self._W0.shape != tuple(prob.shape):
            raise ValueError(f"W0 shape {self._W0.shape} != {prob.shape}")
        self._bg = background_tables(prob)
        with torch.cuda.device(dev):
            init = hydro_init_conserved if conserved else hydro_init
            self.h = init(self.cp, ptrs[0], ptrs[1], ptrs[2], self._W0, self._bg, self.stream.cuda_stream)

    # stepping ---------------------------------------------------------
    def step(self, want_dt: bool = False):
        return hydro_step(self.h, want_dt)

    def advance_to(self, t_end: float, max_steps: int = 1 << 40):
        return hydro_advance_to(self.h, t_end, max_steps)

    def run_steps(self, n: int):
        """n free steps (no t_end clamp) without synchronising."""
        for _ in range(n):
            hydro_step(self.h, False)

    # reductions -------------------------------------------------------
    def totals(self) -> np.ndarray:
        return hydro_reduce(self.h, HYDRO_RED_TOTALS, self.prob.nvar)

    @property
    def dt(self) -> float:
        return float(hydro_reduce(self.h, HYDRO_RED_DT)[0])

    @property
    def t(self) -> float:
        return float(hydro_reduce(self.h, HYDRO_RED_TIME)[0])

    @property
    def nstep(self) -> int:
        return int(hydro_reduce(self.h, HYDRO_RED_STEP)[0])

    @property
    def dt_last(self) -> float:
        return float(hydro_reduce(self.h, HYDRO_RED_DT_LAST)[0])

    @property
    def max_speed(self) -> float:
        return float(hydro_reduce(self.h, HYDRO_RED_MAXSPEED)[0])

    # fields -----------------------------------------------------------
    def conserved(self) -> np.ndarray:
        out = np.empty(self.prob.shape, dtype=np.float64)
        hydro_get_fields(self.h, 0, out)
        return out

    def primitive(self) -> np.ndarray:
        out = np.empty(self.prob.shape, dtype=np.float64)
        hydro_get_fields(self.h, 1, out)
        return out

    def get_state(self) -> np.ndarray:
        dt = np.float32 if self.prob.precision == inputs.FP32 else np.float64
        out = np.empty(self.prob.shape, dtype=dt)
        hydro_get_state(self.h, out)
        return out

    def set_state(self, raw: np.ndarray, t: float, step: int):
        raw = np.ascontiguousarray(raw)
        if raw.nbytes != self.state_bytes:
            raise ValueError("state size mismatch")
        hydro_set_state(self.h, raw, t, step)

    def save_checkpoint(self, path: str):
        """State, time and step to a file (hydro_checkpoint_save)."""
        _check(load().hydro_checkpoint_save(self.h, os.fsencode(path)), "hydro_checkpoint_save")

    def load_checkpoint(self, path: str):
        """Restart from a file written for the same problem."""
        _check(load().hydro_checkpoint_load(self.h, os.fsencode(path)), "hydro_checkpoint_load")

    def current_ptr(self) -> int:
        return hydro_current(self.h)

    def launches(self) -> int:
        return hydro_launch_count(self.h)

    def set_zchunk(self, z: int):
        hydro_set_zchunk(self.h, z)

    def set_tile(self, variant: int):
        _check(load().hydro_set_tile(self.h, int(variant)), "hydro_set_tile")

    def configure(self, variant: int, zchunk: int = 0):
        """Tile shape and z-chunk of the 3D step (the autotuner's knobs)."""
        self.set_tile(variant)
        self.set_zchunk(zchunk)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            hydro_destroy(self.h)
            self.h = None
        self._bufs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- batches

def hydro_batch_variant_shape(v: int):
    tx, ty = C.c_int(), C.c_int()
    _check(load().hydro_batch_variant_shape(int(v), C.byref(tx), C.byref(ty)), "hydro_batch_variant_shape")
    return tx.value, ty.value


# paired-cell FP32 MUSCL-Hancock tile variants of single 3D solves
PAIR_VARIANTS = (8, 9, 10)
# hydro_set_zchunk: the balanced grid instead of z-chunks
ZCHUNK_BALANCED = -1


def tile_shape(variant: int):
    """Cell tile (tx, ty) of a single-solve 3D variant (0..10)."""
    tx, ty = C.c_int(), C.c_int()
    _check(load().hydro_tile_shape(int(variant), C.byref(tx), C.byref(ty)), "hydro_tile_shape")
    return tx.value, ty.value


def sim_variants():
    """Variant indices of single 3D solves with their cell tiles."""
    out = []
    for v in range(0, 11):
        tx, ty = C.c_int(), C.c_int()
        if load().hydro_tile_shape(v, C.byref(tx), C.byref(ty)) == HYDRO_OK:
            out.append((v, (tx.value, ty.value)))
    return out


def batch_variants():
    """Tile shapes (TX, TY) the batched 3D step can use, by variant index."""
    out = []
    v = 0
    while load().hydro_batch_variant_shape(v, C.byref(C.c_int()), C.byref(C.c_int())) == HYDRO_OK:
        out.append(hydro_batch_variant_shape(v))
        v += 1
    return out


class Batch:
    """Independent instances (list of (Problem, W0)) advanced together by
    the batched persistent step.  Runs on its own torch CUDA stream so that
    the step can be captured into a CUDA graph."""

    def __init__(self, items, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libhydro needs a CUDA device")
        self.probs = [p for p, _ in items]
        n = len(items)
        arr = (hydro_problem * n)(*[make_problem(p) for p in self.probs])
        self._arr = arr
        wb = load().hydro_batch_workspace_bytes(arr, n)
        if wb == 0:
            raise HydroError(HYDRO_ERR_INVALID_ARG, "batch problems")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        dev = torch.device("cuda", torch.cuda.current_device())
        self._bufs = []
        ua, ub = [], []
        for p in self.probs:
            sb = hydro_state_bytes(make_problem(p))
            for lst in (ua, ub):
                t = torch.empty(sb + 256, dtype=torch.uint8, device=dev)
                self._bufs.append(t)
                lst.append((t.data_ptr() + 255) // 256 * 256)
        wt = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
        self._bufs.append(wt)
        work = (wt.data_ptr() + 255) // 256 * 256
        self._W = [np.ascontiguousarray(W, dtype=np.float64) for _, W in items]
        self._bg = [background_tables(p) for p in self.probs]
        VP = C.c_void_p * n
        Wp = VP(*[w.ctypes.data for w in self._W])
        Bp = VP(*[(b.ctypes.data if b is not None else None) for b in self._bg])
        torch.cuda.synchronize()
        h = C.c_void_p()
        rc = load().hydro_batch_init(arr, n, VP(*ua), VP(*ub), C.c_void_p(work), Wp, Bp,
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != HYDRO_OK and h.value:
            load().hydro_batch_destroy(h)
        _check(rc, "hydro_batch_init")
        self.h = h
        self.count = n

    def configure(self, variant: int, zchunk: int = 0):
        _check(load().hydro_batch_configure(self.h, int(variant), int(zchunk)), "hydro_batch_configure")

    def step(self, n: int = 1):
        _check(load().hydro_batch_step(self.h, int(n)), "hydro_batch_step")

    def reduce(self, i: int, what: int) -> np.ndarray:
        out = np.zeros(max(self.probs[i].nvar, 1), dtype=np.float64)
        _check(load().hydro_batch_reduce(self.h, int(i), int(what), _dptr(out)), "hydro_batch_reduce")
        return out

    def t(self, i: int) -> float:
        return float(self.reduce(i, HYDRO_RED_TIME)[0])

    def nstep(self, i: int) -> int:
        return int(self.reduce(i, HYDRO_RED_STEP)[0])

    def totals(self, i: int) -> np.ndarray:
        return self.reduce(i, HYDRO_RED_TOTALS)

    def conserved(self, i: int) -> np.ndarray:
        out = np.empty(self.probs[i].shape, dtype=np.float64)
        _check(load().hydro_batch_get_fields(self.h, int(i), 0, _dptr(out)), "hydro_batch_get_fields")
        return out

    def get_state(self, i: int) -> np.ndarray:
        p = self.probs[i]
        out = np.empty(p.shape, dtype=np.float32 if p.precision == inputs.FP32 else np.float64)
        _check(load().hydro_batch_get_state(self.h, int(i), C.c_void_p(out.ctypes.data)),
               "hydro_batch_get_state")
        return out

    def launches(self) -> int:
        return load().hydro_batch_launch_count(self.h)

    def items(self):
        v = [C.c_int() for _ in range(4)]
        _check(load().hydro_batch_items(self.h, *[C.byref(x) for x in v]), "hydro_batch_items")
        return tuple(x.value for x in v)

    def cells(self) -> int:
        return sum(p.ncell for p in self.probs)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().hydro_batch_destroy(self.h)
            self.h = None
        self._bufs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------- z-slab decomposition

def hydro_slab_extent(prob: hydro_problem, nranks: int, rank: int):
    """(first global plane, plane count) of slab `rank`."""
    z0, nz = C.c_int(), C.c_int()
    _check(load().hydro_slab_extent(C.byref(prob), int(nranks), int(rank), C.byref(z0), C.byref(nz)),
           "hydro_slab_extent")
    return z0.value, nz.value


def hydro_slabs_exchange_plan(prob: hydro_problem, nranks: int):
    """Halo copies of one step: list of (src rank, src first interior plane,
    dst rank, dst first stored plane), each moving two planes of every
    variable.  Host-only: needs no GPU."""
    L = load()
    n = L.hydro_slabs_exchange_plan(C.byref(prob), int(nranks), None, 0)
    if n < 0:
        raise HydroError(n, "hydro_slabs_exchange_plan")
    out = (C.c_int * (4 * max(n, 1)))()
    m = L.hydro_slabs_exchange_plan(C.byref(prob), int(nranks), out, n)
    if m < 0:
        raise HydroError(m, "hydro_slabs_exchange_plan")
    return [tuple(out[4 * i:4 * i + 4]) for i in range(m)]


class Slabs:
    """One 3D problem cut into `nranks` z slabs advanced as virtual ranks on
    the current device: per step a depth-2 halo exchange, the step kernel on
    every slab and a max-reduction of the CFL signal speed.  Results are
    bitwise those of ``Simulation`` on the undivided grid."""

    def __init__(self, prob: "inputs.Problem", W0: np.ndarray, nranks: int, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libhydro needs a CUDA device")
        self.prob, self.nranks = prob, int(nranks)
        self.cp = make_problem(prob)
        L = load()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._bufs = []

        def alloc(n):
            if n == 0:
                raise HydroError(HYDRO_ERR_INVALID_ARG, "slab decomposition")
            t = torch.empty(n + 256, dtype=torch.uint8, device=dev)
            self._bufs.append(t)
            return (t.data_ptr() + 255) // 256 * 256

        ua, ub, wk = [], [], []
        for r in range(self.nranks):
            sb = L.hydro_slab_state_bytes(C.byref(self.cp), self.nranks, r)
            wb = L.hydro_slab_workspace_bytes(C.byref(self.cp), self.nranks, r)
            ua.append(alloc(sb))
            ub.append(alloc(sb))
            wk.append(alloc(wb))
        self._W0 = np.ascontiguousarray(W0, dtype=np.float64)
        if self._W0.shape != tuple(prob.shape):
            raise ValueError(f"W0 shape {self._W0.shape} != {prob.shape}")
        self._bg = background_tables(prob)
        VP = C.c_void_p * self.nranks
        h = C.c_void_p()
        _check(L.hydro_slabs_init(C.byref(self.cp), self.nranks, VP(*ua), VP(*ub), VP(*wk),
                                  _dptr(self._W0), _dptr(self._bg), C.c_void_p(self.stream.cuda_stream),
                                  C.byref(h)), "hydro_slabs_init")
        self.h = h

    def configure(self, variant: int, zchunk: int = 0):
        _check(load().hydro_slabs_configure(self.h, int(variant), int(zchunk)), "hydro_slabs_configure")

    def step(self, n: int = 1):
        _check(load().hydro_slabs_step(self.h, int(n)), "hydro_slabs_step")

    def reduce(self, what: int) -> np.ndarray:
        out = np.zeros(self.prob.nvar, dtype=np.float64)
        _check(load().hydro_slabs_reduce(self.h, int(what), _dptr(out)), "hydro_slabs_reduce")
        return out

    def totals(self) -> np.ndarray:
        return self.reduce(HYDRO_RED_TOTALS)

    @property
    def t(self) -> float:
        return float(self.reduce(HYDRO_RED_TIME)[0])

    @property
    def dt(self) -> float:
        return float(self.reduce(HYDRO_RED_DT)[0])

    @property
    def nstep(self) -> int:
        return int(self.reduce(HYDRO_RED_STEP)[0])

    def get_state(self) -> np.ndarray:
        dt = np.float32 if self.prob.precision == inputs.FP32 else np.float64
        out = np.empty(self.prob.shape, dtype=dt)
        _check(load().hydro_slabs_get_state(self.h, C.c_void_p(out.ctypes.data)), "hydro_slabs_get_state")
        return out

    def conserved(self) -> np.ndarray:
        out = np.empty(self.prob.shape, dtype=np.float64)
        _check(load().hydro_slabs_get_fields(self.h, 0, _dptr(out)), "hydro_slabs_get_fields")
        return out

    def primitive(self) -> np.ndarray:
        out = np.empty(self.prob.shape, dtype=np.float64)
        _check(load().hydro_slabs_get_fields(self.h, 1, _dptr(out)), "hydro_slabs_get_fields")
        return out

    def launches(self) -> int:
        return load().hydro_slabs_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().hydro_slabs_destroy(self.h)
            self.h = None
        self._bufs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
