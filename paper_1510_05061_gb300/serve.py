"""Continuous-batching server for solve requests.

Requests (2D Kelvin-Helmholtz and 3D Rayleigh-Taylor solves of different
sizes, each for a given number of steps) arrive over time.  The server keeps
every admitted solve's state on the device and advances all of them together:
each tick is one batched step (one persistent launch over the device work
list for the 3D solves, one for the 2D solves).  A request is admitted as
soon as it has arrived, a slot is free and its device memory (two state
buffers and its work buffer) fits the HBM budget; finished solves leave the
batch at the end of the tick that completes them, which frees their slot and
memory for waiting requests.  Latency is completion time minus arrival time.

The paper motivates this as capacity computing: large suites of simulations
for parameter studies and uncertainty quantification ("Increasing computing
power", "Capabilities needed").
"""

from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import hydro, inputs


@dataclasses.dataclass
class Request:
    id: int
    arrival: float            # seconds after the server starts
    family: str               # "kh2d" or "rt3d"
    n: int
    steps: int
    seed: int
    prob: Optional[inputs.Problem] = None
    W: Optional[np.ndarray] = None
    admit: float = math.nan
    done: float = math.nan
    slot: int = -1
    result: Optional[np.ndarray] = None

    @property
    def work(self) -> int:
        return self.prob.ncell * self.steps


def make_payload(req: Request, precision: int = inputs.FP32) -> Request:
    """Build the request's problem and initial fields (seeded)."""
    if req.family == "kh2d":
        u = inputs.draw_uniform(req.seed, 30, np.arange(2, dtype=np.uint64))
        req.prob, req.W = inputs.kelvin_helmholtz(req.n, ndim=2, U=0.5 + 1.5 * float(u[0]),
                                                  ratio=1.0 + 3.0 * float(u[1]), seed=req.seed,
                                                  instance=req.id, precision=precision)
    else:
        req.prob, req.W = inputs.rayleigh_taylor(req.n, seed=req.seed, precision=precision,
                                                 hse_subtract=1)
    return req


def requests_from_inputs(count: int, rate: float, seed: int = 151005063, precision: int = inputs.FP32,
                         lazy: bool = False, **kw) -> List[Request]:
    """The seeded request stream; with lazy the payloads are left to the
    server, which builds them ahead of admission on a background thread."""
    reqs = [Request(id=r["id"], arrival=r["arrival"], family=r["family"], n=r["n"], steps=r["steps"],
                    seed=r["seed"]) for r in inputs.served_requests(count=count, rate=rate, seed=seed, **kw)]
    return reqs if lazy else [make_payload(r, precision) for r in reqs]


class PayloadPrefetcher:
    """Builds request payloads in arrival order on a background thread, at
    most `depth` ahead of admission, so that a long request stream never
    holds all its initial fields in host memory at once."""

    def __init__(self, requests: List[Request], precision: int, depth: int = 8):
        self._order = [r for r in sorted(requests, key=lambda r: r.arrival) if r.prob is None]
        self.ids = {r.id for r in self._order}
        self._precision = precision
        self._room = threading.Semaphore(depth)
        self._cv = threading.Condition()
        self._ready = set()
        self._error: Optional[BaseException] = None
        self._thread = threading.Thread(target=self._work, daemon=True)
        self._thread.start()

    def _work(self):
        try:
            for r in self._order:
                self._room.acquire()
                make_payload(r, self._precision)
                with self._cv:
                    self._ready.add(r.id)
                    self._cv.notify_all()
        except BaseException as e:   # reported to the waiting server thread
            with self._cv:
                self._error = e
                self._cv.notify_all()

    def wait(self, req: Request):
        with self._cv:
            while req.id not in self._ready and self._error is None:
                self._cv.wait()
            if self._error is not None and req.id not in self._ready:
                raise RuntimeError("payload generation failed") from self._error

    def release(self, req: Request):
        """The request's fields are on the device: free them and make room."""
        req.W = None
        self._room.release()


class Server:
    """Admission by slots and HBM budget, one batched step per tick."""

    def __init__(self, budget_bytes: float = 150e9, max_active: int = 64,
                 precision: int = inputs.FP32, max_items3d: Optional[int] = None,
                 max_items2d: Optional[int] = None, use_graph: bool = False, stream=None):
        import torch

        self.torch = torch
        self.budget = float(budget_bytes)
        self.used = 0.0
        self.max_active = max_active
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        # work-list capacity: max_active solves of the largest sizes served
        if max_items3d is None:
            p, _ = inputs.rayleigh_taylor(4, nz=4, perturb=False)
            big = p.replace(n=(256, 256, 256))
            max_items3d = max_active * hydro.load().hydro_problem_max_items(hydro.make_problem(big))
        if max_items2d is None:
            p, _ = inputs.kelvin_helmholtz(2048, ndim=2, precision=precision)
            max_items2d = max_active * hydro.load().hydro_problem_max_items(hydro.make_problem(p))
        nbytes = hydro.load().hydro_batch_create_bytes(max_active, int(max_items3d), int(max_items2d))
        self._work = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        wptr = (self._work.data_ptr() + 255) // 256 * 256
        h = hydro.C.c_void_p()
        hydro._check(hydro.load().hydro_batch_create(max_active, int(max_items3d), int(max_items2d), precision,
                                                     hydro.C.c_void_p(wptr),
                                                     hydro.C.c_void_p(self.stream.cuda_stream),
                                                     hydro.C.byref(h)), "hydro_batch_create")
        self.h = h
        hydro._check(hydro.load().hydro_batch_set_graph(h, 1 if use_graph else 0), "hydro_batch_set_graph")
        self.active: Dict[int, Request] = {}
        self._bufs: Dict[int, list] = {}
        self._steps: Dict[int, int] = {}
        self.ticks = 0
        self.busy_s = 0.0
        self.zone_updates = 0
        self.bytes_moved = 0

    # memory of one request: two state buffers and its work buffer
    def request_bytes(self, req: Request) -> int:
        cp = hydro.make_problem(req.prob)
        return 2 * hydro.hydro_state_bytes(cp) + hydro.load().hydro_instance_work_bytes(cp)

    def try_admit(self, req: Request, now: float) -> bool:
        if len(self.active) >= self.max_active:
            return False
        need = self.request_bytes(req)
        if self.used + need > self.budget:
            return False
        torch = self.torch
        cp = hydro.make_problem(req.prob)
        sb = hydro.hydro_state_bytes(cp)
        wb = hydro.load().hydro_instance_work_bytes(cp)
        bufs = [torch.empty(n + 256, dtype=torch.uint8, device=self.dev) for n in (sb, sb, wb)]
        ptrs = [(b.data_ptr() + 255) // 256 * 256 for b in bufs]
        bg = hydro.background_tables(req.prob)
        W = np.ascontiguousarray(req.W, dtype=np.float64)
        sid = hydro.C.c_int(-1)
        rc = hydro.load().hydro_batch_add(self.h, hydro.C.byref(cp), hydro.C.c_void_p(ptrs[0]),
                                          hydro.C.c_void_p(ptrs[1]), hydro.C.c_void_p(ptrs[2]),
                                          hydro._dptr(W), hydro._dptr(bg), req.steps, hydro.C.byref(sid))
        if rc == hydro.HYDRO_ERR_OOM:
            return False
        hydro._check(rc, "hydro_batch_add")
        req.slot = sid.value
        req.admit = now
        self.active[req.slot] = req
        self._bufs[req.slot] = bufs
        self._steps[req.slot] = 0
        self.used += need
        return True

    def tick(self) -> List[Request]:
        """One step of every active solve; returns the solves it finished."""
        t0 = time.perf_counter()
        hydro._check(hydro.load().hydro_batch_step(self.h, 1), "hydro_batch_step")
        self.stream.synchronize()
        self.busy_s += time.perf_counter() - t0
        self.ticks += 1
        finished = []
        for sid, req in list(self.active.items()):
            self._steps[sid] += 1
            b = 4 if self.precision == inputs.FP32 else 8
            self.zone_updates += req.prob.ncell
            self.bytes_moved += 2 * req.prob.nvar * b * req.prob.ncell
            if self._steps[sid] >= req.steps:
                finished.append(req)
        return finished

    def get_state(self, req: Request) -> np.ndarray:
        out = np.empty(req.prob.shape, dtype=np.float32 if self.precision == inputs.FP32 else np.float64)
        hydro._check(hydro.load().hydro_batch_get_state(self.h, req.slot, hydro.C.c_void_p(out.ctypes.data)),
                     "hydro_batch_get_state")
        return out

    def retire(self, req: Request, keep_result: bool = False):
        if keep_result:
            req.result = self.get_state(req)
        hydro._check(hydro.load().hydro_batch_remove(self.h, req.slot), "hydro_batch_remove")
        del self.active[req.slot]
        del self._bufs[req.slot]
        del self._steps[req.slot]
        self.used -= self.request_bytes(req)

    def run(self, requests: List[Request], keep_results: Callable[[Request], bool] = lambda r: False,
            time_scale: float = 1.0) -> dict:
        """Serve `requests` (arrival times scaled by time_scale) to completion."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        prefetch = PayloadPrefetcher(requests, self.precision) if any(r.prob is None for r in requests) else None
        finished: List[Request] = []
        launches0 = hydro.load().hydro_batch_launch_count(self.h)
        t0 = time.perf_counter()
        while pending or self.active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival * time_scale <= now:
                lazy = prefetch is not None and pending[0].id in prefetch.ids
                if lazy:
                    prefetch.wait(pending[0])
                if not self.try_admit(pending[0], now):
                    break
                if lazy:
                    prefetch.release(pending[0])
                pending.popleft()
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival * time_scale - now, 0.01)))
                continue
            for req in self.tick():
                req.done = time.perf_counter() - t0
                self.retire(req, keep_results(req))
                finished.append(req)
        makespan = time.perf_counter() - t0
        lat = np.array([r.done - r.arrival * time_scale for r in finished])
        work = sum(r.work for r in finished)
        return {
            "requests": len(finished),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "makespan_s": makespan,
            "zone_updates": work,
            "zone_updates_per_s": work / makespan,
            "busy_s": self.busy_s,
            "busy_zone_updates_per_s": self.zone_updates / self.busy_s if self.busy_s else None,
            "busy_hbm_gbs": self.bytes_moved / self.busy_s / 1e9 if self.busy_s else None,
            "ticks": self.ticks,
            "launches": hydro.load().hydro_batch_launch_count(self.h) - launches0,
        }

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            hydro.load().hydro_batch_destroy(self.h)
            self.h = None
        self._bufs = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
