"""Continuous-batching server for solve requests.

Requests (2D Kelvin-Helmholtz and 3D Rayleigh-Taylor solves of different
sizes, each for a given number of steps) arrive over time.  The server keeps
every admitted solve's state on the device and advances all of them together:
each step is one batched step (one persistent launch for the 3D solves, one
for the 2D solves, whose CTAs claim work items from the batch's
device-resident queue).  A request is admitted as soon as it has arrived, a
slot is free and its device memory (two state buffers and its work buffer)
fits the HBM budget; it leaves the batch right after the step that completes
it.  The host never waits for the whole stream: admissions (an asynchronous
copy of the initial fields from pinned memory and the device conversion),
retirements (an asynchronous copy of the result to pinned memory and the
removal from the device queue) and the steps are all enqueued on the batch
stream, and the host only polls events, keeping up to `lookahead` steps in
flight.  Each request's step limit lives in the device instance table, so a
solve that finishes inside an enqueued run of steps stops there by itself.
Latency is the time the host sees a request's completion event minus its
arrival time.

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
    first_launch: int = 0             # batched steps enqueued before the request joined
    result_pinned: Optional[object] = None

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
    """Admission by slots and HBM budget; steps, admissions and retirements
    enqueued on one stream without synchronising it."""

    def __init__(self, budget_bytes: float = 150e9, max_active: int = 64,
                 precision: int = inputs.FP32, max_items3d: Optional[int] = None,
                 max_items2d: Optional[int] = None, use_graph: bool = True, stream=None,
                 lookahead: int = 8, chunk: int = 2):
        import torch

        self.torch = torch
        self.budget = float(budget_bytes)
        self.used = 0.0
        self.max_active = max_active
        self.precision = precision
        self.lookahead = max(1, int(lookahead))
        self.chunk = max(1, int(chunk))
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
        with torch.cuda.stream(self.stream):
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
        self.launched = 0            # batched steps enqueued so far
        self._pending_keep = []      # pinned and device copies of admitted fields, until the next mark
        self._marks = collections.deque()   # (event, launched, requests retired with it, keepalive)
        self._timing = []            # (start event, end event, zone-updates, bytes) per enqueued run
        self.ticks = 0
        self.zone_updates = 0
        self.bytes_moved = 0

    # memory of one request: two state buffers and its work buffer
    def request_bytes(self, req: Request) -> int:
        cp = hydro.make_problem(req.prob)
        return 2 * hydro.hydro_state_bytes(cp) + hydro.load().hydro_instance_work_bytes(cp)

    def try_admit(self, req: Request, now: float) -> bool:
        """Admit `req` if a slot and memory are free: its buffers are taken
        from the stream's memory pool, its initial fields copied from pinned
        memory and converted on the device, all enqueued on the stream."""
        if len(self.active) >= self.max_active:
            return False
        need = self.request_bytes(req)
        if self.used + need > self.budget:
            return False
        torch = self.torch
        cp = hydro.make_problem(req.prob)
        sb = hydro.hydro_state_bytes(cp)
        wb = hydro.load().hydro_instance_work_bytes(cp)
        # memory allocated on the batch stream: once freed, the caching
        # allocator hands it out again only to work ordered after what was
        # enqueued on this stream, so buffers of a removed solve need no wait
        with torch.cuda.stream(self.stream):
            bufs = [torch.empty(n + 256, dtype=torch.uint8, device=self.dev) for n in (sb, sb, wb)]
            W = np.ascontiguousarray(req.W, dtype=np.float64)
            w_pin = torch.from_numpy(W).pin_memory()
            w_dev = torch.empty(W.shape, dtype=torch.float64, device=self.dev)
            w_dev.copy_(w_pin, non_blocking=True)
        ptrs = [(b.data_ptr() + 255) // 256 * 256 for b in bufs]
        bg = hydro.background_tables(req.prob)
        sid = hydro.C.c_int(-1)
        rc = hydro.load().hydro_batch_add_async(self.h, hydro.C.byref(cp), hydro.C.c_void_p(ptrs[0]),
                                                hydro.C.c_void_p(ptrs[1]), hydro.C.c_void_p(ptrs[2]),
                                                hydro.C.c_void_p(w_dev.data_ptr()), hydro._dptr(bg), req.steps,
                                                hydro.C.byref(sid))
        if rc == hydro.HYDRO_ERR_OOM:
            return False
        hydro._check(rc, "hydro_batch_add_async")
        # the pinned copy must outlive its transfer: released with the next mark
        self._pending_keep += [w_pin, w_dev]
        req.slot = sid.value
        req.admit = now
        req.first_launch = self.launched
        self.active[req.slot] = req
        self._bufs[req.slot] = bufs
        self.used += need
        return True

    def _steps_to_next_finish(self) -> int:
        return min(r.first_launch + r.steps - self.launched for r in self.active.values())

    def advance(self, keep_results: Callable[[Request], bool]) -> List[Request]:
        """Enqueue the steps up to the next completion (at most `chunk`), then
        the retirement of every solve they complete; returns those solves
        (complete once the mark recorded with them has been passed)."""
        torch = self.torch
        k = max(1, min(self.chunk, self._steps_to_next_finish()))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        hydro._check(hydro.load().hydro_batch_step(self.h, k), "hydro_batch_step")
        e1.record(self.stream)
        b = 4 if self.precision == inputs.FP32 else 8
        zu = sum(r.prob.ncell * min(k, r.first_launch + r.steps - self.launched) for r in self.active.values())
        by = sum(2 * r.prob.nvar * b * r.prob.ncell * min(k, r.first_launch + r.steps - self.launched)
                 for r in self.active.values())
        self._timing.append((e0, e1, zu, by))
        self.launched += k
        self.ticks += k
        finished = [r for r in self.active.values() if r.first_launch + r.steps <= self.launched]
        keep, self._pending_keep = self._pending_keep, []
        for req in finished:
            if keep_results(req):
                dt = np.float32 if self.precision == inputs.FP32 else np.float64
                out = torch.empty(tuple(req.prob.shape), dtype=torch.float32 if dt == np.float32 else torch.float64,
                                  pin_memory=True)
                hydro._check(hydro.load().hydro_batch_get_state_async(self.h, req.slot,
                                                                      hydro.C.c_void_p(out.data_ptr())),
                             "hydro_batch_get_state_async")
                req.result_pinned = out
            hydro._check(hydro.load().hydro_batch_remove_async(self.h, req.slot), "hydro_batch_remove_async")
            del self.active[req.slot]
            keep.append(self._bufs.pop(req.slot))
            self.used -= self.request_bytes(req)
        mark = torch.cuda.Event()
        mark.record(self.stream)
        self._marks.append((mark, self.launched, finished, keep))
        return finished

    def poll(self, block: bool = False) -> List[Request]:
        """Requests whose completion the device has reached (the oldest mark
        is waited for when `block`)."""
        done = []
        while self._marks:
            mark, launched, reqs, keep = self._marks[0]
            if not mark.query():
                if not block:
                    break
                mark.synchronize()
                block = False
            self._marks.popleft()
            for r in reqs:
                if getattr(r, "result_pinned", None) is not None:
                    r.result = r.result_pinned.numpy().copy()
                    r.result_pinned = None
            done.extend(reqs)
        return done

    def in_flight(self) -> int:
        """Enqueued steps the device has not passed yet (by the oldest open mark)."""
        return self.launched - self._marks[0][1] + self.chunk if self._marks else 0

    def busy_seconds(self) -> float:
        return sum(a.elapsed_time(b) for a, b, _, _ in self._timing) * 1e-3

    def run(self, requests: List[Request], keep_results: Callable[[Request], bool] = lambda r: False,
            time_scale: float = 1.0) -> dict:
        """Serve `requests` (arrival times scaled by time_scale) to completion."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        prefetch = PayloadPrefetcher(requests, self.precision) if any(r.prob is None for r in requests) else None
        finished: List[Request] = []
        launches0 = hydro.load().hydro_batch_launch_count(self.h)
        t0 = time.perf_counter()
        while pending or self.active or self._marks:
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
            if self.active:
                self.advance(keep_results)
            for req in self.poll(block=self.in_flight() > self.lookahead or (not self.active and not pending)):
                req.done = time.perf_counter() - t0
                finished.append(req)
            if not self.active and not self._marks and pending:
                time.sleep(max(0.0, min(pending[0].arrival * time_scale - (time.perf_counter() - t0), 0.01)))
        makespan = time.perf_counter() - t0
        self.torch.cuda.synchronize()
        busy = self.busy_seconds()
        self.zone_updates = sum(t[2] for t in self._timing)
        self.bytes_moved = sum(t[3] for t in self._timing)
        lat = np.array([r.done - r.arrival * time_scale for r in finished])
        work = sum(r.work for r in finished)
        return {
            "requests": len(finished),
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "makespan_s": makespan,
            "zone_updates": work,
            "zone_updates_per_s": work / makespan,
            "busy_s": busy,
            "busy_zone_updates_per_s": self.zone_updates / busy if busy else None,
            "busy_hbm_gbs": self.bytes_moved / busy / 1e9 if busy else None,
            "ticks": self.ticks,
            "launches": hydro.load().hydro_batch_launch_count(self.h) - launches0,
        }

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            hydro.load().hydro_batch_destroy(self.h)
            self.h = None
        self._bufs = {}
        self._marks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
