"""Continuous-batching server for fracture simulations on one GPU.

Requests (a specimen, a scheme, a precision) arrive at any time.  A request is admitted
when a worker slot is free and its device footprint (pf_footprint_bytes) fits in the HBM
budget left by the running simulations; admission is first come, first served.  Each
admitted simulation keeps u, d and H resident on the device for its whole load path and
runs on its own CUDA stream, so the kernels of all running simulations overlap on the
GPU; a finished path frees its slot and memory for the next request.  Per-step device
latency (CUDA events inside pf_load_step) and per-path latency (arrival to completion)
are recorded.  The kernels are deterministic, so a simulation gives the same result
alone and in the mix.
"""
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import binding


@dataclass
class Request:
    spec: object                     # specimens.Specimen (carries the load increments)
    scheme: int = binding.S1
    precision: int = binding.FP32_IR
    precond: int = binding.PRECOND_GMG
    tol: float = 1e-5
    options: Optional[dict] = None
    keep_fields: bool = False
    rid: int = -1
    arrival: float = 0.0


@dataclass
class Result:
    rid: int
    ok: bool = False
    error: str = ""
    reactions: List[float] = field(default_factory=list)
    stag_iters: List[int] = field(default_factory=list)
    converged: List[int] = field(default_factory=list)
    step_ms: List[float] = field(default_factory=list)
    queue_s: float = 0.0
    path_s: float = 0.0
    footprint: int = 0
    d: Optional[np.ndarray] = None


def run_path(req: Request) -> Result:
    """Run one request's full load path on the current device (the default runner)."""
    res = Result(req.rid)
    sim = binding.Simulation(req.spec, precision=req.precision, precond=req.precond,
                             options=req.options)
    try:
        for du in req.spec.increments:
            r = sim.load_step(du, req.scheme, req.tol)
            res.reactions.append(r["reaction"])
            res.stag_iters.append(r["stag_iters"])
            res.converged.append(r["converged"])
            res.step_ms.append(r["ms"])
        if req.keep_fields:
            res.d = sim.fields()[1]
        res.ok = True
    finally:
        sim.close()
    return res


class Server:
    """FIFO admission by slot and HBM footprint; one worker thread per slot."""

    def __init__(self, hbm_budget: int, slots: int,
                 runner: Callable[[Request], Result] = run_path,
                 footprint: Optional[Callable[[Request], int]] = None,
                 device: Optional[int] = None):
        if slots < 1 or hbm_budget <= 0:
            raise ValueError("need at least one slot and a positive budget")
        self.budget = int(hbm_budget)
        self.slots = int(slots)
        self.runner = runner
        self.footprint = footprint or (lambda r: binding.footprint_bytes(r.spec, r.precision,
                                                                         r.precond))
        self.device = device
        self._cv = threading.Condition()
        self._queue: List[Request] = []
        self._running = 0
        self._in_use = 0
        self._next = 0
        self._closed = False
        self.results = {}
        self.admitted_order: List[int] = []
        self.peak_in_use = 0
        self.peak_running = 0
        self._workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for w in self._workers:
            w.start()

    def submit(self, req: Request) -> int:
        fp = self.footprint(req)
        if fp > self.budget:
            raise ValueError(f"request needs {fp} B, more than the whole budget {self.budget} B")
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            req.rid = self._next
            self._next += 1
            req.arrival = time.perf_counter()
            self._queue.append(req)
            self._cv.notify_all()
            return req.rid

    def _take(self):
        """Block until the head request fits; reserve its slot and memory."""
        with self._cv:
            while True:
                if self._queue:
                    head = self._queue[0]
                    fp = self.footprint(head)
                    if self._in_use + fp <= self.budget:
                        self._queue.pop(0)
                        self._in_use += fp
                        self._running += 1
                        self.peak_in_use = max(self.peak_in_use, self._in_use)
                        self.peak_running = max(self.peak_running, self._running)
                        self.admitted_order.append(head.rid)
                        return head, fp
                elif self._closed:
                    return None, 0
                self._cv.wait()

    def _worker(self):
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)
        while True:
            req, fp = self._take()
            if req is None:
                return
            t0 = time.perf_counter()
            try:
                res = self.runner(req)
            except Exception as e:   # keep serving; the failure is reported per request
                res = Result(req.rid, ok=False, error=repr(e))
            res.queue_s = t0 - req.arrival
            res.path_s = time.perf_counter() - req.arrival
            res.footprint = fp
            with self._cv:
                self.results[req.rid] = res
                self._in_use -= fp
                self._running -= 1
                self._cv.notify_all()

    def drain(self, timeout: Optional[float] = None) -> bool:
        """Wait until every submitted request has finished."""
        deadline = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while self._queue or self._running:
                left = None if deadline is None else deadline - time.perf_counter()
                if left is not None and left <= 0:
                    return False
                self._cv.wait(left)
        return True

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for w in self._workers:
            w.join()


def latency_percentiles(results, q=(50, 99)):
    """p50/p99 of per-step device latency and of per-path latency over finished requests."""
    steps = [ms for r in results.values() if r.ok for ms in r.step_ms]
    paths = [r.path_s for r in results.values() if r.ok]
    pct = lambda a, p: float(np.percentile(a, p)) if a else None
    return ({f"p{p}": pct(steps, p) for p in q}, {f"p{p}": pct(paths, p) for p in q})
