"""Continuous-batching serving loop for parallel-in-time solves.

Requests (a problem and its initial data) arrive at any time.  They are admitted
in arrival order as soon as a slot is free and their device footprint
(``pint_footprint`` plus the result and input buffers) fits the HBM budget;
admitted requests run concurrently, each on its own CUDA stream with its own
handle (the iteration loop of each window is one CUDA graph), so requests that
arrive while others are on the GPU overlap with them.  Results stay on the
device (a torch tensor) until the caller takes them.  Every solve is a libpint
call; this module only schedules.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

from . import pint


@dataclass
class Result:
    U: object                      # torch CUDA tensor [nt, nspace] (last window)
    stats: dict
    dof: int
    arrival: float
    start: float
    end: float

    @property
    def latency(self) -> float:
        return self.end - self.arrival


@dataclass
class _Request:
    problem: dict
    u0: object
    footprint: int
    dof: int
    arrival: float
    future: cf.Future = field(default_factory=cf.Future)


class Server:
    """Admission by HBM footprint, up to ``max_slots`` concurrent solves."""

    def __init__(self, hbm_budget_bytes: float = 150e9, max_slots: int = 32, precision: str = "mixed_ff",
                 tol: float = 1e-8, max_iter: int = 200, tol_update: float = 1e-10):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_slots = max_slots
        self.defaults = dict(precision=precision, tol=tol, max_iter=max_iter, init_guess=2, tol_update=tol_update)
        self.streams = [torch.cuda.Stream() for _ in range(max_slots)]
        self.free = list(range(max_slots))
        self.reserved = 0
        self.pending: collections.deque[_Request] = collections.deque()
        self.cv = threading.Condition()
        self.pool = cf.ThreadPoolExecutor(max_workers=max_slots)
        self.running = True
        self.completed: list[Result] = []
        self.busy: list[tuple[float, float]] = []
        self.peak_reserved = 0
        self.rejected = 0
        self.scheduler = threading.Thread(target=self._loop, daemon=True)
        self.scheduler.start()

    # -- client side -----------------------------------------------------------
    def footprint(self, problem: dict) -> int:
        kw = dict(self.defaults, **problem)
        ns = kw["nx"] * (kw.get("ny", 1) if kw.get("dim", 1) == 2 else 1)
        fp = pint.footprint(**kw)
        if fp < 0:
            raise pint.PintError(fp, "pint_footprint")
        return fp + 8 * ns * (kw["nt"] + 1)

    def submit(self, u0, **problem) -> cf.Future:
        """Queue one solve; the future resolves to a Result."""
        fp = self.footprint(problem)
        if fp > self.budget:
            self.rejected += 1
            raise ValueError(f"request needs {fp} bytes, more than the HBM budget {self.budget}")
        ns = problem["nx"] * (problem.get("ny", 1) if problem.get("dim", 1) == 2 else 1)
        req = _Request(problem=dict(problem), u0=u0, footprint=fp, dof=ns * problem["nt"] * problem.get("n_windows", 1),
                       arrival=time.perf_counter())
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()
        return req.future

    def drain(self, timeout: float | None = None) -> None:
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.cv:
            while self.pending or len(self.free) < self.max_slots:
                if timeout is not None and time.perf_counter() - t0 > timeout:
                    raise TimeoutError("serving queue did not drain")
                self.cv.wait(0.05)

    def close(self) -> None:
        self.drain()
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self.scheduler.join()
        self.pool.shutdown(wait=True)

    # -- scheduling ------------------------------------------------------------
    def _loop(self) -> None:
        while True:
            with self.cv:
                while self.running and not (self.pending and self.free and
                                            self.reserved + self.pending[0].footprint <= self.budget):
                    self.cv.wait(0.05)
                if not self.running:
                    return
                req = self.pending.popleft()
                slot = self.free.pop()
                self.reserved += req.footprint
                self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.pool.submit(self._run, req, slot)

    def _run(self, req: _Request, slot: int) -> None:
        torch = self.torch
        stream = self.streams[slot]
        start = time.perf_counter()
        try:
            kw = dict(self.defaults, **req.problem)
            with torch.cuda.stream(stream):
                u0 = req.u0
                if not (hasattr(u0, "is_cuda") and u0.is_cuda):
                    u0 = torch.as_tensor(u0, dtype=torch.float64).to("cuda", non_blocking=True)
                ns = u0.numel()
                U = torch.empty(kw["nt"], ns, dtype=torch.float64, device="cuda")
                with pint.Solver(stream=stream, **kw) as s:
                    st = s.solve(u0, U, check=False)
                stream.synchronize()
            end = time.perf_counter()
            res = Result(U=U, stats=st, dof=req.dof, arrival=req.arrival, start=start, end=end)
            with self.cv:
                self.completed.append(res)
                self.busy.append((start, end))
            req.future.set_result(res)
        except Exception as ex:  # surfaced through the future
            req.future.set_exception(ex)
        finally:
            with self.cv:
                self.reserved -= req.footprint
                self.free.append(slot)
                self.cv.notify_all()

    # -- metrics ---------------------------------------------------------------
    def report(self, results: list[Result] | None = None) -> dict:
        res = self.completed if results is None else results
        if not res:
            return {"n": 0}
        lat = sorted(r.latency for r in res)
        t0 = min(r.arrival for r in res)
        t1 = max(r.end for r in res)
        spans = sorted((r.start, r.end) for r in res)
        busy, cur_s, cur_e = 0.0, None, None
        for s_, e_ in spans:
            if cur_e is None or s_ > cur_e:
                if cur_e is not None:
                    busy += cur_e - cur_s
                cur_s, cur_e = s_, e_
            else:
                cur_e = max(cur_e, e_)
        busy += cur_e - cur_s

        def pct(q):
            return lat[min(len(lat) - 1, int(q * len(lat)))]

        return {"n": len(res), "p50_s": pct(0.5), "p99_s": pct(0.99), "mean_s": sum(lat) / len(lat),
                "dof_per_s": sum(r.dof for r in res) / (t1 - t0), "busy_fraction": busy / (t1 - t0),
                "failed": sum(1 for r in res if r.stats.get("rc", 0) != 0),
                "peak_reserved_bytes": self.peak_reserved}
