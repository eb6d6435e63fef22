"""Continuous-batching serving loop for parallel-in-time solves.

Requests (a problem and its initial data) arrive at any time.  They are
admitted in arrival order as soon as a slot is free and their device memory
fits the HBM budget; admitted requests run concurrently, each on its own CUDA
stream, so requests that arrive while others are on the GPU overlap with them.
Every solve is a libpint call; this module only schedules and accounts.

Memory accounting (all of it counts against the budget):
  * a solver entry: the handle's workspace (``pint_footprint``) plus its own
    device input and output buffers.  Entries are cached per problem shape and
    reused by later requests of the same shape, so such a request pays neither
    ``pint_create`` nor the capture of the iteration loop's CUDA graph (the
    graph refers to the entry's fixed buffers).  Idle entries are evicted, least
    recently used first, when a request of another shape needs their memory;
  * a result: the solution tensor handed to the caller.  Its bytes stay
    reserved until the caller releases it (``Result.release()``) or the tensor
    is garbage collected.  A caller that keeps every result (and its future)
    alive can therefore exhaust the budget, and admission then waits until
    results are released: release each result once it has been used.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
import weakref
from dataclasses import dataclass, field

from . import pint


@dataclass
class Metrics:
    stats: dict
    dof: int
    arrival: float
    start: float
    end: float

    @property
    def latency(self) -> float:
        return self.end - self.arrival


@dataclass
class Result(Metrics):
    U: object = None               # torch CUDA tensor [nt, nspace] (last window); None once released
    _release: object = None

    def release(self) -> None:
        """Drop the solution tensor and return its bytes to the server's budget."""
        self.U = None
        if self._release is not None:
            self._release()
            self._release = None


@dataclass
class _Request:
    problem: dict
    u0: object
    key: tuple
    entry_bytes: int
    result_bytes: int
    dof: int
    arrival: float
    ready: object = None           # CUDA event recorded on the submitting stream (device u0)
    future: cf.Future = field(default_factory=cf.Future)


class _Entry:
    """A cached solver for one problem shape: handle, stream and fixed I/O buffers."""

    def __init__(self, torch, key, kw, nbytes):
        self.key = key
        self.bytes = nbytes
        self.stream = torch.cuda.Stream()
        ns = kw["nx"] * (kw.get("ny", 1) if kw.get("dim", 1) == 2 else 1)
        self.U = torch.zeros(kw["nt"], ns, dtype=torch.float64, device="cuda")
        self.u0 = torch.zeros(ns, dtype=torch.float64, device="cuda")
        self.solver = pint.Solver(stream=self.stream, **kw)
        self.last_used = time.perf_counter()

    def close(self) -> None:
        self.solver.close()
        self.U = self.u0 = None


class Server:
    """Admission by HBM footprint, up to ``max_slots`` concurrent solves."""

    def __init__(self, hbm_budget_bytes: float = 150e9, max_slots: int = 32, precision: str = "mixed",
                 tol: float = 1e-8, max_iter: int = 200, tol_update: float = 1e-10, cache_solvers: bool = True):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_slots = max_slots
        self.cache_solvers = cache_solvers
        self.defaults = dict(precision=precision, tol=tol, max_iter=max_iter, init_guess=2, tol_update=tol_update)
        self.slots = max_slots
        self.reserved = 0              # entries (busy and idle) + live results
        self.live_result_bytes = 0
        self.idle: dict[tuple, list[_Entry]] = collections.defaultdict(list)
        self.pending: collections.deque[_Request] = collections.deque()
        self.freed: collections.deque[int] = collections.deque()   # result bytes released (any thread)
        self.cv = threading.Condition()
        self.pool = cf.ThreadPoolExecutor(max_workers=max_slots)
        self.running = True
        self.completed: list[Metrics] = []
        self.peak_reserved = 0
        self.rejected = 0
        self.created = 0               # solver entries created
        self.reused = 0                # requests served by a cached entry
        self.scheduler = threading.Thread(target=self._loop, daemon=True)
        self.scheduler.start()

    # -- client side -----------------------------------------------------------
    def _key(self, problem: dict) -> tuple:
        kw = dict(self.defaults, **problem)
        return tuple(sorted(kw.items()))

    def _sizes(self, problem: dict) -> tuple[int, int]:
        kw = dict(self.defaults, **problem)
        ns = kw["nx"] * (kw.get("ny", 1) if kw.get("dim", 1) == 2 else 1)
        fp = pint.footprint(**kw)
        if fp < 0:
            raise pint.PintError(fp, "pint_footprint")
        return fp + 8 * ns * (kw["nt"] + 1), 8 * ns * kw["nt"]

    def footprint(self, problem: dict) -> int:
        """Device bytes one request of this shape may hold: solver entry plus result."""
        e, r = self._sizes(problem)
        return e + r

    def submit(self, u0, **problem) -> cf.Future:
        """Queue one solve; the future resolves to a Result.  A CUDA u0 is read on the
        solve's stream after the work queued so far on the submitting stream."""
        eb, rb = self._sizes(problem)
        if eb + rb > self.budget:
            self.rejected += 1
            raise ValueError(f"request needs {eb + rb} bytes, more than the HBM budget {self.budget}")
        ns = problem["nx"] * (problem.get("ny", 1) if problem.get("dim", 1) == 2 else 1)
        ready = None
        if hasattr(u0, "is_cuda") and u0.is_cuda:
            ready = self.torch.cuda.Event()
            ready.record(self.torch.cuda.current_stream())
        req = _Request(problem=dict(problem), u0=u0, key=self._key(problem), entry_bytes=eb, result_bytes=rb,
                       dof=ns * problem["nt"] * problem.get("n_windows", 1), arrival=time.perf_counter(), ready=ready)
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()
        return req.future

    def drain(self, timeout: float | None = None) -> None:
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.cv:
            while self.pending or self.slots < self.max_slots:
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
        with self.cv:
            for lst in self.idle.values():
                for e in lst:
                    self.reserved -= e.bytes
                    e.close()
            self.idle.clear()

    # -- scheduling ------------------------------------------------------------
    def _collect_freed(self) -> None:
        while self.freed:
            b = self.freed.popleft()
            self.reserved -= b
            self.live_result_bytes -= b

    def _admit(self, req: _Request):
        """Under the lock: reserve memory for req (reusing or evicting idle entries);
        returns (entry or None, bytes reserved for a new entry) or None if it must wait."""
        cached = self.idle.get(req.key)
        if cached:
            e = cached.pop()
            if self.reserved + req.result_bytes > self.budget and not self._evict(req.result_bytes, keep=req.key):
                cached.append(e)
                return None
            self.reserved += req.result_bytes
            self.live_result_bytes += req.result_bytes
            return e, 0
        need = req.entry_bytes + req.result_bytes
        if self.reserved + need > self.budget and not self._evict(need, keep=None):
            return None
        self.reserved += need
        self.live_result_bytes += req.result_bytes
        return None, req.entry_bytes

    def _evict(self, need: int, keep) -> bool:
        """Destroy least recently used idle entries (not of shape `keep`) until `need` fits."""
        cands = sorted((e for k, lst in self.idle.items() if k != keep for e in lst), key=lambda e: e.last_used)
        for e in cands:
            if self.reserved + need <= self.budget:
                break
            self.idle[e.key].remove(e)
            self.reserved -= e.bytes
            e.close()
        return self.reserved + need <= self.budget

    def _loop(self) -> None:
        while True:
            with self.cv:
                adm = None
                while self.running:
                    self._collect_freed()
                    if self.pending and self.slots > 0:
                        adm = self._admit(self.pending[0])
                        if adm is not None:
                            break
                    self.cv.wait(0.02)
                if not self.running:
                    return
                req = self.pending.popleft()
                self.slots -= 1
                self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.pool.submit(self._run, req, *adm)

    def _release_result(self, nbytes: int) -> None:
        # May run from a garbage-collection finalizer in any thread, possibly one that
        # holds the lock: only an atomic append here; the scheduler collects it.
        self.freed.append(nbytes)

    def _run(self, req: _Request, entry, new_bytes: int) -> None:
        torch = self.torch
        start = time.perf_counter()
        made = False
        res, err = None, None
        try:
            kw = dict(self.defaults, **req.problem)
            if entry is None:
                entry = _Entry(torch, req.key, kw, new_bytes)
                made = True
            st_ = entry.stream
            if req.ready is not None:
                st_.wait_event(req.ready)
            with torch.cuda.stream(st_):
                u0 = req.u0
                if not (hasattr(u0, "is_cuda") and u0.is_cuda):
                    u0 = torch.as_tensor(u0, dtype=torch.float64)
                entry.u0.copy_(u0.reshape(-1), non_blocking=True)
                st = entry.solver.solve(entry.u0, entry.U, check=False)
                U = entry.U.clone()
            st_.synchronize()
            end = time.perf_counter()
            res = Result(stats=st, dof=req.dof, arrival=req.arrival, start=start, end=end, U=U)
            # calling the finalizer releases the bytes once; garbage collection of U does the same
            res._release = weakref.finalize(U, self._release_result, req.result_bytes)
        except Exception as ex:  # surfaced through the future
            err = ex
            self._release_result(req.result_bytes)
            if made or entry is None:
                # a new entry that failed (in construction or in its solve) gives its bytes back
                if entry is not None:
                    entry.close()
                with self.cv:
                    self.reserved -= new_bytes
                entry = None
        # the entry and the slot are returned before the caller sees the result, so that a
        # request admitted right after it finds the entry idle
        with self.cv:
            if res is not None:
                if made:
                    self.created += 1
                else:
                    self.reused += 1
                self.completed.append(Metrics(stats=res.stats, dof=req.dof, arrival=req.arrival, start=start,
                                              end=res.end))
            if entry is not None:
                entry.last_used = time.perf_counter()
                if self.cache_solvers:
                    self.idle[entry.key].append(entry)
                else:
                    self.reserved -= entry.bytes
                    entry.close()
            self.slots += 1
            self.cv.notify_all()
        if err is not None:
            req.future.set_exception(err)
        else:
            req.future.set_result(res)

    # -- metrics ---------------------------------------------------------------
    def report(self, results: list | None = None) -> dict:
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
                "peak_reserved_bytes": self.peak_reserved, "solvers_created": self.created,
                "solvers_reused": self.reused}
