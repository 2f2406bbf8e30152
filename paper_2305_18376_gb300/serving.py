"""Serving loop: many independent Dash streams on one GPU.

Each stream owns one DashModel (its factors and per-slice summaries stay in
device memory between updates) on its own CUDA stream.  Requests are a
stream's initial fit or one of its update batches (Algorithm 1).  The loop
admits them in arrival order as slots and device memory free up:

* a request is admitted once it has arrived, no earlier request of its
  stream is waiting or running (a stream's updates are sequential), and
  fewer than `max_inflight` requests are running;
* a stream's model is created at its first admitted request if the device
  bytes of the resident models plus its own (dash_config_bytes, computed
  without allocating) stay within `hbm_budget`; otherwise models of streams
  with no requests left are retired (their final state handed to
  `on_retire`, then freed) and, failing that, the request waits while later
  requests of resident streams go ahead;
* admitted work is issued asynchronously (append + dash_update on the
  model's stream), so requests of different streams overlap on the device;
  completion is polled without blocking (dash_query).

Host scheduling only: every step of an update runs in the library's
kernels.  The arithmetic of a stream does not depend on what else runs, so
its results are the same alone and in the mix.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    """One unit of work of a stream: kind "init" (append the initial tensor,
    then `init_iters` static ALS iterations) or "update" (append one batch,
    then one Dash update)."""
    stream: int
    arrival: float                 # seconds after the loop starts
    kind: str                      # "init" | "update"
    slice_ids: Any
    row_ptr: Any
    X: Any                         # host array or CUDA tensor of the model's input dtype
    init_iters: int = 1
    rows: int = 0
    admitted: Optional[float] = None
    done: Optional[float] = None
    issue_s: Optional[float] = None    # host time spent issuing it (append + update calls)
    failed: Optional[str] = None       # why it was not served (its stream's numerics failed)

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class ServingError(RuntimeError):
    pass


NUMERIC_FAILURE = 5    # DASH_ENUMERIC: a non-finite value reached a stream's factors


class ServingLoop:
    """Admission, issue and completion of requests of many streams.

    specs[s]: keyword arguments of stream s's DashModel (J, R, lam, precision,
    capacities ...).  `factory(**spec)` builds a model, `bytes_of(spec)` gives
    its device bytes before it exists; both default to the library's
    (DashModel, dash_config_bytes) and are replaceable for host-only tests.
    `prepare(stream, model)` runs once after a model is created (e.g. to set
    its initial factors); `on_retire(stream, model)` runs before a model is
    freed, at retirement or at the end of run()."""

    def __init__(self, specs: Dict[int, dict], hbm_budget: int, max_inflight: int = 8,
                 factory: Optional[Callable[..., Any]] = None,
                 bytes_of: Optional[Callable[[dict], int]] = None,
                 prepare: Optional[Callable[[int, Any], None]] = None,
                 on_retire: Optional[Callable[[int, Any], None]] = None,
                 clock: Callable[[], float] = time.perf_counter, poll_sleep: float = 20e-6):
        if factory is None or bytes_of is None:
            from ._native import DashModel, config_bytes
            factory = factory or DashModel
            bytes_of = bytes_of or (lambda spec: config_bytes(**spec)[0])
        if max_inflight < 1:
            raise ValueError("max_inflight must be at least 1")
        self.specs = specs
        self.budget = int(hbm_budget)
        self.max_inflight = max_inflight
        self.factory, self.bytes_of = factory, bytes_of
        self.prepare, self.on_retire = prepare, on_retire
        self.clock, self.poll_sleep = clock, poll_sleep
        self.models: Dict[int, Any] = {}
        self.model_bytes: Dict[int, int] = {}
        self.resident = 0
        self.peak_resident = 0
        self.retired: List[int] = []
        self.events: List[tuple] = []      # (time, "admit"|"done"|"create"|"retire"|"fail", stream)
        self.failed: Dict[int, str] = {}   # streams stopped by a numerical failure
        self._t0 = clock()
        self._final = True

    # ---- model residency ---------------------------------------------------
    def _retire(self, s: int, now: float):
        m = self.models.pop(s)
        if self.on_retire:
            self.on_retire(s, m)
        m.close()
        self.resident -= self.model_bytes.pop(s)
        self.retired.append(s)
        self.events.append((now, "retire", s))

    def _make_room(self, need: int, left: Dict[int, int], busy: set, now: float) -> bool:
        if self.resident + need <= self.budget:
            return True
        if not self._final:
            return False
        for s in sorted(self.models):
            if self.resident + need <= self.budget:
                break
            if left.get(s, 0) == 0 and s not in busy:
                self._retire(s, now)
        return self.resident + need <= self.budget

    def _ensure_model(self, s: int, left: Dict[int, int], busy: set, now: float) -> bool:
        if s in self.models:
            return True
        spec = self.specs[s]
        need = int(self.bytes_of(spec))
        if need > self.budget:
            raise ServingError(f"stream {s} needs {need} device bytes, above the budget {self.budget}")
        if not self._make_room(need, left, busy, now):
            return False
        m = self.factory(**spec)
        have = int(m.device_bytes()) if hasattr(m, "device_bytes") else need
        self.models[s] = m
        self.model_bytes[s] = max(have, need)
        self.resident += self.model_bytes[s]
        self.peak_resident = max(self.peak_resident, self.resident)
        self.events.append((now, "create", s))
        if self.prepare:
            self.prepare(s, m)
        return True

    # ---- issue ---------------------------------------------------------------
    @staticmethod
    def _issue(m, r: Request):
        ids, rp = np.asarray(r.slice_ids), np.asarray(r.row_ptr)
        if r.kind not in ("init", "update"):
            raise ValueError(f"unknown request kind {r.kind!r}")
        if getattr(r.X, "is_cuda", False):
            # a device-resident batch is read in place (no staging copy)
            if r.kind == "init":
                m.fit_initial_device(ids, rp, r.X, r.init_iters)
            else:
                m.update_device(ids, rp, r.X)
            return
        m.append_batch(ids, rp, r.X)
        if r.kind == "init":
            m.fit_initial(r.init_iters)
        else:
            m.update()

    # ---- the loop ------------------------------------------------------------
    def run(self, requests: List[Request], realtime: bool = True, final: bool = True) -> List[Request]:
        """Serve `requests` (any order; taken by arrival time, ties in list
        order).  realtime=False lets every request arrive at once (a burst),
        which keeps the admission order and makes the loop's work
        independent of the host's speed.  final=False keeps every model
        resident at the end (no retirement during this run), for streams
        whose later requests come in a later run; a request that does not
        fit then waits for room, and ServingError is raised if none can be
        made.  Returns the requests with their admission and completion times
        filled in."""
        self._final = final
        order = sorted(range(len(requests)), key=lambda i: (requests[i].arrival, i))
        pending = collections.deque(requests[i] for i in order)
        left: Dict[int, int] = collections.Counter(r.stream for r in requests)
        waiting: List[Request] = []
        inflight: Dict[int, Request] = {}          # stream -> its running request
        t0 = self._t0 = self.clock()
        while pending or waiting or inflight:
            now = self.clock() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            progressed = False
            # completions
            for s, r in list(inflight.items()):
                if self.models[s].idle():
                    r.done = self.clock() - t0
                    del inflight[s]
                    left[s] -= 1
                    self.events.append((r.done, "done", s))
                    progressed = True
            # admissions, in arrival order; a blocked stream keeps its later
            # requests waiting, other streams go ahead
            blocked = set()
            keep: List[Request] = []
            for r in waiting:
                s = r.stream
                if s in self.failed:                    # its stream stopped: not served
                    r.failed = self.failed[s]
                    left[s] -= 1
                    progressed = True
                    continue
                if (len(inflight) >= self.max_inflight or s in blocked or s in inflight
                        or not self._ensure_model(s, left, set(inflight), now)):
                    blocked.add(s)
                    keep.append(r)
                    continue
                r.admitted = self.clock() - t0
                try:
                    self._issue(self.models[s], r)
                except Exception as e:          # a stream's numerics failed: stop that stream only
                    if getattr(e, "status", None) != NUMERIC_FAILURE:
                        raise
                    self._fail_stream(s, str(e), r, pending, left, now)
                    blocked.add(s)
                    progressed = True
                    continue
                r.issue_s = self.clock() - t0 - r.admitted
                inflight[s] = r
                blocked.add(s)
                self.events.append((r.admitted, "admit", s))
                progressed = True
            waiting = keep
            if not progressed:
                if not inflight and not pending and waiting:
                    raise ServingError("requests left that can never be admitted")
                if self.poll_sleep:
                    time.sleep(self.poll_sleep)
        return requests

    def _fail_stream(self, s: int, why: str, r: Request, pending, left, now: float):
        """Mark stream s failed: this request and every later one of the
        stream are not served; its model is closed (its state is not
        trustworthy) and its memory released."""
        self.failed[s] = why
        r.failed = why
        left[s] -= 1
        for q in list(pending):
            if q.stream == s:
                q.failed = why
                left[s] -= 1
                pending.remove(q)
        m = self.models.pop(s)
        m.close()
        self.resident -= self.model_bytes.pop(s)
        self.events.append((now, "fail", s))

    def close(self):
        """Hand every resident model to on_retire, then free it."""
        now = self.clock() - self._t0
        for s in sorted(self.models):
            self._retire(s, now)


def latency_summary(requests: List[Request], kind: str = "update") -> dict:
    """p50/p99 latency (ms) and rows/s of the completed requests of a kind."""
    rs = [r for r in requests if r.kind == kind and r.done is not None]
    if not rs:
        return {"requests": 0}
    lat = np.array([r.latency for r in rs]) * 1e3
    span = max(r.done for r in rs) - min(r.arrival for r in rs)
    rows = sum(r.rows for r in rs)
    return {"requests": len(rs), "rows": rows, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "rows_per_s": rows / span if span > 0 else None,
            "span_s": span}
