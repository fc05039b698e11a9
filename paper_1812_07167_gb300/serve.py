"""Request loop over resident HPS solvers on one GPU: continuous batching of
solves and memory-admitted builds.

A built solver (Algorithm 1's output: the leaf operators and the per-merge
operators) stays resident in HBM.  A solve request (Algorithm 2 for its own
right-hand sides) joins its solver's queue.  Whenever that solver's stream
has a free slot, every queued request, in arrival order and up to
``max_batch_rhs`` right-hand sides, goes to the GPU as ONE
``hps_solve_batch`` call: the operators, which are the dominant bytes and
flops of Algorithm 2, are then read once per batch instead of once per
request.  Requests that arrive while a batch is on the GPU wait for the next
slot and are batched together there.

A build request is admitted when a build slot is free and the device has room
for the operators plus the build's transient scratch (``hps_plan``).  When it
has not, finished built solvers are released, oldest first, until it has; a
build that cannot fit even on an otherwise empty device fails with
``HPS_ENOMEM``.  Builds run on low-priority streams and solves on
high-priority streams, so their kernels share the GPU and the solves' blocks
are scheduled first.

A request's latency is the host time at which its batch's completion event
is first seen minus its arrival time.  The loop is a single host thread that
polls events; nothing in it blocks on the device.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Any, Callable, Optional

import numpy as np

from . import hps


@dataclass
class Request:
    """One solve (``kind == "solve"``: s [nrhs, leaves, (p-2)^2] and
    t [nrhs, 4 m (p-2)] against the resident solver ``key``) or one build
    (``kind == "build"``: ``problem`` and its c [leaves, (p-2)^2])."""
    rid: int
    arrival: float
    kind: str = "solve"
    key: Any = None
    s: Any = None
    t: Any = None
    nrhs: int = 0
    problem: Optional[hps.Problem] = None
    c: Any = None
    # written by the loop
    u: Any = None
    handle: Any = None
    launched: float = math.nan
    done: float = math.nan
    batch: int = -1
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def take_batch(queue: "collections.deque[Request]", max_rhs: int) -> list:
    """The next batch of a solver's queue: the head request always (even when
    it alone exceeds max_rhs), then the following ones in arrival order while
    the batch's right-hand sides stay within max_rhs."""
    out = [queue.popleft()]
    total = out[0].nrhs
    while queue and total + queue[0].nrhs <= max_rhs:
        r = queue.popleft()
        out.append(r)
        total += r.nrhs
    return out


class GpuBackend:
    """Device side of the loop: streams, events and the libhps calls."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)

    def solve_stream(self):
        return self.torch.cuda.Stream(device=self.dev, priority=-1)

    def build_stream(self):
        return self.torch.cuda.Stream(device=self.dev, priority=0)

    def free_bytes(self) -> int:
        return int(self.torch.cuda.mem_get_info(self.dev)[0])

    def build_bytes(self, problem: hps.Problem) -> int:
        info = hps.hps_plan(problem)
        return int(info.operator_bytes + info.build_scratch_bytes)

    def reserve(self, handle, nrhs: int):
        hps.hps_reserve(handle, nrhs)

    def launch_solves(self, handle, batch: list, stream):
        torch = self.torch
        pr = handle.pr
        with torch.cuda.stream(stream):
            for r in batch:
                r.u = torch.empty((r.nrhs, pr.leaves, pr.n), dtype=torch.complex128, device=self.dev)
        hps.hps_solve_batch(handle, [r.s for r in batch], [r.t for r in batch], [r.u for r in batch],
                            [r.nrhs for r in batch], stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    def launch_build(self, problem: hps.Problem, c, stream):
        h = hps.hps_build(problem, c, stream)
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return h, ev

    def build_status(self, handle, stream) -> int:
        return hps.hps_status(handle, stream)[0]

    def done(self, ev) -> bool:
        return ev.query()

    def release(self, handle):
        handle.free()


@dataclass
class _Solver:
    handle: Any
    stream: Any
    queue: "collections.deque[Request]" = field(default_factory=collections.deque)
    inflight: "collections.deque" = field(default_factory=collections.deque)  # (batch, event)


class Server:
    """The request loop.  ``add_solver`` makes a built handle resident under a
    key; ``run`` serves a list of requests in real time and returns them with
    their timings filled in (see ``summarize``)."""

    def __init__(self, backend=None, max_batch_rhs: int = 128, slots_per_solver: int = 1,
                 build_slots: int = 2, reserve_bytes: int = 2 << 30):
        self.be = backend if backend is not None else GpuBackend()
        self.max_rhs = int(max_batch_rhs)
        self.slots = int(slots_per_solver)
        self.reserve_bytes = int(reserve_bytes)
        self.solvers: dict = {}
        self.build_streams = [self.be.build_stream() for _ in range(int(build_slots))]
        self.built: "collections.OrderedDict[int, Any]" = collections.OrderedDict()
        self.batches = 0

    def add_solver(self, key, handle):
        self.be.reserve(handle, self.max_rhs)
        self.solvers[key] = _Solver(handle, self.be.solve_stream())

    def release_built(self):
        while self.built:
            _, h = self.built.popitem(last=False)
            self.be.release(h)

    # --- the loop ---------------------------------------------------------
    def run(self, requests: list, clock: Callable[[], float] = time.perf_counter,
            sleep: Callable[[float], None] = time.sleep, idle_s: float = 20e-6,
            on_done: Optional[Callable[[Request], None]] = None) -> list:
        """Serve ``requests`` (arrival times in seconds from now); ``on_done``
        is called with each request as its completion is seen."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if r.kind == "solve" and r.key not in self.solvers:
                raise KeyError(f"request {r.rid}: no resident solver {r.key!r}")
        build_q: "collections.deque[Request]" = collections.deque()
        building: dict = {}  # stream index -> (request, event)
        left = len(pending)
        i = 0
        t0 = clock()
        while left:
            now = clock() - t0
            busy = False
            while i < len(pending) and pending[i].arrival <= now:
                r = pending[i]
                i += 1
                (self.solvers[r.key].queue if r.kind == "solve" else build_q).append(r)
            # completions
            for sv in self.solvers.values():
                while sv.inflight and self.be.done(sv.inflight[0][1]):
                    batch, _ = sv.inflight.popleft()
                    t = clock() - t0
                    for r in batch:
                        r.done = t
                        if on_done:
                            on_done(r)
                    left -= len(batch)
                    busy = True
            for k in list(building):
                r, ev = building[k]
                if self.be.done(ev):
                    r.done = clock() - t0
                    code = self.be.build_status(r.handle, self.build_streams[k])
                    if code != hps.HPS_OK:
                        r.error = hps.hps_strerror(code)
                        self.be.release(r.handle)
                        r.handle = None
                    else:
                        self.built[r.rid] = r.handle
                    if on_done:
                        on_done(r)
                    del building[k]
                    left -= 1
                    busy = True
            # solve launches: every free slot takes the next batch
            for sv in self.solvers.values():
                while sv.queue and len(sv.inflight) < self.slots:
                    batch = take_batch(sv.queue, self.max_rhs)
                    t = clock() - t0
                    for r in batch:
                        r.launched = t
                        r.batch = self.batches
                    self.batches += 1
                    sv.inflight.append((batch, self.be.launch_solves(sv.handle, batch, sv.stream)))
                    busy = True
            # build admission: a free slot and room on the device
            while build_q and len(building) < len(self.build_streams):
                r = build_q[0]
                need = self.be.build_bytes(r.problem) + self.reserve_bytes
                while self.be.free_bytes() < need and self.built:
                    _, h = self.built.popitem(last=False)
                    self.be.release(h)
                if self.be.free_bytes() < need:
                    if building:
                        break  # wait for a build in flight to finish
                    build_q.popleft()
                    r.error = hps.hps_strerror(hps.HPS_ENOMEM)
                    r.done = clock() - t0
                    left -= 1
                    busy = True
                    continue
                build_q.popleft()
                k = next(j for j in range(len(self.build_streams)) if j not in building)
                r.launched = clock() - t0
                busy = True
                try:
                    r.handle, ev = self.be.launch_build(r.problem, r.c, self.build_streams[k])
                except hps.HPSError as exc:
                    # the free-memory estimate can be wrong either way (the
                    # allocator caches and pools): fail this request, keep serving
                    r.handle = None
                    r.error = hps.hps_strerror(exc.code)
                    r.done = clock() - t0
                    if on_done:
                        on_done(r)
                    left -= 1
                    continue
                building[k] = (r, ev)
            if not busy:
                sleep(idle_s)
        return requests


def summarize(requests: list) -> dict:
    """Throughput and latency percentiles of a served request list."""
    ok = [r for r in requests if r.error is None]
    solves = [r for r in ok if r.kind == "solve"]
    builds = [r for r in ok if r.kind == "build"]
    t_first = min(r.arrival for r in requests)
    span = max(r.done for r in requests) - t_first
    out = {
        "requests": len(requests),
        "solves": len(solves),
        "builds": len(builds),
        "failed": len(requests) - len(ok),
        "makespan_s": span,
        "req_per_s": len(requests) / span if span > 0 else math.inf,
        "rhs_per_s": sum(r.nrhs for r in solves) / span if span > 0 else math.inf,
    }
    for name, rs in (("solve", solves), ("build", builds)):
        if rs:
            lat = np.array([r.latency for r in rs]) * 1e3
            out[f"{name}_p50_ms"] = float(np.percentile(lat, 50))
            out[f"{name}_p99_ms"] = float(np.percentile(lat, 99))
    if solves:
        nb = len({r.batch for r in solves})
        out["batches"] = nb
        out["mean_batch_rhs"] = sum(r.nrhs for r in solves) / nb
    return out
