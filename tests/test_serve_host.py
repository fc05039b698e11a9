"""Host logic of the request loop (paper_1812_07167_gb300.serve) on a
simulated device: a virtual clock, streams that run their work in order, and
a memory account.  No GPU."""
import collections

import pytest

from paper_1812_07167_gb300 import hps, serve
from paper_1812_07167_gb300 import workloads as W


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class Stream:
    def __init__(self):
        self.free_at = 0.0


class Event:
    def __init__(self, t):
        self.t = t


class Handle:
    def __init__(self, nbytes):
        self.nbytes = nbytes
        self.alive = True


class FakeBackend:
    """Solves take a + b * (batch right-hand sides) on their stream; builds take
    build_s[m] and hold build_bytes[m] from launch until released."""

    def __init__(self, clock, total_bytes=100, a=1e-3, b=1e-4, build_s=None, build_bytes=None):
        self.clock = clock
        self.total = total_bytes
        self.a, self.b = a, b
        self.build_s = build_s or {16: 0.01, 32: 0.03, 64: 0.1}
        self.bytes = build_bytes or {16: 1, 32: 4, 64: 16}
        self.alive = []
        self.batch_rhs = []
        self.released = 0

    def solve_stream(self):
        return Stream()

    def build_stream(self):
        return Stream()

    def free_bytes(self):
        return self.total - sum(h.nbytes for h in self.alive)

    def build_bytes(self, problem):
        return self.bytes[problem.m]

    def reserve(self, handle, nrhs):
        pass

    def launch_solves(self, handle, batch, stream):
        rhs = sum(r.nrhs for r in batch)
        self.batch_rhs.append(rhs)
        start = max(self.clock(), stream.free_at)
        stream.free_at = start + self.a + self.b * rhs
        for r in batch:
            r.u = ("u", r.rid)
        return Event(stream.free_at)

    def launch_build(self, problem, c, stream):
        h = Handle(self.bytes[problem.m])
        self.alive.append(h)
        start = max(self.clock(), stream.free_at)
        stream.free_at = start + self.build_s[problem.m]
        return h, Event(stream.free_at)

    def build_status(self, handle, stream):
        return hps.HPS_OK

    def done(self, ev):
        return self.clock() >= ev.t

    def release(self, handle):
        handle.alive = False
        self.alive.remove(handle)
        self.released += 1


def _requests(rate, count=200, seed=4, **kw):
    out = []
    for k, d in enumerate(W.request_stream(seed, count, rate, **kw)):
        if d["kind"] == "solve":
            out.append(serve.Request(k, d["arrival"], "solve", key="main", nrhs=d["nrhs"]))
        else:
            out.append(serve.Request(k, d["arrival"], "build",
                                     problem=hps.Problem(d["m"], 16, d["kappa"], d["kappa"])))
    return out


def _serve(reqs, be, clock, **kw):
    kw.setdefault("reserve_bytes", 0)
    srv = serve.Server(be, **kw)
    srv.add_solver("main", Handle(0))
    srv.run(reqs, clock=clock, sleep=clock.sleep)
    return srv


def test_every_request_completes_once_in_order():
    clock = Clock()
    be = FakeBackend(clock)
    reqs = _requests(rate=300.0)
    srv = _serve(reqs, be, clock, max_batch_rhs=96)
    for r in reqs:
        assert r.error is None
        assert r.arrival <= r.launched <= r.done
    solves = sorted((r for r in reqs if r.kind == "solve"), key=lambda r: r.arrival)
    # arrival order is kept: batch ids never decrease along the arrivals
    assert all(a.batch <= b.batch for a, b in zip(solves, solves[1:]))
    # a batch exceeds the limit only when its single request does
    by_batch = collections.defaultdict(list)
    for r in solves:
        by_batch[r.batch].append(r)
    for rs in by_batch.values():
        assert sum(r.nrhs for r in rs) <= 96 or len(rs) == 1
    assert sorted(be.batch_rhs) == sorted(sum(r.nrhs for r in rs) for rs in by_batch.values())
    assert srv.batches == len(by_batch)


def test_requests_arriving_during_a_batch_share_the_next():
    clock = Clock()
    be = FakeBackend(clock, a=0.05, b=0.0)
    reqs = [serve.Request(k, 0.001 * k, "solve", key="main", nrhs=2) for k in range(10)]
    _serve(reqs, be, clock)
    # request 0 runs alone; requests 1..9 arrive during it and form one batch
    assert be.batch_rhs == [2, 18]
    assert len({r.batch for r in reqs[1:]}) == 1


def test_backlog_is_cut_at_the_batch_limit():
    clock = Clock()
    be = FakeBackend(clock)
    reqs = [serve.Request(k, 0.0, "solve", key="main", nrhs=10) for k in range(25)]
    _serve(reqs, be, clock, max_batch_rhs=64)
    assert be.batch_rhs == [60, 60, 60, 60, 10]


def test_idle_requests_see_only_their_service_time():
    clock = Clock()
    be = FakeBackend(clock, a=1e-3, b=1e-4)
    reqs = [serve.Request(k, 1.0 * k, "solve", key="main", nrhs=5) for k in range(5)]
    _serve(reqs, be, clock)
    for r in reqs:
        assert r.latency == pytest.approx(1e-3 + 5e-4, abs=1e-4)


def test_two_slots_pipeline_batches():
    clock = Clock()
    be = FakeBackend(clock, a=0.05, b=0.0)
    reqs = [serve.Request(k, 0.001 * k, "solve", key="main", nrhs=1) for k in range(3)]
    _serve(reqs, be, clock, slots_per_solver=2)
    # the second request goes out at once into the free slot
    assert be.batch_rhs == [1, 1, 1]


def test_builds_are_admitted_by_memory_with_eviction():
    clock = Clock()
    be = FakeBackend(clock, total_bytes=40)
    reqs = [serve.Request(k, 0.2 * k, "build", problem=hps.Problem(64, 16, 50.0, 50.0)) for k in range(4)]
    srv = _serve(reqs, be, clock, reserve_bytes=2)
    assert all(r.error is None for r in reqs)
    # 16 bytes each in 40 (2 reserved): the third and fourth builds evict the oldest
    assert be.released == 2
    assert [r.handle.alive for r in reqs] == [False, False, True, True]
    assert len(srv.built) == 2


def test_build_waits_for_memory_held_by_a_build_in_flight():
    clock = Clock()
    be = FakeBackend(clock, total_bytes=20)
    reqs = [serve.Request(0, 0.0, "build", problem=hps.Problem(64, 16, 50.0, 50.0)),
            serve.Request(1, 0.0, "build", problem=hps.Problem(32, 16, 50.0, 50.0))]
    _serve(reqs, be, clock, reserve_bytes=1)
    a, b = reqs
    assert a.error is None and b.error is None
    assert b.launched >= a.done  # admitted only once the first finished and was evicted


def test_build_larger_than_the_device_fails_with_enomem():
    clock = Clock()
    be = FakeBackend(clock, total_bytes=10)
    reqs = [serve.Request(0, 0.0, "build", problem=hps.Problem(64, 16, 50.0, 50.0)),
            serve.Request(1, 0.0, "solve", key="main", nrhs=3)]
    _serve(reqs, be, clock)
    assert reqs[0].error == hps.hps_strerror(hps.HPS_ENOMEM)
    assert reqs[1].error is None


class FailingBuildBackend(FakeBackend):
    """launch_build raises for problems of size fail_m, as hps_build does when
    its arena allocation fails although the free-memory estimate admitted it."""

    def __init__(self, clock, fail_m, **kw):
        super().__init__(clock, **kw)
        self.fail_m = fail_m

    def launch_build(self, problem, c, stream):
        if problem.m == self.fail_m:
            raise hps.HPSError(hps.HPS_ENOMEM, "hps_build")
        return super().launch_build(problem, c, stream)


def test_failed_build_launch_fails_only_its_request():
    clock = Clock()
    be = FailingBuildBackend(clock, fail_m=32)
    reqs = [serve.Request(0, 0.0, "build", problem=hps.Problem(32, 16, 50.0, 50.0)),
            serve.Request(1, 0.0, "solve", key="main", nrhs=3),
            serve.Request(2, 0.001, "build", problem=hps.Problem(16, 16, 50.0, 50.0)),
            serve.Request(3, 0.002, "solve", key="main", nrhs=1)]
    seen = []
    srv = serve.Server(be, reserve_bytes=0)
    srv.add_solver("main", Handle(0))
    srv.run(reqs, clock=clock, sleep=clock.sleep, on_done=seen.append)
    bad, s1, good, s2 = reqs
    assert bad.error == hps.hps_strerror(hps.HPS_ENOMEM) and bad.handle is None
    assert bad.done >= bad.launched
    assert good.error is None and good.handle is not None and good.handle.alive
    assert s1.error is None and s2.error is None and s1.u is not None and s2.u is not None
    # every request completed exactly once
    assert sorted(r.rid for r in seen) == [0, 1, 2, 3]


def test_unknown_solver_is_refused():
    clock = Clock()
    srv = serve.Server(FakeBackend(clock))
    with pytest.raises(KeyError):
        srv.run([serve.Request(0, 0.0, "solve", key="nope", nrhs=1)], clock=clock, sleep=clock.sleep)


def test_summary_counts_and_percentiles():
    clock = Clock()
    be = FakeBackend(clock, a=1e-3, b=0.0)
    reqs = [serve.Request(k, 1.0 * k, "solve", key="main", nrhs=k + 1) for k in range(4)]
    _serve(reqs, be, clock)
    s = serve.summarize(reqs)
    assert s["requests"] == 4 and s["solves"] == 4 and s["builds"] == 0 and s["failed"] == 0
    assert s["batches"] == 4 and s["mean_batch_rhs"] == pytest.approx(2.5)
    assert s["solve_p50_ms"] == pytest.approx(1.0, abs=0.05)
    assert s["makespan_s"] == pytest.approx(3.001, abs=1e-3)


def test_request_stream_mix_and_rate():
    rs = W.request_stream(4, 4000, 5.0)
    gaps = [b["arrival"] - a["arrival"] for a, b in zip(rs, rs[1:])]
    assert sum(gaps) / len(gaps) == pytest.approx(0.2, rel=0.05)
    solves = [r for r in rs if r["kind"] == "solve"]
    assert len(solves) / len(rs) == pytest.approx(0.9, abs=0.02)
    assert min(r["nrhs"] for r in solves) == 1 and max(r["nrhs"] for r in solves) == 64
    assert {r["m"] for r in rs if r["kind"] == "build"} == {16, 32, 64}
    # the same requests at another load, only the arrival times scale
    rs2 = W.request_stream(4, 4000, 10.0)
    assert [(a["kind"], a["nrhs"], a["m"]) for a in rs] == [(b["kind"], b["nrhs"], b["m"]) for b in rs2]
    assert rs2[100]["arrival"] == pytest.approx(rs[100]["arrival"] / 2)
