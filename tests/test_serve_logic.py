"""Host logic of the serving loop, with fake channels, streams and events (no GPU)."""
import numpy as np

from paper_1808_06461_b300.serve import Request, Server, poisson_requests, serving_dt


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances it: the loop always makes progress
        return self.t


class FakeStream:
    def __init__(self, clock):
        self.clock, self.busy_until = clock, 0.0


class FakeEvent:
    def __init__(self, clock):
        self.clock, self.t = clock, None

    def record(self, stream):
        self.t = max(stream.busy_until, self.clock.t)

    def query(self):
        return self.clock.t >= self.t

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class FakeChannel:
    live = 0
    peak = 0

    def __init__(self, r, stream, clock):
        self.r, self.stream, self.clock, self.steps = r, stream, clock, 0
        FakeChannel.live += 1
        FakeChannel.peak = max(FakeChannel.peak, FakeChannel.live)

    def step(self, k):
        self.steps += k
        self.stream.busy_until = max(self.stream.busy_until, self.clock.t) + 1e-3 * k

    def get_state(self):
        return dict(steps=self.steps, rid=self.r.rid)

    def close(self):
        FakeChannel.live -= 1


def _server(budget, slots, clock, log):
    def factory(r, stream):
        log.append(("admit", r.rid, clock.t))
        return FakeChannel(r, stream, clock)
    return Server(budget, max_slots=slots, factory=factory, footprint=lambda r: r.Nx * r.Ny * r.Nz,
                  make_stream=lambda: FakeStream(clock), make_event=lambda: FakeEvent(clock), clock=clock,
                  idle_sleep=0.0)


def test_every_request_completes_with_all_its_substeps():
    clock, log = Clock(), []
    reqs = poisson_requests(20, rate=50.0, seed=42, length=(10, 40))
    res, m = _server(10 ** 9, 4, clock, log).run(reqs)
    assert sorted(res) == [r.rid for r in reqs]
    for r in reqs:
        assert res[r.rid]["steps"] == r.nsub
    assert m["requests"] == 20 and m["step_ms_p50"] is not None and m["step_ms_p99"] >= m["step_ms_p50"]


def test_admission_respects_slots_budget_and_arrivals():
    clock, log = Clock(), []
    FakeChannel.live = FakeChannel.peak = 0
    reqs = [Request(i, 0.01 * i, 180.0, 3.1, 1.5, 32, 49, 32, 1e-3, 30, i) for i in range(12)]
    budget = 3 * 32 * 49 * 32           # room for three runs at a time
    res, m = _server(budget, 8, clock, log).run(reqs)
    assert FakeChannel.peak <= 3 and m["max_concurrency"] <= 3
    for _, rid, t in log:
        assert t >= reqs[rid].t_arrival - 1e-12   # never admitted before it arrived
    assert len(res) == 12
    FakeChannel.live = FakeChannel.peak = 0
    res, m = _server(10 ** 9, 2, Clock(), []).run(reqs)
    assert m["max_concurrency"] <= 2 and FakeChannel.peak <= 2


def test_oversized_request_is_rejected():
    clock = Clock()
    r = Request(0, 0.0, 180.0, 3.1, 1.5, 128, 129, 128, 1e-3, 30, 0)
    try:
        _server(1000, 2, clock, []).run([r])
    except ValueError as e:
        assert "budget" in str(e)
    else:
        raise AssertionError("expected a ValueError")


def test_serving_mix_and_dt():
    reqs = poisson_requests(50, rate=50.0, seed=42)
    gaps = np.diff([r.t_arrival for r in reqs])
    assert 0.01 < gaps.mean() < 0.04                      # mean 1/50 s
    assert {r.re_tau for r in reqs} <= {180.0, 395.0, 550.0}
    assert {r.Nx for r in reqs} <= {32, 64, 128} and {r.Ny for r in reqs} <= {49, 97, 129}
    assert all(100 <= r.nsub <= 2000 for r in reqs)
    assert all(0 < r.dt <= 1e-3 for r in reqs)
    assert serving_dt(180.0, np.pi, np.pi / 2, 32, 32) <= 1e-3
    again = poisson_requests(50, rate=50.0, seed=42)
    assert [(r.Nx, r.Ny, r.nsub) for r in again] == [(r.Nx, r.Ny, r.nsub) for r in reqs]


class FakeBatch:
    built = 0

    def __init__(self, chans, stream):
        self.chans, self.stream = chans, stream
        FakeBatch.built += 1

    def step(self, k):
        for ch in self.chans:
            ch.steps += k
        self.stream.busy_until = max(self.stream.busy_until, self.stream.clock.t) + 1e-3 * k

    def close(self):
        pass


def test_packed_mode_completes_every_run_exactly():
    clock, log = Clock(), []
    reqs = poisson_requests(15, rate=50.0, seed=3, length=(10, 40))
    srv = _server(10 ** 9, 6, clock, log)
    srv.packed = True
    srv.make_batch = lambda chans, stream: FakeBatch(chans, stream)
    res, m = srv.run(reqs)
    for r in reqs:
        assert res[r.rid]["steps"] == r.nsub      # packed steps plus the per-run tail add up
    assert m["packed"] and m["batches_built"] >= 1


def test_a_slow_set_up_does_not_stall_the_other_runs():
    """Admission builds the run on the set-up thread: while a slow factory call is under
    way, the loop keeps issuing steps of the runs already active."""
    import threading
    import time as _time
    clock = Clock()
    gate = threading.Event()
    issued_while_building = []

    class Tracked(FakeChannel):
        def step(self, k):
            if gate.is_set():
                issued_while_building.append(self.r.rid)
            super().step(k)

    def factory(r, stream):
        if r.rid == 1:           # the second run takes a while to build
            gate.set()
            _time.sleep(0.05)
            gate.clear()
        return Tracked(r, stream, clock)

    reqs = [Request(i, 0.0, 180.0, 3.1, 1.5, 32, 49, 32, 1e-3, 3000, i) for i in range(2)]
    srv = Server(10 ** 9, max_slots=2, factory=factory, footprint=lambda r: 1,
                 make_stream=lambda: FakeStream(clock), make_event=lambda: FakeEvent(clock), clock=clock,
                 idle_sleep=0.0)
    res, m = srv.run(reqs)
    assert 0 in issued_while_building
    assert res[0]["steps"] == res[1]["steps"] == 3000 and m["setup_threads"] == 1


def test_retired_runs_drop_their_packed_batches():
    clock, log = Clock(), []
    closed = []

    class ClosingBatch(FakeBatch):
        def close(self):
            closed.append(tuple(ch.r.rid for ch in self.chans))

    reqs = poisson_requests(12, rate=50.0, seed=5, length=(10, 60))
    srv = _server(10 ** 9, 4, clock, log)
    srv.packed = True
    srv.make_batch = lambda chans, stream: ClosingBatch(chans, stream)
    res, m = srv.run(reqs)
    assert len(closed) == m["batches_built"]            # every batch is closed exactly once
    assert all(res[r.rid]["steps"] == r.nsub for r in reqs)


class FakeEachBatch(FakeBatch):
    """A persistent batch: run r advances by its own count; at most 16 runs."""

    def __init__(self, chans, stream):
        assert len(chans) <= 16
        super().__init__(chans, stream)

    def step_each(self, ks):
        assert len(ks) == len(self.chans) and all(k >= 0 for k in ks)
        for ch, k in zip(self.chans, ks):
            ch.steps += k
        self.stream.busy_until = max(self.stream.busy_until, self.stream.clock.t) + 1e-3 * max(ks)


def test_persistent_mode_completes_every_run_exactly_and_never_steps_a_run_alone():
    clock, log = Clock(), []
    reqs = poisson_requests(40, rate=50.0, seed=5, length=(10, 100))
    srv = _server(10 ** 9, 20, clock, log)
    srv.packed, srv.batch_runs, srv.persist_chunk = "persistent", 16, 12
    srv.make_batch = lambda chans, stream: FakeEachBatch(chans, stream)
    inner = srv.factory

    def no_solo_steps(r, stream):
        ch = inner(r, stream)
        ch.step = None     # a run of a persistent server is only ever stepped by its batch
        return ch
    srv.factory = no_solo_steps
    res, m = srv.run(reqs)
    for r in reqs:
        assert res[r.rid]["steps"] == r.nsub      # whole and partial chunks add up in the launches
    assert m["packed"] == "persistent" and m["batches_built"] >= 2 and m["max_concurrency"] >= 2
