"""Host logic of the continuous-batching server, on the CPU: admission by table memory,
ticks pipelined one deep, and a retired session's table freed only after the tick holding
its last iteration has completed.  The device side is replaced by fakes that record what
the server asks of it (tables, batches, events)."""

import pytest

from paper_2005_07547_b300 import serve


class _Clock:
    """Device-completion order of the fake events: an event completes when synchronized or
    when a later event is synchronized (one stream)."""

    def __init__(self):
        self.recorded = []
        self.done_upto = -1


class FakeEvent:
    clock = None

    def __init__(self, enable_timing=False):
        self.index = None

    def record(self, stream=None):
        self.index = len(self.clock.recorded)
        self.clock.recorded.append(self)

    def synchronize(self):
        assert self.index is not None, "synchronizing an event that was never recorded"
        self.clock.done_upto = max(self.clock.done_upto, self.index)

    def done(self):
        return self.index is not None and self.index <= self.clock.done_upto

    def elapsed_time(self, other):
        return 0.5 * (other.index - self.index)


class FakeTable:
    live = []
    peak_bytes = 0

    def __init__(self, cfg):
        self.cfg = cfg
        self.nbytes = 1000 * cfg.log2_capacity
        self.closed = False
        self.last_event = None  # the end event of the tick that last used this table
        FakeTable.live.append(self)
        FakeTable.peak_bytes = max(FakeTable.peak_bytes, sum(t.nbytes for t in FakeTable.live))

    def close(self, synchronize=True):
        assert not self.closed
        if not synchronize:
            # the server must know the table's last work has completed
            assert self.last_event is not None and self.last_event.done(), "table freed while in flight"
        self.closed = True
        FakeTable.live.remove(self)

    # plain mode
    def insert_slots(self, v, P, D, slots=None):
        pass

    def update(self):
        pass

    def query_cv_slots(self, v, slots, P, D, out=None):
        pass

    def step(self, v, P, D, out=None):
        pass


class FakeBatch:
    def __init__(self, max_items, **knobs):
        self.entries = []

    def set(self, entries):
        self.entries = list(entries)

    def launch(self):
        pass

    def close(self):
        pass


def _requests(n, iters=3):
    return [dict(name=f"r{k}", arrival_s=0.0, width=8, height=4, depth=2, iterations=iters + (k % 3),
                 log2_capacity=8 + (k % 4), pos_bits=3, dir_bits=2, alpha_min=0.1, cache_fp16=False)
            for k in range(n)]


@pytest.fixture
def fakes(monkeypatch):
    import torch

    FakeEvent.clock = _Clock()
    FakeTable.live = []
    FakeTable.peak_bytes = 0
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(serve, "Table", FakeTable)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "table_bytes", lambda req, bits=None, key_layout=0: 1000 * req["log2_capacity"])
    yield


class _Server(serve.Server):
    """The server with host buffers and a hook that tags each table with its tick's end event."""

    def _empty(self, shape, dtype):
        import torch

        return torch.empty(shape, dtype=dtype)

    def _tick(self):
        sessions = list(self.live)
        super()._tick()
        end = self._inflight[-1][1][-1]  # this tick's end event (the pipeline keeps the newest tick)
        for s in sessions:
            s.table.last_event = end


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_every_session_runs_its_iterations_within_the_budget(fakes, mode):
    reqs = _requests(9)
    budget = 3 * 1000 * 11  # about three tables at a time
    seen = []
    srv = _Server(lambda req, it: None, budget_bytes=budget, mode=mode, use_graph=False,
                  on_retire=lambda s: seen.append((s.request["name"], s.done)))
    rep = srv.run(reqs, duration_s=5.0, drain=True)
    srv.close()
    assert rep["sessions_finished"] == len(reqs) and rep["requests_waiting_at_end"] == 0
    assert sorted(seen) == sorted((r["name"], r["iterations"]) for r in reqs)
    assert FakeTable.peak_bytes <= budget
    assert not FakeTable.live  # every table freed
    assert rep["iteration_latency_ms"]["p50"] is not None


def test_batched_ticks_carry_every_live_session_and_its_slots(fakes):
    reqs = _requests(4, iters=2)
    counts = []

    class Tracking(_Server):
        def _tick(self):
            super()._tick()
            counts.append([(e[0], len(e)) for e in self.batch.entries])

    srv = Tracking(lambda req, it: None, budget_bytes=1e12, mode="batched", use_graph=False)
    srv.run(reqs, duration_s=5.0, drain=True)
    srv.close()
    assert counts and all(n == 6 for tick in counts for _, n in tick)  # slot cache: 6-element entries
    assert len(counts[0]) == len(reqs)  # all admitted at once under an ample budget


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_tick_log_records_every_iteration_once(fakes, mode):
    """With log_ticks, every completed tick carries its device time and the (request,
    iteration, log2 capacity) of each session it ran: every iteration of every session
    appears exactly once, in order."""
    reqs = _requests(5)
    srv = _Server(lambda r, k: None, budget_bytes=1e9, mode=mode, use_graph=False, log_ticks=True)
    srv.run(reqs, duration_s=60.0, drain=True)
    assert len(srv.tick_log) == srv.ticks
    seen = {}
    for tick in srv.tick_log:
        assert tick["ms"] > 0
        for req, it, log2cap in tick["items"]:
            assert log2cap == req["log2_capacity"]
            assert it == seen.get(req["name"], -1) + 1
            seen[req["name"]] = it
    assert seen == {r["name"]: r["iterations"] - 1 for r in reqs}
