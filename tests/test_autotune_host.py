"""The autotuner's search on the CPU: every candidate of the space is timed on a fresh
scratch table and the fastest is returned (fake tables and timer events give each knob
setting a known cost)."""

import pytest

from paper_2005_07547_b300 import _abi, autotune


class _Events:
    """A timer whose elapsed time between two records is the cost the current table charged."""

    now = 0.0

    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = _Events.now

        def elapsed_time(self, other):
            return other.t - self.t


class FakeTable:
    closed = []

    def __init__(self, cfg):
        self.cfg = cfg
        self.knobs = {}
        self.nbytes = 64 << cfg.log2_capacity

    def set_launch(self, **knobs):
        self.knobs = knobs

    def step(self, verts, P, D, out=None):
        k = self.knobs
        cost = 10.0 + 3.0 * k.get("insert_mode", 0) + 2.0 * (k.get("vertex_staging", 0) & 1) \
            + (1.0 if k.get("sum_reduction", 0) else 0.0) + 0.5 * abs(k.get("insert_blocks_per_sm", 0) - 4) \
            + 0.25 * abs(self.cfg.log2_capacity - 9) + (0.0 if self.cfg.key_layout == 2 else 0.75)
        if "key_layout" in k:
            raise AssertionError("the key layout is a table field, not a launch knob")
        _Events.now += cost

    def stats(self):
        return {"max_probe": 1}

    def close(self):
        FakeTable.closed.append(self)


@pytest.fixture
def fakes(monkeypatch):
    import torch

    monkeypatch.setattr(torch.cuda, "Event", _Events.Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch, "empty", lambda *a, **k: None)
    monkeypatch.setattr(autotune, "Table", FakeTable)
    FakeTable.closed = []
    yield


class _Batch:
    def __init__(self):
        self.device = "cpu"


def test_tune_table_returns_the_fastest_candidate(fakes):
    cfg = _abi.make_config(log2_capacity=9)
    space = {"insert_mode": (1, 0), "vertex_staging": (1, 0), "sum_reduction": (1, 0),
             "insert_blocks_per_sm": (0, 4, 2)}
    res = autotune.tune_table(cfg, [_Batch()], P=4, D=2, space=space, warmup=1, iters=3)
    assert res["best"] == {"insert_mode": 0, "vertex_staging": 0, "sum_reduction": 0, "insert_blocks_per_sm": 4}
    assert res["best_ms"] == pytest.approx(10.75)
    assert len(res["all"]) == 2 * 2 * 2 * 3 == len(FakeTable.closed)  # each candidate on its own table
    assert [r["ms"] for r in res["all"]] == sorted(r["ms"] for r in res["all"])


def test_tune_capacity_times_each_load_factor(fakes):
    cfg = _abi.make_config(log2_capacity=16)
    res = autotune.tune_capacity(cfg, [_Batch()], P=100, D=2, extra_bits=(0, 1, 2), warmup=1, iters=2)
    # V = 200 -> ceil(log2 V) = 8; the fake cost is lowest at 2^9 slots
    assert [r["log2_capacity"] for r in res["all"]] == [8, 9, 10]
    assert res["best"] == 9


def test_tune_table_lays_out_a_table_per_key_layout(fakes):
    """A table field in the space reaches the candidate's table configuration, not its launch
    knobs, and is reported with the candidate."""
    cfg = _abi.make_config(log2_capacity=9)
    res = autotune.tune_table(cfg, [_Batch()], P=4, D=2, space={"key_layout": (1, 2), "insert_mode": (1, 0)},
                              warmup=1, iters=2)
    assert res["best"] == {"key_layout": 2, "insert_mode": 0}
    assert sorted(t.cfg.key_layout for t in FakeTable.closed) == [1, 1, 2, 2]
    assert cfg.key_layout == 0  # the caller's configuration is left as it was


def test_tune_batch_passes_table_fields_by_name(fakes, monkeypatch):
    calls = []

    class FakeBatch:
        def __init__(self, n, **knobs):
            self.knobs = knobs

        def set(self, entries):
            self.entries = entries

        def launch(self):
            f = self.entries[0][0]
            _Events.now += 5.0 + f["capacity_bits"] + (0.0 if f["key_layout"] == 2 else 1.0) + self.knobs["insert_mode"]

        def status(self):
            return 0

        def close(self):
            pass

    class _T:
        def __init__(self, fields):
            self.fields = fields

        def __getitem__(self, k):
            return self.fields[k]

        def close(self):
            pass

    def make(capacity_bits=1, key_layout=0):
        calls.append((capacity_bits, key_layout))
        return [(_T({"capacity_bits": capacity_bits, "key_layout": key_layout}),)]

    monkeypatch.setattr(autotune, "Batch", FakeBatch)
    res = autotune.tune_batch(make, 1, space={"insert_mode": (1, 0), "capacity_bits": (2, 1), "key_layout": (1, 2)},
                              warmup=1, iters=2)
    assert res["best"] == {"insert_mode": 0, "capacity_bits": 1, "key_layout": 2}
    assert sorted(set(calls)) == [(1, 1), (1, 2), (2, 1), (2, 2)] and len(calls) == 8
