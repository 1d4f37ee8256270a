"""Continuous-batching server for render sessions.

Requests (render sessions: image size, path depth, number of iterations) arrive over
time.  Each server tick:

  1. admits queued requests, first come first served, while their tables fit the
     device-memory budget and a batch slot is free (a new session's table is created
     in caller-owned memory and lives on the device until the session retires);
  2. runs ONE iteration of every live session: in "batched" mode a single fused
     persistent kernel for all of them (captured once in a CUDA graph and replayed;
     joins and leaves only rewrite the device descriptors), in "plain" mode one
     psf_step per session, back to back;
  3. retires sessions that reached their iteration count.

Ticks are pipelined one deep in both modes: the host prepares and enqueues tick k+1 while
the device runs tick k, and waits only for tick k-1's completion event, so the device does
not idle while the host builds descriptors, admits or retires.  A retired session's table
is freed once the tick holding its last iteration has completed (psf_destroy makes no CUDA
call, so freeing never waits on the device); its memory counts against the budget until
then.  A session's iterations are ordered on the one stream.  Per-iteration latency is the
device time from the start of a tick to the completion of that session's iteration;
admission delay is the time from arrival to admission.  Every session's results are
independent of who else is in the batch.
"""

from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from .batch import Batch
from .table import Table


@dataclass
class Session:
    request: dict
    table: Table
    out: object
    P: int
    D: int
    arrival: float
    admitted: float
    slots: object = None  # the session's slot cache (int32, P*D), or None
    done: int = 0
    latencies_ms: list = field(default_factory=list)


def table_config(req: dict, capacity_bits: int | None = None, key_layout: int = 0) -> _abi.Config:
    """A request's table: its own log2_capacity, or with capacity_bits (the load factor an
    autotuner chose) 2^(ceil(log2 V) + capacity_bits) slots for its V vertices per iteration;
    the cell grid is the request's either way; key_layout as in psf_config (0: the library's
    rule, 1: a dense key array, 2: keys inside the slot records)."""
    log2cap = req["log2_capacity"]
    if capacity_bits is not None:
        log2cap = max(4, int(math.ceil(math.log2(max(2, req["width"] * req["height"] * req["depth"]))))
                      + capacity_bits)
    return _abi.make_config(log2_capacity=log2cap, pos_bits=req["pos_bits"], dir_bits=req["dir_bits"],
                            alpha_min=req["alpha_min"], cache_fp16=req.get("cache_fp16", True), key_layout=key_layout)


def table_bytes(req: dict, capacity_bits: int | None = None, key_layout: int = 0) -> int:
    import ctypes

    return int(_abi.load().psf_table_bytes(ctypes.byref(table_config(req, capacity_bits, key_layout))))


class Server:
    def __init__(self, vertex_source, budget_bytes: float = 60e9, max_live: int = _abi.MAX_BATCH,
                 mode: str = "batched", use_graph: bool = True, batch_knobs: dict | None = None,
                 on_retire=None, slot_cache: bool = True, capacity_bits: int | None = None,
                 log_ticks: bool = False, key_layout: int = 0):
        """vertex_source(request, iteration) -> (P*D, 16) float32 CUDA tensor of that iteration;
        on_retire(session), if given, sees each session (table still open) before it is freed;
        slot_cache: each session's insert notes its vertices' slots and its query reads them
        (psf_insert_slots / psf_query_cv_slots, or the batch item's slots), in both modes;
        capacity_bits: each session's table gets 2^(ceil(log2 V) + capacity_bits) slots (the
        load factor, e.g. autotune.tune_batch's choice) instead of its request's log2_capacity;
        key_layout: where each session's table keeps its keys (psf_config.key_layout, e.g. the
        tuner's choice);
        log_ticks: keep, per completed tick, its device time and the (request, iteration, log2
        capacity) of every session it ran (`tick_log`, for a roofline of the served form)."""
        if mode not in ("batched", "plain"):
            raise ValueError("mode must be 'batched' or 'plain'")
        self.source = vertex_source
        self.budget = float(budget_bytes)
        self.max_live = min(max_live, _abi.MAX_BATCH)
        self.mode = mode
        self.use_graph = use_graph and mode == "batched"
        self.batch = Batch(self.max_live, **(batch_knobs or {})) if mode == "batched" else None
        self.graph = None
        self.live: list[Session] = []
        self.used = 0
        self.finished: list[Session] = []
        self.ticks = 0
        self.vertices = 0
        self.admission_ms: list[float] = []
        self.on_retire = on_retire
        self.slot_cache = slot_cache
        self.capacity_bits = capacity_bits
        self.key_layout = key_layout
        self._inflight: deque = deque()  # (start event, end event(s), sessions, retiring sessions, items)
        self.tick_log: list | None = [] if log_ticks else None

    # -- membership ---------------------------------------------------------------------
    def _admit(self, queue: deque, now: float) -> bool:
        import torch

        changed = False
        while queue and len(self.live) < self.max_live:
            req = queue[0]
            need = table_bytes(req, self.capacity_bits, self.key_layout)
            if self.used + need > self.budget:
                break
            queue.popleft()
            P, D = req["width"] * req["height"], req["depth"]
            t = Table(table_config(req, self.capacity_bits, self.key_layout))
            out = self._empty((P * D, 3), torch.float32)
            slots = self._empty((P * D,), torch.int32) if self.slot_cache else None
            self.live.append(Session(req, t, out, P, D, req["arrival_s"], now, slots))
            self.used += t.nbytes
            self.admission_ms.append(1e3 * (now - req["arrival_s"]))
            changed = True
        return changed

    def _empty(self, shape, dtype):
        """A session's device buffer (outputs, slot cache)."""
        import torch

        return torch.empty(shape, dtype=dtype, device="cuda")

    def _retire(self) -> list:
        """Sessions that have had their last iteration enqueued leave the live set (their
        tables are freed once that iteration has completed)."""
        keep, done = [], []
        for s in self.live:
            (done if s.done >= s.request["iterations"] else keep).append(s)
        self.live = keep
        return done

    def _complete(self, keep: int) -> None:
        """Wait for all but the newest `keep` ticks; record their latencies and free the
        tables of the sessions they retired."""
        while len(self._inflight) > keep:
            start, ends, sessions, retiring, items = self._inflight.popleft()
            ends[-1].synchronize()
            if self.tick_log is not None:
                self.tick_log.append({"ms": start.elapsed_time(ends[-1]), "items": items})
            for s, e in zip(sessions, ends if len(ends) == len(sessions) else [ends[-1]] * len(sessions)):
                s.latencies_ms.append(start.elapsed_time(e))
            for s in retiring:
                if self.on_retire is not None:
                    self.on_retire(s)
                self.used -= s.table.nbytes
                s.table.close(synchronize=False)  # its last iteration has completed
                s.out = None
                s.slots = None
                self.finished.append(s)

    # -- one iteration of every live session ---------------------------------------------
    def _entries(self):
        return [(s.table, self.source(s.request, s.done), s.out, s.P, s.D) + ((s.slots,) if s.slots is not None else ())
                for s in self.live]

    def _tick(self) -> None:
        import torch

        start = torch.cuda.Event(enable_timing=True)
        sessions = list(self.live)
        if self.mode == "batched":
            end = torch.cuda.Event(enable_timing=True)
            # the descriptors point at each session's input of its current iteration (the copy
            # is ordered after the previous tick's kernel on the stream)
            self.batch.set(self._entries())
            if self.use_graph and self.graph is None:
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self.batch.launch()
            start.record()
            if self.use_graph:
                self.graph.replay()
            else:
                self.batch.launch()
            end.record()
            ends = [end]
        else:
            ends = []
            start.record()
            for s in sessions:
                v = self.source(s.request, s.done)
                if s.slots is not None:
                    s.table.insert_slots(v, s.P, s.D, slots=s.slots)
                    s.table.update()
                    s.table.query_cv_slots(v, s.slots, s.P, s.D, out=s.out)
                else:
                    s.table.step(v, s.P, s.D, out=s.out)
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                ends.append(e)
        items = [(s.request, s.done, int(s.table.cfg.log2_capacity)) for s in sessions] \
            if self.tick_log is not None else None
        for s in sessions:
            s.done += 1
            self.vertices += s.P * s.D
        self.ticks += 1
        self._inflight.append((start, ends, sessions, self._retire(), items))
        self._complete(keep=1)

    # -- driver ---------------------------------------------------------------------------
    def run(self, requests: list[dict], duration_s: float, drain: bool = False) -> dict:
        """Serve `requests` (sorted by arrival_s) for duration_s of wall time (then optionally
        until every admitted session has finished).  Returns the report."""
        pending = deque(sorted(requests, key=lambda r: r["arrival_s"]))
        queue: deque = deque()
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while pending and pending[0]["arrival_s"] <= now:
                queue.append(pending.popleft())
            if now < duration_s:
                self._admit(queue, now)
            elif not drain or not self.live:
                break
            if not self.live:
                self._complete(keep=0)
                if not pending:
                    break
                time.sleep(max(0.0, min(pending[0]["arrival_s"] - now, 0.01)))
                continue
            self._tick()
        self._complete(keep=0)
        wall = time.perf_counter() - t0
        lat = [x for s in self.finished + self.live for x in s.latencies_ms]
        report = {
            "mode": self.mode, "graph": self.use_graph, "wall_s": wall, "ticks": self.ticks,
            "vertices": self.vertices, "vertices_per_s": self.vertices / wall if wall > 0 else 0.0,
            "sessions_finished": len(self.finished), "sessions_live_at_end": len(self.live),
            "requests_waiting_at_end": len(queue) + len(pending),
            "iteration_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat else None,
                                     "p99": float(np.percentile(lat, 99)) if lat else None},
            "admission_delay_ms": {"p50": float(np.percentile(self.admission_ms, 50)) if self.admission_ms else None,
                                   "p99": float(np.percentile(self.admission_ms, 99)) if self.admission_ms else None},
            "peak_table_bytes_budget": self.budget,
        }
        return report

    def close(self) -> None:
        self._complete(keep=0)
        for s in self.live:
            s.table.close()
        self.live = []
        if self.batch is not None:
            self.batch.close()
        self.graph = None
