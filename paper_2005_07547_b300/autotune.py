"""Autotuner for the launch knobs and the table load factor.

Every knob changes only the order of the integer additions (or the table's slot
layout), never a result, so candidates are timed on scratch tables fed the caller's
own device-resident vertex batches and the fastest is returned.  Timing uses CUDA
events on the current stream after warm-up iterations.  With verify=True the tuner also
checks that premise: every candidate has run the same iterations, and its tables' cell
maps (exported in key order) must be identical, bit for bit.

  tune_table(cfg, batches, P, D)   -> insert mode, vertex staging, sum path and per-kernel
                                      grid caps for psf_step, and, when the space holds
                                      "key_layout", where the table keeps its keys
  tune_capacity(cfg, batches, P, D)-> log2 capacity (load factor) for a session size
  tune_batch(make_entries, n)      -> insert mode, blocks/SM and, when the space holds
                                      "capacity_bits" / "key_layout", the sessions' load
                                      factor (2^(ceil(log2 V) + bits) slots) and key layout
                                      for the batched kernel

The probe window is not a knob: every probe visits one slot per step.  Windows of two and
four consecutive slots per step were measured on the B300 (1280x720, depth 4: 117 and
143 us against 112 us for the insert) and lost to the extra loads and registers.  The block
shape is searched as the grid: resident blocks per SM per kernel (the *_blocks_per_sm knobs)
set each kernel's resident warps; the threads per block stay 256, since 128-thread blocks
with retuned caps were measured slower (1920x1080: blend 144 -> 152 us, query 202 -> 213 us;
64 sessions 13.9 -> 13.6 G vertices/s).
"""

from __future__ import annotations

import ctypes
import itertools
import math

from . import _abi
from .batch import Batch
from .table import Table

TABLE_SPACE = {
    "vertex_staging": (0, 1, 2, 3),
    "sum_reduction": (0, 1),
    "insert_mode": (0, 1),
    "insert_blocks_per_sm": (0, 4, 2),
    "query_blocks_per_sm": (0, 4),
    "update_blocks_per_sm": (0, 2),
    "query_layout": (0, 1),
}
BATCH_SPACE = {"insert_mode": (0, 1), "blocks_per_sm": (0, 3, 2), "update_blocks_per_sm": (0, 2),
               "query_blocks_per_sm": (0, 2)}

# Fields of the table configuration a search space may hold beside the launch knobs: they lay
# the table out differently (1: a dense key array, 2: keys inside the slot records), so each
# candidate gets its own table; results do not depend on them either.
CONFIG_KNOBS = ("key_layout",)


def _split(knobs: dict) -> tuple[dict, dict]:
    """(table-config fields, launch knobs) of a candidate."""
    conf = {k: v for k, v in knobs.items() if k in CONFIG_KNOBS}
    return conf, {k: v for k, v in knobs.items() if k not in CONFIG_KNOBS}


def _time_ms(fn, iters: int) -> float:
    import torch

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    for k in range(iters):
        fn(k)
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / iters


def _clone_config(cfg: _abi.Config, **over) -> _abi.Config:
    c = _abi.Config()
    ctypes.memmove(ctypes.byref(c), ctypes.byref(cfg), ctypes.sizeof(cfg))
    for k, v in over.items():
        setattr(c, k, v)
    return c


class _Same:
    """Holds the first candidate's exported tables and checks every later one against them."""

    def __init__(self, enabled: bool):
        self.enabled = enabled
        self.ref = None
        self.checked = 0

    def __call__(self, tables, knobs) -> None:
        if not self.enabled:
            return
        got = [t.export().tobytes() for t in tables]
        if self.ref is None:
            self.ref = got
        elif got != self.ref:
            raise AssertionError(f"autotune: candidate {knobs} changed the tables")
        self.checked += 1


def tune_table(cfg: _abi.Config, batches, P: int, D: int, space: dict | None = None, warmup: int = 2,
               iters: int = 4, verify: bool = False, slot_cache: bool = False) -> dict:
    """Fastest launch knobs of one iteration (psf_step, or with slot_cache the slot-cache insert,
    the blend and the slot-cache query) for this configuration and input (list of (P*D, 16)
    tensors)."""
    import torch

    space = space or TABLE_SPACE
    out = torch.empty((P * D, 3), dtype=torch.float32, device=batches[0].device)
    slots = torch.empty(P * D, dtype=torch.int32, device=batches[0].device) if slot_cache else None
    results = []
    same = _Same(verify)
    keys = list(space)

    def step(t, v):
        if slots is None:
            t.step(v, P, D, out=out)
        else:
            t.insert_slots(v, P, D, slots=slots)
            t.update()
            t.query_cv_slots(v, slots, P, D, out=out)

    for values in itertools.product(*(space[k] for k in keys)):
        knobs = dict(zip(keys, values))
        conf, launch = _split(knobs)
        t = Table(_clone_config(cfg, **conf) if conf else cfg)
        t.set_launch(**launch)
        for k in range(warmup):
            step(t, batches[k % len(batches)])
        ms = _time_ms(lambda k: step(t, batches[(warmup + k) % len(batches)]), iters)
        same([t], knobs)
        t.close()
        results.append((ms, knobs))
    results.sort(key=lambda r: r[0])
    return {"best": results[0][1], "best_ms": results[0][0], "all": [{"ms": ms, **k} for ms, k in results],
            "verified": same.checked}


def tune_capacity(cfg: _abi.Config, batches, P: int, D: int, extra_bits=(1, 2), warmup: int = 2,
                  iters: int = 4, verify: bool = False) -> dict:
    """Load factor: capacity 2^(ceil(log2 V) + e) for each e, timed; returns the fastest
    and its table bytes (more slots cost memory, fewer cost longer probes)."""
    import torch

    V = P * D
    out = torch.empty((V, 3), dtype=torch.float32, device=batches[0].device)
    res = []
    same = _Same(verify)
    for e in extra_bits:
        log2cap = max(4, int(math.ceil(math.log2(max(V, 2)))) + e)
        c = _clone_config(cfg, log2_capacity=log2cap)
        t = Table(c)
        for k in range(warmup):
            t.step(batches[k % len(batches)], P, D, out=out)
        ms = _time_ms(lambda k: t.step(batches[(warmup + k) % len(batches)], P, D, out=out), iters)
        res.append({"log2_capacity": log2cap, "ms": ms, "table_bytes": t.nbytes, "max_probe": t.stats()["max_probe"]})
        same([t], {"log2_capacity": log2cap})
        t.close()
    best = min(res, key=lambda r: r["ms"])
    return {"best": best["log2_capacity"], "all": res, "verified": same.checked}


def tune_batch(make_entries, n_items: int, space: dict | None = None, warmup: int = 2, iters: int = 3,
               verify: bool = False) -> dict:
    """Fastest batched-kernel knobs.  make_entries(**fields) must return fresh (table, vertices,
    out, P, D [, slots]) entries (scratch tables) for each candidate; the space's table fields
    are passed to it by name: "capacity_bits" (each session's table gets 2^(ceil(log2 V) +
    capacity_bits) slots) and "key_layout" (where its keys live)."""
    space = space or BATCH_SPACE
    keys = list(space)
    results = []
    same = _Same(verify)
    table_fields = ("capacity_bits",) + CONFIG_KNOBS
    for values in itertools.product(*(space[k] for k in keys)):
        knobs = dict(zip(keys, values))
        fields = {k: knobs.pop(k) for k in table_fields if k in knobs}
        entries = make_entries(**fields)
        b = Batch(n_items, **knobs)
        b.set(entries)
        for _ in range(warmup):
            b.launch()
        ms = _time_ms(lambda k: b.launch(), iters)
        if b.status() != 0:
            ms = float("inf")
        knobs.update(fields)
        same([e[0] for e in entries], knobs)
        b.close()
        for e in entries:
            e[0].close()
        results.append((ms, knobs))
    results.sort(key=lambda r: r[0])
    return {"best": results[0][1], "best_ms": results[0][0], "all": [{"ms": ms, **k} for ms, k in results],
            "verified": same.checked}
