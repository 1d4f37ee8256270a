"""The exchange step of one session sharded across ranks (host-side logic).

Independent sessions need no communication: each rank runs its own.  A single session
too large for one GPU would split its vertex stream across ranks; each rank inserts its
share into a local table, whose fixed-point records (key, three sums, c_new) are the
rank's pre-aggregated contributions.  One all-to-all then sends every record to the
rank that owns its key -- owner = (fmix64(key) >> 32) mod world, the same mixer as the
table's home slot -- and the owner adds the sums.  Integer addition is associative, so
the merged map is bit-exact under any partition of the vertices; the owner then blends
the cells it owns (the approximant of a cell is only ever written by its owner).

The boxes this project runs on have one GPU each, so this path is exercised with CPU
process groups (gloo); the records would come from psf_export on each rank's table.
"""

from __future__ import annotations

import numpy as np

_M1 = np.uint64(0xFF51AFD7ED558CCD)
_M2 = np.uint64(0xC4CEB9FE1A85EC53)


def fmix64(keys: np.ndarray) -> np.ndarray:
    """MurmurHash3's 64-bit finaliser (Appleby, public domain), vectorised."""
    k = np.asarray(keys, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        k ^= k >> np.uint64(33)
        k *= _M1
        k ^= k >> np.uint64(33)
        k *= _M2
        k ^= k >> np.uint64(33)
    return k


def owner_of(keys: np.ndarray, world: int) -> np.ndarray:
    return ((fmix64(keys) >> np.uint64(32)) % np.uint64(world)).astype(np.int64)


RECORD = np.dtype([("key", "<u8"), ("sum", "<i8", (3,)), ("c_new", "<i8")])


def contributions(records: np.ndarray) -> np.ndarray:
    """The exchanged part of exported cells: key, this iteration's sums and counter."""
    out = np.zeros(len(records), dtype=RECORD)
    out["key"] = records["key"]
    out["sum"] = records["sum"]
    out["c_new"] = records["c_new"]
    return out[out["c_new"] != 0]


def partition(records: np.ndarray, world: int) -> list[np.ndarray]:
    own = owner_of(records["key"], world)
    return [records[own == r] for r in range(world)]


def merge(parts: list[np.ndarray]) -> np.ndarray:
    """Sum the records of equal keys (exact int64 sums); ascending key order."""
    allr = np.concatenate([p for p in parts if len(p)]) if any(len(p) for p in parts) else np.zeros(0, RECORD)
    if len(allr) == 0:
        return allr
    keys, inv = np.unique(allr["key"], return_inverse=True)
    out = np.zeros(len(keys), dtype=RECORD)
    out["key"] = keys
    for c in range(3):
        np.add.at(out["sum"][:, c], inv, allr["sum"][:, c])
    np.add.at(out["c_new"], inv, allr["c_new"])
    return out


def exchange(records: np.ndarray, group=None) -> np.ndarray:
    """All-to-all of pre-aggregated records to their owner ranks; returns this rank's
    merged cells.  Uses torch.distributed (any backend that has all_gather_object)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = partition(contributions(records), world)
    gathered: list = [None] * world
    dist.all_gather_object(gathered, [p.tobytes() for p in parts], group=group)
    mine = [np.frombuffer(g[rank], dtype=RECORD) for g in gathered]
    return merge(mine)
