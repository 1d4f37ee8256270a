"""One render session sharded across ranks (host-side logic of the single-session split).

Independent sessions need no communication: each rank runs its own.  A single session too
large for one GPU splits its paths across ranks, and every iteration runs four steps:

  1. pre-aggregate: each rank inserts its share of the vertices into a scratch table and
     takes the touched cells' fixed-point records (key, three sums, c_new);
  2. exchange: one all-to-all sends every record to the rank that owns its key, and only
     there -- owner = (fmix64(key) >> 32) mod world, the same mixer as the table's home
     slot; the split sizes travel first, then the records;
  3. owner blend: the owner adds the records it received to its table (integer sums, so its
     cells are bit-exact under any split of the vertices, eq. (5)-(6)) and blends the cells
     it owns (eq. (10)-(11)); the approximant of a cell is only ever computed by its owner;
  4. query exchange: an all-gather of the cells blended this iteration (key, approximant)
     brings every rank the approximant of the cells it does not own; each rank writes them
     into its table and answers the control-variate query for its own paths.

The per-rank work sits behind a small backend interface (contributions, merge_and_blend,
set_approximant, query_cv): `TableShard` runs it on the GPU library through the C ABI
(psf_insert, psf_export, psf_insert_records, psf_update, psf_set_approximant, psf_query_cv).
`step` drives one iteration over torch.distributed (gloo with host tensors, NCCL with device
tensors); `step_in_process` runs the same four steps for several ranks in
one process, one rank after the other, with the exchanges done by array slicing.
"""

from __future__ import annotations

import numpy as np

_M1 = np.uint64(0xFF51AFD7ED558CCD)
_M2 = np.uint64(0xC4CEB9FE1A85EC53)

RECORD = np.dtype([("key", "<u8"), ("sum", "<i8", (3,)), ("c_new", "<i8")])  # psf_record
CELL = np.dtype([("key", "<u8"), ("L", "<f4", (3,))])  # a blended cell's approximant


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


def contributions(records: np.ndarray) -> np.ndarray:
    """The exchanged part of exported cells: key, this iteration's sums and counter, for the
    cells touched this iteration."""
    out = np.zeros(len(records), dtype=RECORD)
    out["key"] = records["key"]
    out["sum"] = records["sum"]
    out["c_new"] = records["c_new"]
    return out[out["c_new"] != 0]


def partition(records: np.ndarray, world: int) -> list[np.ndarray]:
    own = owner_of(records["key"], world)
    return [records[own == r] for r in range(world)]


def merge(parts: list[np.ndarray]) -> np.ndarray:
    """Sum the records of equal keys (int64 sums, modulo 2^64 like the tables); ascending key
    order."""
    allr = np.concatenate([p for p in parts if len(p)]) if any(len(p) for p in parts) else np.zeros(0, RECORD)
    if len(allr) == 0:
        return allr
    keys, inv = np.unique(allr["key"], return_inverse=True)
    out = np.zeros(len(keys), dtype=RECORD)
    out["key"] = keys
    with np.errstate(over="ignore"):
        for c in range(3):
            np.add.at(out["sum"][:, c], inv, allr["sum"][:, c])
        np.add.at(out["c_new"], inv, allr["c_new"])
    return out


# ------------------------------------------------------------------------------------------
# exchanges over torch.distributed
# ------------------------------------------------------------------------------------------

def _as_i64(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64).reshape(-1))


def _device(group):
    """Where the collectives' tensors live: NCCL exchanges device tensors, gloo host ones."""
    import torch
    import torch.distributed as dist

    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def all_to_all_records(parts: list[np.ndarray], group=None) -> list[np.ndarray]:
    """parts[r] goes to rank r; returns the parts every rank sent here (in rank order)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = _device(group)
    words = RECORD.itemsize // 8
    send_counts = torch.tensor([len(p) for p in parts], dtype=torch.int64, device=dev)
    recv_counts = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    recv_counts = recv_counts.cpu()
    send = _as_i64(np.concatenate(parts) if sum(len(p) for p in parts) else np.zeros(0, RECORD)).to(dev)
    recv = torch.empty(int(recv_counts.sum()) * words, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv, send, output_split_sizes=[int(c) * words for c in recv_counts],
                           input_split_sizes=[int(c) * words for c in send_counts.cpu()], group=group)
    flat = recv.cpu().numpy().view(RECORD)
    offs = np.concatenate([[0], np.cumsum(recv_counts.numpy())])
    return [flat[offs[r]:offs[r + 1]] for r in range(world)]


def all_gather_cells(cells: np.ndarray, group=None) -> list[np.ndarray]:
    """Every rank's blended cells, in rank order (sizes first, then the padded cells)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = _device(group)
    n = torch.tensor([len(cells)], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    top = max(sizes)
    buf = np.zeros(top, dtype=CELL)
    buf[:len(cells)] = cells
    words = CELL.itemsize // 4
    mine = torch.from_numpy(buf.view(np.int32).reshape(-1).copy()).to(dev)
    got = [torch.zeros(top * words, dtype=torch.int32, device=dev) for _ in range(world)]
    dist.all_gather(got, mine, group=group)
    return [g.cpu().numpy().view(CELL)[:k] for g, k in zip(got, sizes)]


def step(backend, vertices, P: int, D: int, group=None):
    """One iteration of this rank's share (P paths of depth D, depth-major) of a sharded
    session; every rank of `group` calls it together.  Returns this rank's query output."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    received = all_to_all_records(partition(backend.contributions(vertices), world), group)
    blended = backend.merge_and_blend(merge(received))
    cells = all_gather_cells(blended, group)
    foreign = [c for r, c in enumerate(cells) if r != rank and len(c)]
    backend.set_approximant(np.concatenate(foreign) if foreign else np.zeros(0, CELL))
    return backend.query_cv(vertices, P, D)


def step_in_process(backends: list, shares: list, D: int) -> list:
    """The same iteration for all ranks in one process: backends[r] holds rank r's tables,
    shares[r] = (vertices, P) its paths.  Returns every rank's query output."""
    world = len(backends)
    parts = [partition(b.contributions(v), world) for b, (v, _) in zip(backends, shares)]
    blended = [backends[r].merge_and_blend(merge([parts[s][r] for s in range(world)])) for r in range(world)]
    for r in range(world):
        foreign = [blended[s] for s in range(world) if s != r and len(blended[s])]
        backends[r].set_approximant(np.concatenate(foreign) if foreign else np.zeros(0, CELL))
    return [b.query_cv(v, P, D) for b, (v, P) in zip(backends, shares)]


# ------------------------------------------------------------------------------------------
# the per-rank work on the GPU library
# ------------------------------------------------------------------------------------------

class TableShard:
    """A rank's tables for a sharded session: a scratch table that pre-aggregates the rank's
    vertices each iteration, and the rank's table proper, which owns the cells of its keys
    (their counters and blend) and holds a copy of the approximant of every other cell for
    the query.  Both take the session's configuration."""

    def __init__(self, cfg, device=None):
        from .table import Table

        self.cfg = cfg
        self.scratch = Table(cfg, device=device)
        self.table = Table(cfg, device=device)

    def contributions(self, vertices) -> np.ndarray:
        self.scratch.insert(vertices)
        rec = contributions(self.scratch.export())
        self.scratch.update()  # clears the scratch sums (its own approximant is never read)
        return rec

    def merge_and_blend(self, records: np.ndarray) -> np.ndarray:
        """Add the received records, blend, and return the blended cells' approximants (read
        from a full export of the table: host-side, O(live cells) per iteration)."""
        import torch

        if len(records):
            self.table.insert_records(torch.from_numpy(records.view(np.int64).reshape(-1, 5).copy()).to(
                self.table.device))
        self.table.update()
        if not len(records):
            return np.zeros(0, CELL)
        ex = self.table.export()
        at = np.searchsorted(ex["key"], records["key"])
        out = np.zeros(len(records), dtype=CELL)
        out["key"] = records["key"]
        out["L"] = ex["L"][at]
        return out

    def set_approximant(self, cells: np.ndarray) -> None:
        import torch

        if len(cells):
            dev = self.table.device
            keys = torch.from_numpy(cells["key"].view(np.int64).copy()).to(dev)
            L = torch.from_numpy(np.ascontiguousarray(cells["L"], dtype=np.float32)).to(dev)
            self.table.set_approximant(keys, L)

    def query_cv(self, vertices, P: int, D: int):
        return self.table.query_cv(vertices, P, D)

    def close(self) -> None:
        self.scratch.close()
        self.table.close()
