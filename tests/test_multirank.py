"""Multi-rank host logic on CPU process groups (gloo, world size 2):
  * the benchmark's whole-job aggregation (max over ranks, every rank's vertices);
  * a session sharded across ranks (paper_2005_07547_b300.shard): per-rank pre-aggregated
    fixed-point records, an all-to-all that delivers each record to its owner only, the
    owner's blend, an all-gather of the blended cells, and each rank's query of its own
    paths -- checked over several iterations against one oracle holding the whole session.
The per-rank compute here is the oracle (OracleShard below), so these tests check the host
logic of the split; the GPU backend of the same steps is checked in test_gpu_shard.py."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _bench_worker(rank, world, port, q):
    import torch

    dist = _init(rank, world, port)
    import bench

    elapsed = [100.0, 130.0][rank]
    t = torch.tensor([elapsed], dtype=torch.float64)
    g = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(g, t)
    agg = bench.aggregate([float(x.item()) for x in g], 1000, 10, world)
    q.put((rank, agg, bench.rank_seed_offset(rank)))
    dist.destroy_process_group()


class OracleShard:
    """A rank's share of a sharded session computed by the oracle (tests only): a fresh
    oracle pre-aggregates each iteration's vertices; the rank's oracle table owns its keys'
    cells and holds the approximant of the others (their exchanged FP32 values)."""

    def __init__(self, **kw):
        import oracle

        self.oracle = oracle
        self.kw = kw
        self.table = oracle.Oracle(**kw)

    def contributions(self, v):
        from paper_2005_07547_b300 import shard

        s = self.oracle.Oracle(**self.kw)
        s.insert(v)
        return shard.contributions(s.export())

    def _import(self, keys, sums, c_new, L=None):
        ex = self.table.export()
        at = {int(k): i for i, k in enumerate(ex["key"])}
        rec = np.zeros(len(keys), dtype=self.oracle.RECORD_DTYPE)
        rec["key"] = keys
        for i, k in enumerate(keys):
            j = at.get(int(k))
            if j is not None:
                rec["c_old"][i] = ex["c_old"][j]
                rec["L"][i] = ex["L"][j]
        rec["sum"] = sums
        rec["c_new"] = c_new
        if L is not None:
            rec["L"] = L
        self.table.import_records(rec)

    def merge_and_blend(self, records):
        from paper_2005_07547_b300 import shard

        self._import(records["key"], records["sum"], records["c_new"])
        self.table.update()
        ex = self.table.export()
        cells = np.zeros(len(records), dtype=shard.CELL)
        cells["key"] = records["key"]
        cells["L"] = ex["L"][np.searchsorted(ex["key"], records["key"])]
        return cells

    def set_approximant(self, cells):
        if len(cells):
            self._import(cells["key"], 0, 0, cells["L"].astype(np.float64))

    def query_cv(self, v, P, D):
        return self.table.query_cv(v, P, D)


def _paths_of(v, P, D, rank, world):
    """Rank r's share of the session: paths r, r + world, ... (all their depths)."""
    mine = np.ascontiguousarray(v.reshape(D, P, 16)[:, rank::world].reshape(-1, 16))
    return mine, mine.shape[0] // D


def _shard_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    from paper_2005_07547_b300 import shard
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    P, D = w["width"] * w["height"], w["depth"]
    be = OracleShard(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(w["alpha_min"])))
    outs, tables = [], []
    for it in range(3):
        mine, Pr = _paths_of(iteration_vertices(w, it), P, D, rank, world)
        outs.append(shard.step(be, mine, Pr, D))
        ex = be.table.export()
        tables.append(ex[shard.owner_of(ex["key"], world) == rank].tobytes())  # the cells this rank owns
    q.put((rank, tables, outs))
    dist.destroy_process_group()


def _run(worker, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda x: x[0])


def test_bench_aggregates_max_over_ranks():
    res = _run(_bench_worker)
    for rank, agg, off in res:
        assert agg["ms_per_step"] == pytest.approx(13.0)  # the slower rank
        assert agg["value"] == pytest.approx(2 * 1000 * 10 / 0.130)
    assert res[0][2] != res[1][2]  # ranks render different sessions


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_session_matches_one_table(oracle_mod, world):
    """Owners' cells equal the whole-session oracle's bit for bit (keys, c_old and the FP64
    blend of identical integer sums) after every iteration; each rank's control-variate
    outputs for its own paths equal the whole session's within the FP32 tolerance (cells a
    rank does not own arrive as FP32 approximants)."""
    from parity import check_cv
    from synth.scene import iteration_vertices, workload

    res = _run(_shard_worker, world)
    w = workload("64x64_d3")
    P, D = w["width"] * w["height"], w["depth"]
    ref = oracle_mod.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(w["alpha_min"])))
    for it in range(3):
        v = iteration_vertices(w, it)
        ref.insert(v)
        ref.update()
        want = ref.export()
        owned = np.concatenate([np.frombuffer(res[r][1][it], dtype=oracle_mod.RECORD_DTYPE) for r in range(world)])
        owned = owned[np.argsort(owned["key"])]
        assert owned.tobytes() == want.tobytes(), it  # every cell has one owner, and it is exact
        for r in range(world):
            mine, Pr = _paths_of(v, P, D, r, world)
            check_cv(res[r][2][it], ref.query_cv(mine, Pr, D), mine, ref.lookup(mine), Pr, D, 1.0, 0xFFFFFFFF,
                     want["L"])


def test_all_to_all_delivers_each_record_to_its_owner_only():
    res = _run(_exchange_worker, 3)
    from paper_2005_07547_b300 import shard

    sent = [shard.partition(_records(r), 3) for r in range(3)]
    for r, got in res:
        assert len(got) == 3
        for s in range(3):
            assert got[s] == sent[s][r].tobytes()  # exactly what rank s addressed to rank r


def _records(rank):
    from paper_2005_07547_b300 import shard

    rng = np.random.default_rng(rank)
    rec = np.zeros(50 + 17 * rank, dtype=shard.RECORD)
    rec["key"] = rng.integers(0, 2 ** 62, size=len(rec), dtype=np.uint64)
    rec["sum"] = rng.integers(-2 ** 40, 2 ** 40, size=(len(rec), 3))
    rec["c_new"] = rng.integers(1, 2 ** 30, size=len(rec))
    return rec


def _exchange_worker(rank, world, port, q):
    _init(rank, world, port)
    import torch.distributed as dist

    from paper_2005_07547_b300 import shard

    got = shard.all_to_all_records(shard.partition(_records(rank), world))
    q.put((rank, [g.tobytes() for g in got]))
    dist.destroy_process_group()


def test_owner_partition_is_total_and_balanced():
    from paper_2005_07547_b300 import shard

    rng = np.random.default_rng(0)
    keys = rng.integers(0, 2 ** 62, size=100000, dtype=np.uint64)
    for world in (2, 3, 8):
        own = shard.owner_of(keys, world)
        counts = np.bincount(own, minlength=world)
        assert counts.sum() == len(keys)
        assert counts.min() > 0.9 * len(keys) / world


def test_exchange_tensors_follow_the_backend(monkeypatch):
    """NCCL exchanges device tensors, gloo host ones."""
    import torch
    import torch.distributed as dist

    from paper_2005_07547_b300 import shard

    monkeypatch.setattr(dist, "get_backend", lambda group=None: "gloo")
    assert shard._device(None) == torch.device("cpu")
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "nccl")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert shard._device(None) == torch.device("cuda", 3)
