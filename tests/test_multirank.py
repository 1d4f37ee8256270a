"""Multi-rank host logic on CPU process groups (gloo, world size 2):
  * the benchmark's whole-job aggregation (max over ranks, every rank's vertices);
  * the exchange step of a session sharded across ranks: per-rank pre-aggregated
    fixed-point records, all-to-all to owner ranks, merged map bit-exact against one
    rank inserting everything."""

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


def _shard_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import oracle
    from paper_2005_07547_b300 import shard
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    v = iteration_vertices(w, 0)
    mine = v[rank::world]  # an interleaved split of the vertex stream
    o = oracle.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"])
    o.insert(mine)
    owned = shard.exchange(o.export())
    keys = owned["key"]
    assert np.all(shard.owner_of(keys, world) == rank)
    q.put((rank, owned.tobytes()))
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


def test_sharded_session_merges_bit_exact(oracle_mod):
    from paper_2005_07547_b300 import shard
    from synth.scene import iteration_vertices, workload

    res = _run(_shard_worker)
    merged = shard.merge([np.frombuffer(b, dtype=shard.RECORD) for _, b in res])
    w = workload("64x64_d3")
    o = oracle_mod.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"])
    o.insert(iteration_vertices(w, 0))
    ref = shard.contributions(o.export())
    assert merged.tobytes() == ref.tobytes()
    # every key has exactly one owner
    assert len(np.unique(merged["key"])) == len(merged)


def test_owner_partition_is_total_and_balanced():
    from paper_2005_07547_b300 import shard

    rng = np.random.default_rng(0)
    keys = rng.integers(0, 2 ** 62, size=100000, dtype=np.uint64)
    for world in (2, 3, 8):
        own = shard.owner_of(keys, world)
        counts = np.bincount(own, minlength=world)
        assert counts.sum() == len(keys)
        assert counts.min() > 0.9 * len(keys) / world
