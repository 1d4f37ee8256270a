"""A session sharded across ranks on the GPU library (psf_insert_records, psf_set_approximant
and the shard module's four steps), with the ranks run one after the other in one process:
every owner's cells and every rank's control-variate outputs equal, bit for bit, those of
one table that holds the whole session (the owner blends the same integer sums with the same
kernel; the other ranks read the owner's FP32 approximant)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _share(v, P, D, rank, world):
    mine = np.ascontiguousarray(v.reshape(D, P, 16)[:, rank::world].reshape(-1, 16))
    return mine, mine.shape[0] // D


@pytest.mark.parametrize("world,fp16", [(2, False), (3, True)])
def test_sharded_session_equals_one_table(psf_mod, world, fp16):
    import torch

    from paper_2005_07547_b300 import shard
    from synth.scene import iteration_vertices, make_scene, workload

    w = workload("64x64_d3")
    scene = make_scene(w["seed"])
    P, D = w["width"] * w["height"], w["depth"]
    cfg = psf_mod.make_config(log2_capacity=w["log2_capacity"], pos_bits=w["pos_bits"], dir_bits=w["dir_bits"],
                              alpha_min=w["alpha_min"], cache_fp16=fp16)
    whole = psf_mod.Table(cfg)
    ranks = [shard.TableShard(cfg) for _ in range(world)]
    for it in range(4):
        v = iteration_vertices(w, it, scene)
        out_whole = whole.step(torch.from_numpy(v).cuda(), P, D).cpu().numpy()
        shares = [_share(v, P, D, r, world) for r in range(world)]
        outs = shard.step_in_process(ranks, [(torch.from_numpy(m).cuda(), Pr) for m, Pr in shares], D)
        ref = whole.export()
        owned = []
        for r, b in enumerate(ranks):
            ex = b.table.export()
            owned.append(ex[shard.owner_of(ex["key"], world) == r])
            # the rank's table holds the whole session's approximant, the owner's or a copy
            assert np.array_equal(ex["key"], ref["key"]) and np.array_equal(ex["L"], ref["L"])
            assert np.array_equal(ex["L_fp16"], ref["L_fp16"])
        owned = np.concatenate(owned)
        owned = owned[np.argsort(owned["key"])]
        assert owned.tobytes() == ref.tobytes(), it
        for r in range(world):
            want = out_whole.reshape(D, P, 3)[:, r::world].reshape(-1, 3)
            assert np.array_equal(outs[r].cpu().numpy(), want), (it, r)
    for b in ranks:
        assert b.table.stats()["status"] == 0
        b.close()
    whole.close()


def test_inserting_records_equals_inserting_their_vertices(psf_mod):
    """A table's exported contributions, re-inserted as records into an empty table (in two
    pieces, one key in both), give the same table after the blend."""
    import torch

    from helpers import random_vertices
    from paper_2005_07547_b300 import shard

    rng = np.random.default_rng(3)
    v = torch.from_numpy(random_vertices(rng, 5000, q=3, cells_per_axis=4)).cuda()
    cfg = psf_mod.make_config(log2_capacity=12, pos_bits=3, dir_bits=2)
    a, b = psf_mod.Table(cfg), psf_mod.Table(cfg)
    a.insert(v)
    rec = shard.contributions(a.export())
    half = rec.copy()
    half["sum"] //= 2
    half["c_new"] //= 2
    rest = rec.copy()
    rest["sum"] -= half["sum"]
    rest["c_new"] -= half["c_new"]
    for part in (half, rest):
        b.insert_records(torch.from_numpy(part.view(np.int64).reshape(-1, 5).copy()).cuda())
    assert shard.contributions(b.export()).tobytes() == rec.tobytes()
    a.update()
    b.update()
    assert a.export().tobytes() == b.export().tobytes()
    # a record whose key is not a cell key is dropped with the range status
    bad = np.zeros(1, dtype=shard.RECORD)
    bad["key"] = np.uint64(1) << np.uint64(63)
    b.insert_records(torch.from_numpy(bad.view(np.int64).reshape(-1, 5).copy()).cuda())
    st = b.stats()
    assert st["status"] == psf_mod.STATUS_RANGE and st["dropped_vertices"] == 1
    a.close()
    b.close()
