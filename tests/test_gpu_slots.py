"""The slot cache: psf_insert_slots leaves the same table as psf_insert and notes each
vertex's slot; psf_query_cv_slots gives the same outputs as psf_query_cv, bit for bit."""

import numpy as np
import pytest

from parity import check_cv
from test_gpu_parity import _cfg_for, _oracle_for, _workload_batches

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("over,knobs", [(dict(), dict()), (dict(cache_fp16=True), dict()),
                                        (dict(key_layout=1), dict()), (dict(key_layout=2, cache_fp16=True), dict()),
                                        (dict(levels=3, log2_capacity=18), dict()), (dict(), dict(insert_mode=1)),
                                        (dict(levels=2, log2_capacity=18), dict(insert_mode=1))])
def test_slots_give_the_same_tables_and_outputs(psf_mod, oracle_mod, over, knobs):
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg_for(psf_mod, w, **over)
    P, D = w["width"] * w["height"], w["depth"]
    plain, cached = psf_mod.Table(cfg), psf_mod.Table(cfg)
    for t in (plain, cached):
        t.set_launch(**knobs)
    ora = _oracle_for(oracle_mod, cfg)
    cap = 1 << cfg.log2_capacity
    prev = 0  # vertices not added (range rule, zero weight) before this iteration
    for v in batches:
        dv = torch.from_numpy(v).cuda()
        plain.insert(dv)
        slots = cached.insert_slots(dv, P, D)
        assert plain.export().tobytes() == cached.export().tobytes()
        s = slots.cpu().numpy().view(np.uint32)
        noted = s != 0xFFFFFFFF
        assert np.all(s[noted] < cap)
        st = cached.stats()
        skipped = st["dropped_vertices"] + st["zero_weight_vertices"]
        assert int((~noted).sum()) == skipped - prev  # no table here fills up
        prev = skipped
        plain.update()
        cached.update()
        a = plain.query_cv(dv, P, D).cpu().numpy()
        b = cached.query_cv_slots(dv, slots, P, D).cpu().numpy()
        assert a.tobytes() == b.tobytes()
        ora.insert(v)
        ora.update()
        check_cv(b, ora.query_cv(v, P, D), v, ora.lookup(v, P, D), P, D, float(cfg.beta), cfg.cv_max_depth,
                 ora.export()["L"], fp16=bool(cfg.cache_fp16))
    plain.close()
    cached.close()


def test_slots_of_dropped_vertices_fall_back_to_probing(psf_mod):
    """A full table: dropped vertices get PSF_NO_SLOT, and on that table the slot query still
    matches psf_query_cv (which keys win the last slots of a full table depends on the order
    of the claims, so the comparison is on one table)."""
    import torch

    from helpers import random_vertices

    rng = np.random.default_rng(9)
    P, D = 300, 2
    v = random_vertices(rng, P * D, q=3, cells_per_axis=6)
    v[7, 0] = np.float32(np.nan)  # range rule
    cfg = psf_mod.make_config(log2_capacity=5, pos_bits=3, dir_bits=2)  # 32 slots: fills up
    cached = psf_mod.Table(cfg)
    dv = torch.from_numpy(v).cuda()
    slots = cached.insert_slots(dv, P, D)
    s = slots.cpu().numpy().view(np.uint32)
    st = cached.stats()
    assert st["status"] & psf_mod.STATUS_TABLE_FULL and s[7] == 0xFFFFFFFF
    assert int((s == 0xFFFFFFFF).sum()) == st["dropped_vertices"] + st["zero_weight_vertices"]
    cached.update()
    assert cached.query_cv(dv, P, D).cpu().numpy().tobytes() == cached.query_cv_slots(dv, slots, P, D).cpu().numpy().tobytes()
    cached.close()


@pytest.mark.parametrize("over", [dict(), dict(cache_fp16=True), dict(key_layout=2, cache_fp16=True)])
def test_query_before_the_update_reads_the_old_approximant(psf_mod, oracle_mod, over):
    """The strictly unbiased order (Section "Temporal averaging" read with the control variate
    of the previous iteration): insert, query, then update.  The query reads the approximant
    blended up to the previous iteration (0 for a cell first touched now), through the probing
    query and the slot cache alike, and the oracle queried in the same order agrees."""
    import torch

    w, batches = _workload_batches("64x64_d3", 4)
    cfg = _cfg_for(psf_mod, w, **over)
    P, D = w["width"] * w["height"], w["depth"]
    plain, cached = psf_mod.Table(cfg), psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    for k, v in enumerate(batches):
        dv = torch.from_numpy(v).cuda()
        plain.insert(dv)
        slots = cached.insert_slots(dv, P, D)
        a = plain.query_cv(dv, P, D).cpu().numpy()
        b = cached.query_cv_slots(dv, slots, P, D).cpu().numpy()
        assert a.tobytes() == b.tobytes()
        ora.insert(v)
        old = ora.lookup(v, P, D)
        if k == 0:
            assert not np.any(old)  # nothing blended yet: every cell reads 0
        check_cv(b, ora.query_cv(v, P, D), v, old, P, D, float(cfg.beta), cfg.cv_max_depth, ora.export()["L"],
                 fp16=bool(cfg.cache_fp16))
        plain.update()
        cached.update()
        ora.update()
        assert plain.export().tobytes() == cached.export().tobytes()
    plain.close()
    cached.close()
