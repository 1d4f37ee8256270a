"""Hierarchy levels on the GPU (Section "Progressive hierarchical solver"): every inserted
vertex lands in its cell at each of the L levels, and a vertex at depth j is read at level
min(j, L - 1).  Compared with the oracle element by element, as the flat tables are: keys,
sums and counters bit-exact, blended values and estimator outputs within the FP32 / FP16
bounds of the flat tables."""

import numpy as np
import pytest

from parity import check_after_insert, check_after_update, check_cv, check_estimator
from test_gpu_parity import _cfg_for, _oracle_for, _run_and_compare, _workload_batches

pytestmark = pytest.mark.gpu


def _cfg(psf, w, levels, **over):
    # up to `levels` times the cells of the flat table: two more bits of capacity
    return _cfg_for(psf, w, levels=levels, log2_capacity=w["log2_capacity"] + 2, **over)


@pytest.mark.parametrize("levels", [2, 3, 4])
@pytest.mark.parametrize("fp16", [False, True])
def test_levels_64x64_all_iterations(psf_mod, oracle_mod, levels, fp16):
    w, batches = _workload_batches("64x64_d3", 5)
    worst = _run_and_compare(psf_mod, oracle_mod, _cfg(psf_mod, w, levels, cache_fp16=fp16), batches,
                             w["width"] * w["height"], w["depth"])
    print("worst relative errors", worst)


@pytest.mark.parametrize("knobs", [dict(vertex_staging=1), dict(insert_mode=1), dict(vertex_staging=3),
                                   dict(vertex_staging=0, insert_mode=1, insert_blocks_per_sm=1), dict(sum_reduction=1),
                                   dict(sum_reduction=1, insert_mode=1)])
def test_levels_launch_knobs_do_not_change_results(psf_mod, knobs):
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg(psf_mod, w, 3)
    P, D = w["width"] * w["height"], w["depth"]
    runs = []
    for setting in ({}, knobs):
        table = psf_mod.Table(cfg)
        table.set_launch(**setting)
        outs = [table.step(torch.from_numpy(v).cuda(), P, D).cpu().numpy() for v in batches]
        runs.append((table.export().tobytes(), np.concatenate(outs).tobytes()))
        table.close()
    assert runs[0] == runs[1]


def test_levels_coarse_cells_regroup_fine_cells_on_the_gpu(psf_mod):
    """The GPU's coarse cells hold exactly the sums of the fine cells they contain."""
    import torch

    w, batches = _workload_batches("64x64_d3", 1)
    table = psf_mod.Table(_cfg(psf_mod, w, 3))
    table.insert(torch.from_numpy(batches[0]).cuda())
    rec = table.export()
    lvl = (rec["key"] >> np.uint64(61)).astype(np.int64)
    fine = rec[lvl == 0]
    for l in (1, 2):
        groups = {}
        for r in fine:
            k = int(r["key"])
            xyz = [((k >> s) & 0xFFFF) - 32768 for s in (32, 16, 0)]
            ck = (l << 61) | (k & 0x1FFF000000000000) | sum(((c >> l) + 32768) << s for c, s in zip(xyz, (32, 16, 0)))
            g = groups.setdefault(ck, np.zeros(4, dtype=np.int64))
            g += np.array([*r["sum"], r["c_new"]], dtype=np.int64)
        coarse = rec[lvl == l]
        assert len(coarse) == len(groups) < len(fine)
        for r in coarse:
            assert np.array_equal(groups[int(r["key"])], np.array([*r["sum"], r["c_new"]], dtype=np.int64))
    table.close()


@pytest.mark.parametrize("gamma,jb,je", [(0.0, 1, 2), (0.5, 0, 0xFFFFFFFF)])
def test_levels_biased_estimator(psf_mod, oracle_mod, gamma, jb, je):
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg(psf_mod, w, 3)
    P, D = w["width"] * w["height"], w["depth"]
    table, ora = psf_mod.Table(cfg), _oracle_for(oracle_mod, cfg)
    for v in batches:
        dv = torch.from_numpy(v).cuda()
        table.insert(dv)
        table.update()
        ora.insert(v)
        ora.update()
        out = table.query_biased(dv, P, D, gamma, jb, je).cpu().numpy()
        check_estimator(out, ora.query_biased(v, P, D, gamma, jb, je), v, ora.lookup(v, P, D), P, D, gamma, gamma,
                        1.0, jb, je, ora.export()["L"])
    table.close()


@pytest.mark.parametrize("field", [0, 1])
def test_levels_progressive_insert(psf_mod, oracle_mod, field):
    """eq. (9) with the next vertex's approximant read at its level; the bound is the flat
    progressive test's (the fed-back value differs by the FP32 vs FP64 approximant)."""
    import torch

    w, batches = _workload_batches("64x64_d3", 4)
    cfg = _cfg(psf_mod, w, 3)
    P, D = w["width"] * w["height"], w["depth"]
    table, ora = psf_mod.Table(cfg), _oracle_for(oracle_mod, cfg)
    for it, v in enumerate(batches):
        dv = torch.from_numpy(v).cuda()
        table.insert_progressive(dv, P, D, field)
        ora.insert_progressive(v, P, D, field)
        g, r = table.export(), ora.export()
        assert np.array_equal(g["key"], r["key"]) and np.array_equal(g["c_new"], r["c_new"])
        slack = 1e-5 * np.abs(r["sum"]).astype(np.float64) + 2.0 * (r["c_new"] / 2.0 ** 24)[:, None] + 2.0
        diff = np.abs(g["sum"].astype(np.float64) - r["sum"].astype(np.float64))
        assert np.all(diff <= slack), (it, np.max(diff / slack))
        table.update()
        ora.update()
        check_after_update(table.export(), ora.export())
    table.close()


def test_levels_ragged_and_invalid_vertices(psf_mod, oracle_mod):
    """Ragged sizes, vertices outside the index range and zero weights at every level."""
    import torch

    from helpers import random_vertices

    rng = np.random.default_rng(11)
    cfg = psf_mod.make_config(log2_capacity=14, pos_bits=3, dir_bits=2, levels=4)
    ora = _oracle_for(oracle_mod, cfg)
    table = psf_mod.Table(cfg)
    v = random_vertices(rng, 4103, q=3, cells_per_axis=7, zero_weight_fraction=0.05)
    v[:, 0:3] -= np.float32(0.5)
    v[5, 0] = np.float32(5000.0)  # outside [-2^15, 2^15) cells at level 0
    v[77, 3] = np.float32(-1.0)
    dv = torch.from_numpy(v).cuda()
    for cut in ((0, 1), (1, 33), (33, 4103)):
        table.insert(dv[cut[0]:cut[1]])
    ora.insert(v)
    check_after_insert(table.export(), ora.export())
    table.update()
    ora.update()
    check_after_update(table.export(), ora.export())
    P, D = 4103, 1
    out = table.query_cv(dv, P, D)
    check_cv(out.cpu().numpy(), ora.query_cv(v, P, D), v, ora.lookup(v, P, D), P, D, 1.0, 0xFFFFFFFF, ora.export()["L"])
    st = table.stats()
    assert (st["dropped_vertices"], st["zero_weight_vertices"]) == ora.counters()
    table.close()


@pytest.mark.slow
def test_levels_1280x720_depth4_full_size(psf_mod, oracle_mod):
    """The full-size workload with 3 levels, in the benchmark's launch configuration."""
    w, batches = _workload_batches("1280x720_d4", 2)
    worst = _run_and_compare(psf_mod, oracle_mod, _cfg(psf_mod, w, 3), batches, w["width"] * w["height"],
                             w["depth"], use_step=True)
    print("worst relative errors", worst)
