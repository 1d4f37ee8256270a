"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Small workloads are compared in full every iteration (tables after insert and after
update, CV outputs).  The full-size workloads over their own iteration counts are in
test_gpu_full_*.py.
"""

import numpy as np
import pytest

from helpers import random_vertices, stack, vertex
from parity import check_after_insert, check_after_update, check_cv

pytestmark = pytest.mark.gpu


def _oracle_for(oracle_mod, cfg):
    return oracle_mod.Oracle(pos_bits=cfg.pos_bits_q, dir_bits=cfg.dir_bits_d, use_normal=bool(cfg.use_normal),
                             frac_bits=cfg.frac_bits, blend_mode=cfg.blend_mode, cv_max_depth=cfg.cv_max_depth,
                             alpha_min=float(np.float32(cfg.alpha_min)), beta=float(np.float32(cfg.beta)),
                             levels=cfg.levels)


def _run_and_compare(psf, oracle_mod, cfg, batches, P, D, *, check_insert=True, use_step=False):
    """Drive a GPU table and the oracle through the same iterations; compare everything."""
    import torch

    table = psf.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    worst = {"L32": 0.0, "L16": 0.0, "cv": 0.0}
    for v in batches:
        dv = torch.from_numpy(v).cuda()
        st = ora.insert(v)
        if use_step:
            out = table.step(dv, P, D)
        else:
            table.insert(dv)
            if check_insert:
                check_after_insert(table.export(), ora.export())
            table.update()
            out = table.query_cv(dv, P, D)
        ora.update()
        r32, r16 = check_after_update(table.export(), ora.export(), fp16=bool(cfg.cache_fp16))
        worst["L32"] = max(worst["L32"], r32)
        worst["L16"] = max(worst["L16"], r16 or 0.0)
        ref = ora.query_cv(v, P, D)
        worst["cv"] = max(worst["cv"], check_cv(out.cpu().numpy(), ref, v, ora.lookup(v, P, D), P, D, float(cfg.beta),
                                                cfg.cv_max_depth, ora.export()["L"], fp16=bool(cfg.cache_fp16)))
        stats = table.stats()
        dropped, zero_w = ora.counters()
        assert stats["dropped_vertices"] == dropped and stats["zero_weight_vertices"] == zero_w
        assert stats["status"] == st or (stats["status"] & ~psf.STATUS_RANGE) == 0
        assert stats["live_cells"] == len(ora)
    table.close()
    return worst


def _workload_batches(name, iterations, seed_offset=0):
    from synth.scene import iteration_vertices, make_scene, workload

    w = workload(name)
    scene = make_scene(w["seed"])
    return w, [iteration_vertices(w, it + seed_offset, scene) for it in range(iterations)]


def _cfg_for(psf, w, **over):
    kw = dict(log2_capacity=w["log2_capacity"], pos_bits=w["pos_bits"], dir_bits=w["dir_bits"],
              alpha_min=w["alpha_min"], cache_fp16=w["cache_fp16"])
    kw.update(over)
    return psf.make_config(**kw)


@pytest.mark.parametrize("fp16", [False, True])
def test_64x64_depth3_all_iterations(psf_mod, oracle_mod, fp16):
    w, batches = _workload_batches("64x64_d3", 8)
    worst = _run_and_compare(psf_mod, oracle_mod, _cfg_for(psf_mod, w, cache_fp16=fp16), batches,
                             w["width"] * w["height"], w["depth"])
    print("worst relative errors", worst)


@pytest.mark.parametrize("over", [dict(use_normal=False), dict(blend_mode=1), dict(cv_max_depth=1),
                                  dict(beta=0.5), dict(frac_bits=16), dict(frac_bits=32), dict(dir_bits=5, pos_bits=6),
                                  dict(dir_bits=0), dict(alpha_min=0.0), dict(key_layout=2),
                                  dict(key_layout=2, cache_fp16=True)])
def test_configuration_variants(psf_mod, oracle_mod, over):
    w, batches = _workload_batches("64x64_d3", 3)
    _run_and_compare(psf_mod, oracle_mod, _cfg_for(psf_mod, w, **over), batches, w["width"] * w["height"], w["depth"])


def test_reset_and_multiple_inserts_per_iteration(psf_mod, oracle_mod):
    import torch

    w, batches = _workload_batches("64x64_d3", 4)
    cfg = _cfg_for(psf_mod, w)
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    P, D = w["width"] * w["height"], w["depth"]
    for it, v in enumerate(batches):
        if it == 2:
            table.reset()
            ora.reset()
        dv = torch.from_numpy(v).cuda()
        cuts = [0, 1, 4097, 9000, len(v)]  # ragged pieces, one of a single vertex
        for a, b in zip(cuts[:-1], cuts[1:]):
            table.insert(dv[a:b])
        ora.insert(v)
        check_after_insert(table.export(), ora.export())
        table.update()
        ora.update()
        check_after_update(table.export(), ora.export())
        out = table.query_cv(dv, P, D)
        check_cv(out.cpu().numpy(), ora.query_cv(v, P, D), v, ora.lookup(v), P, D, 1.0, cfg.cv_max_depth,
                 ora.export()["L"])
    table.close()


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 256, 257, 4103, 70001])
def test_ragged_sizes_and_duplicates(psf_mod, oracle_mod, n):
    rng = np.random.default_rng(n)
    v = random_vertices(rng, n, q=3, cells_per_axis=4, zero_weight_fraction=0.02)
    cfg = psf_mod.make_config(log2_capacity=14, pos_bits=3, dir_bits=2)
    # P paths of depth D with P*D = n where possible, else D = 1
    D = 1
    for d in (4, 3, 2):
        if n % d == 0:
            D = d
            break
    _run_and_compare(psf_mod, oracle_mod, cfg, [v, v[::-1].copy()], n // D, D)


def test_edge_cases(psf_mod, oracle_mod):
    import torch

    cfg = psf_mod.make_config(log2_capacity=10, pos_bits=4, dir_bits=2)
    recs = [
        vertex((0.0, 0.0, 0.0)), vertex((1.0, 1.0, 1.0)), vertex((0.5, 0.25, 0.75)),  # cell faces
        vertex((-0.03125, 0.5, 0.5), n=(0, -1, 0), d=(0, 0, -1)),
        vertex((0.3, 0.3, 0.3), d=(1.0, 0.0, 0.0)), vertex((0.3, 0.3, 0.3), d=(-1.0, 0.0, 0.0)),
        vertex((0.3, 0.3, 0.3), d=(0.0, 1.0, 0.0)), vertex((0.3, 0.3, 0.3), d=(0.0, -1.0, 0.0)),
        vertex((0.3, 0.3, 0.3), d=(0.0, 0.0, 1.0)), vertex((0.3, 0.3, 0.3), d=(0.0, 0.0, -1.0)),
        vertex((0.3, 0.3, 0.3), d=(-0.0, -0.0, -1.0)), vertex((0.3, 0.3, 0.3), n=(1, 1, 0), d=(0.6, -0.8, 0.0)),
        vertex((-2048.0, 0.0, 0.0)), vertex((2047.99, 0.0, 0.0)),  # extreme valid cells
        vertex((0.5, 0.5, 0.5), L=(np.nan, 1.0, 1.0)), vertex((0.5, 0.5, 0.5), L=(1.0, np.inf, 1.0)),
        vertex((0.5, 0.5, 0.5), w=2.0, L=(1.0, 1.0, 20000.0)), vertex((0.5, 0.5, 0.5), w=-0.5),
        vertex((0.5, 0.5, 0.5), w=40000.0), vertex((4096.0, 0.5, 0.5)), vertex((np.nan, 0.5, 0.5)),
        vertex((0.5, 0.5, 0.5), d=(0.0, 0.0, 0.0)), vertex((0.5, 0.5, 0.5), n=(np.inf, 0, 0)),
        vertex((0.5, 0.5, 0.5), w=2.0 ** -30), vertex((0.5, 0.5, 0.5), w=0.0),
        vertex((0.5, 0.5, 0.5), w=1.0, L=(32768.0, -32768.0, 0.0)),
    ]
    v = stack(recs)
    P, D = len(recs), 1
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    # empty iteration and a query of an empty table
    table.insert(torch.zeros((0, 16), dtype=torch.float32, device="cuda"))
    out0 = table.query_cv(torch.from_numpy(v).cuda(), P, D)
    assert np.array_equal(out0.cpu().numpy(), v[:, 12:15], equal_nan=True)  # one record carries a NaN on purpose
    st_ref = ora.insert(v)
    table.insert(torch.from_numpy(v).cuda())
    check_after_insert(table.export(), ora.export())
    table.update()
    ora.update()
    check_after_update(table.export(), ora.export())
    stats = table.stats()
    assert stats["status"] == st_ref == psf_mod.STATUS_RANGE
    assert (stats["dropped_vertices"], stats["zero_weight_vertices"]) == ora.counters()
    # depth-2 query over pairs to exercise the CV terms on the edge vertices
    v2 = np.concatenate([v[:12], v[12:24]])
    out = table.query_cv(torch.from_numpy(v2).cuda(), 12, 2)
    check_cv(out.cpu().numpy(), ora.query_cv(v2, 12, 2), v2, ora.lookup(v2), 12, 2, 1.0, cfg.cv_max_depth,
             ora.export()["L"])
    # the status seen by update() is the sticky bit, copied back without a sync
    table.insert(torch.from_numpy(v).cuda())
    table.update()
    torch.cuda.synchronize()
    assert table.update() & psf_mod.STATUS_RANGE
    table.close()


def test_table_full_is_reported_and_bounded(psf_mod):
    import torch

    cfg = psf_mod.make_config(log2_capacity=4, pos_bits=4, dir_bits=2)
    recs = [vertex(((i % 8) / 16.0 + 0.01, (i // 8) / 16.0 + 0.01, 0.5)) for i in range(40)]
    table = psf_mod.Table(cfg)
    table.insert(torch.from_numpy(stack(recs)).cuda())
    table.update()
    st = table.stats()
    assert st["status"] & psf_mod.STATUS_TABLE_FULL
    assert st["live_cells"] == 16 and st["dropped_vertices"] == 40 - 16
    assert st["max_probe"] == 16
    rec = table.export()
    assert len(rec) == 16 and int(rec["c_old"].sum()) == 16 << 24
    table.close()


def test_deterministic_tables_and_outputs(psf_mod):
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg_for(psf_mod, w, cache_fp16=True)
    P, D = w["width"] * w["height"], w["depth"]
    exports, outs = [], []
    for rep in range(2):
        table = psf_mod.Table(cfg)
        o = []
        for v in batches:
            dv = torch.from_numpy(v if rep == 0 else v[np.r_[P * D - 1:-1:-1]].copy()).cuda()  # reversed order
            table.insert(dv)
            table.update()
            o.append(table.query_cv(torch.from_numpy(v).cuda(), P, D).cpu().numpy())
        exports.append(table.export().tobytes())
        outs.append(np.concatenate(o).tobytes())
        table.close()
    assert exports[0] == exports[1]
    assert outs[0] == outs[1]


@pytest.mark.parametrize("knobs", [dict(insert_mode=1), dict(insert_blocks_per_sm=1, update_blocks_per_sm=1,
                                                              query_blocks_per_sm=1),
                                   dict(insert_mode=1, insert_blocks_per_sm=2), dict(vertex_staging=3),
                                   dict(sum_reduction=1), dict(sum_reduction=1, insert_mode=1, vertex_staging=0),
                                   dict(vertex_staging=3, insert_mode=1, insert_blocks_per_sm=1, query_blocks_per_sm=1),
                                   dict(query_layout=1), dict(query_layout=0, vertex_staging=2),
                                   dict(query_layout=1, query_blocks_per_sm=1)])
def test_launch_knobs_do_not_change_results(psf_mod, knobs):
    """Aggregation mode and grid shape change only the order of the integer additions."""
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg_for(psf_mod, w, cache_fp16=True)
    P, D = w["width"] * w["height"], w["depth"]
    runs = []
    for setting in ({}, knobs):
        table = psf_mod.Table(cfg)
        table.set_launch(**setting)
        assert all(table.get_launch()[k] == v for k, v in setting.items())
        outs = [table.step(torch.from_numpy(v).cuda(), P, D).cpu().numpy() for v in batches]
        runs.append((table.export().tobytes(), np.concatenate(outs).tobytes()))
        table.close()
    assert runs[0] == runs[1]


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("gamma,jb,je", [(0.0, 1, 2), (0.5, 0, 0xFFFFFFFF), (1.0, 0, 0xFFFFFFFF), (0.25, 0, 1)])
def test_biased_estimator(psf_mod, oracle_mod, fp16, gamma, jb, je):
    """Section 'Biased estimation': gamma (L - t C_next) + C; gamma = 0 at the second vertex
    is PSTF-B; gamma = 1 everywhere equals the control variate with beta = 1."""
    import torch

    from parity import check_estimator

    w, batches = _workload_batches("64x64_d3", 3)
    cfg = _cfg_for(psf_mod, w, cache_fp16=fp16)
    P, D = w["width"] * w["height"], w["depth"]
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    for v in batches:
        dv = torch.from_numpy(v).cuda()
        table.insert(dv)
        table.update()
        ora.insert(v)
        ora.update()
        out = table.query_biased(dv, P, D, gamma, jb, je).cpu().numpy()
        ref = ora.query_biased(v, P, D, gamma, jb, je)
        check_estimator(out, ref, v, ora.lookup(v), P, D, gamma, gamma, 1.0, jb, je, ora.export()["L"], fp16=fp16)
        if gamma == 1.0 and jb == 0:
            assert np.array_equal(out, table.query_cv(dv, P, D).cpu().numpy())
    table.close()


@pytest.mark.parametrize("field", [0, 1])
@pytest.mark.parametrize("fp16", [False, True])
def test_progressive_insert(psf_mod, oracle_mod, field, fp16):
    """eq. (9) update values computed in the library from the approximant at the next vertex.
    Cells and counters are exact; the value of a vertex depends on the FP32 (GPU) or FP64
    (oracle) approximant, so the fixed-point sums agree within
      |sum - ref| <= 1e-5 |ref| + 2 * (vertices in the cell) + 2
    (relative error of the fed-back approximant well below 1e-5, plus one rounding of each
    vertex's fixed-point code) and the blended values within the FP32 bound."""
    import torch

    w, batches = _workload_batches("64x64_d3", 4)
    cfg = _cfg_for(psf_mod, w, cache_fp16=fp16)
    P, D = w["width"] * w["height"], w["depth"]
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    for it, v in enumerate(batches):
        dv = torch.from_numpy(v).cuda()
        table.insert_progressive(dv, P, D, field)
        ora.insert_progressive(v, P, D, field)
        g, r = table.export(), ora.export()
        assert np.array_equal(g["key"], r["key"]) and np.array_equal(g["c_new"], r["c_new"])
        assert np.array_equal(g["c_old"], r["c_old"])
        slack = 1e-5 * np.abs(r["sum"]).astype(np.float64) + 2.0 * (r["c_new"] / 2.0 ** 24)[:, None] + 2.0
        diff = np.abs(g["sum"].astype(np.float64) - r["sum"].astype(np.float64))
        assert np.all(diff <= slack), (it, np.max(diff / slack))
        if it == 0 and field == 0:  # empty table: the Alg. 1 value is exactly L_e, so the sums agree
            assert np.max(diff) <= 2.0
        table.update()
        ora.update()
        check_after_update(table.export(), ora.export(), fp16=fp16)
    table.close()


@pytest.mark.parametrize("P,D", [(1, 1), (255, 2), (257, 3), (4103, 2), (70001, 1), (33, 6), (3, 33), (2, 32),
                                 (1000, 7), (77, 17)])
def test_staged_vertex_tiles_with_ragged_tails(psf_mod, P, D):
    """Bulk-copied vertex tiles (256 records) give the same tables and outputs as direct
    loads, including partial last tiles of every depth row."""
    import torch

    rng = np.random.default_rng(P * 10 + D)
    v = random_vertices(rng, P * D, q=3, cells_per_axis=4)
    dv = torch.from_numpy(v).cuda()
    cfg = psf_mod.make_config(log2_capacity=14, pos_bits=3, dir_bits=2, cache_fp16=bool(P % 2))
    res = []
    for staging in (0, 3):
        t = psf_mod.Table(cfg)
        t.set_launch(vertex_staging=staging, query_layout=0 if staging else 1)  # against the depth-split query
        outs = [t.step(dv, P, D).cpu().numpy() for _ in range(2)]
        outs.append(t.query_biased(dv, P, D, 0.5).cpu().numpy())
        res.append((t.export().tobytes(), np.concatenate(outs).tobytes(), t.stats()["status"]))
        t.close()
    assert res[0] == res[1]


@pytest.mark.parametrize("fp16", [False, True])
def test_key_layouts_give_identical_tables(psf_mod, fp16):
    """Keys in a dense array or inside the slot records: same slots, same results."""
    import torch

    w, batches = _workload_batches("64x64_d3", 3)
    P, D = w["width"] * w["height"], w["depth"]
    runs = []
    for layout in (1, 2):
        t = psf_mod.Table(_cfg_for(psf_mod, w, cache_fp16=fp16, key_layout=layout))
        outs = []
        for v in batches:
            dv = torch.from_numpy(v).cuda()
            outs.append(t.step(dv, P, D).cpu().numpy())
            t.insert_progressive(dv, P, D, 0)
            t.update()
            outs.append(t.query_biased(dv, P, D, 0.0, 1, 2).cpu().numpy())
        t.reset()
        st = t.stats()
        runs.append((t.export().tobytes(), np.concatenate(outs).tobytes(), st["live_cells"], st["status"]))
        t.close()
    assert runs[0] == runs[1]


def test_many_tables_reuse_pooled_status_words(psf_mod):
    """Tables take their mapped status words from slabs of 4096: creating and freeing more
    tables than a slab holds, some alive at once, leaves every table working."""
    import torch

    from helpers import random_vertices

    rng = np.random.default_rng(5)
    v = torch.from_numpy(random_vertices(rng, 96, q=2, cells_per_axis=3)).cuda()
    cfg = psf_mod.make_config(log2_capacity=10, pos_bits=2, dir_bits=1)  # 96 crowded vertices fit easily
    alive = []
    for k in range(4500):
        t = psf_mod.Table(cfg)
        if k % 500 == 0:
            t.insert(v)
            assert t.update() >= 0
            st = t.stats()
            assert st["status"] == 0 and st["iterations"] == 1 and st["live_cells"] > 0
        if k % 3 == 0:
            alive.append(t)  # keep a third alive so that words are in use while others recycle
        else:
            torch.cuda.synchronize()
            t.close(synchronize=False)
    for t in alive[::97]:
        t.insert(v)
        t.update()
        assert t.stats()["status"] == 0
    for t in alive:
        t.close()


@pytest.mark.parametrize("n", [65535, 65536])
def test_sum_range_status_and_wrapped_sums(psf_mod, oracle_mod, n):
    """At F = 32 every code is at most 2^47, so sums are exact below 2^16 vertices per
    iteration; at that count PSF_STATUS_SUM_RANGE is set and a sum that leaves the int64 range
    wraps modulo 2^64 -- on the GPU exactly as in the oracle, whatever the order of additions."""
    import torch

    recs = [vertex((0.3, 0.3, 0.3), w=1.0, L=(32768.0, -32768.0, 1.0))] * n
    v = stack(recs)
    cfg = psf_mod.make_config(log2_capacity=8, pos_bits=2, dir_bits=1, frac_bits=32)
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    table.insert(torch.from_numpy(v).cuda())
    st = ora.insert(v)
    check_after_insert(table.export(), ora.export())
    stats = table.stats()
    assert bool(stats["status"] & psf_mod.STATUS_SUM_RANGE) == bool(st & oracle_mod.STATUS_SUM_RANGE) == (n >= 65536)
    assert table.update() & psf_mod.STATUS_SUM_RANGE == (psf_mod.STATUS_SUM_RANGE if n >= 65536 else 0)
    ora.update()
    check_after_update(table.export(), ora.export())
    table.close()


@pytest.mark.parametrize("field", [0, 1])
def test_progressive_value_saturates_like_the_oracle(psf_mod, oracle_mod, field):
    """Progressive values at and past |w value| = 2^15 are saturated on both sides (keys,
    counters and dropped counts exact), and a record outside the range rule is dropped by
    its own emission even where its progressive value is small."""
    import torch

    C = 32767.0
    first = stack([vertex((0.53, 0.53, 0.53), L=(C, C, C))])
    paths = []
    for t0, le0 in ((1.0, 1.0), (1.0000001, 1.0), (2.0, 1.0), (1e30, 0.5), (0.5, 40000.0), (float("nan"), 1.0)):
        paths.append((vertex((0.03, 0.03, 0.03), L=(le0, le0, le0), t=(t0, t0, t0)), vertex((0.53, 0.53, 0.53))))
    P, D = len(paths), 2
    v = stack([p[0] for p in paths] + [p[1] for p in paths])
    cfg = psf_mod.make_config(log2_capacity=8, pos_bits=4, dir_bits=2)
    table = psf_mod.Table(cfg)
    ora = _oracle_for(oracle_mod, cfg)
    table.insert(torch.from_numpy(first).cuda())
    table.update()
    ora.insert(first)
    ora.update()
    table.insert_progressive(torch.from_numpy(v).cuda(), P, D, field)
    st = ora.insert_progressive(v, P, D, field)
    g, r = table.export(), ora.export()
    assert np.array_equal(g["key"], r["key"]) and np.array_equal(g["c_new"], r["c_new"])
    stats = table.stats()
    assert (stats["dropped_vertices"], stats["zero_weight_vertices"]) == ora.counters()
    assert stats["status"] == st == psf_mod.STATUS_RANGE
    # the saturated cell sums agree up to the FP32 rounding of the values below the bound
    assert np.all(np.abs(g["sum"].astype(np.float64) - r["sum"]) <= 1e-6 * np.abs(r["sum"]) + 2 * P)
    table.close()
