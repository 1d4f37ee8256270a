"""Pins for the oracle's hierarchy levels (Section "Progressive hierarchical solver": a
hierarchy of finite elements H_l, and eq. (9) reads a suitably chosen level).

Level l uses cells 2^l times wider than level 0 along each position axis (the level sits in
the key's level bits; the direction and normal bins do not change).  Every vertex lands in
one cell per level; a vertex at path depth j reads level min(j, levels - 1).  Checked here
against keys derived by hand, an integer regrouping of the level-0 cells, flat tables at
the coarser resolution and flat tables holding each vertex's read value at level 0."""

import numpy as np
import pytest

from helpers import random_vertices, stack, vertex

REC_FIELDS = ("sum", "c_new", "c_old", "L")


def _level(key):
    return (int(key) >> 61) & 3


def _split(key):
    k = int(key)
    return ((k >> 58) & 7, (k >> 48) & 0x3FF, ((k >> 32) & 0xFFFF) - 32768, ((k >> 16) & 0xFFFF) - 32768,
            (k & 0xFFFF) - 32768)


def _join(level, nb, dbin, x, y, z):
    return (level << 61) | (nb << 58) | (dbin << 48) | ((x + 32768) << 32) | ((y + 32768) << 16) | (z + 32768)


def test_level_keys_by_hand(oracle_mod):
    # p = (-0.3, 0.7, 0.05), q = 4: cell width 2^(l-4); floor(p * 2^(4-l)) per level.
    # level 0: (-5, 11, 0); level 1: (-3, 5, 0); level 2: (-2, 2, 0); level 3: (-1, 1, 0).
    # Normal +z -> bin 4; omega_o = +z -> octahedral (0, 0) -> bins (2, 2) at d = 2 -> dbin 10.
    cfg = oracle_mod.make_config(pos_bits=4, dir_bits=2, levels=4)
    v = vertex((-0.3, 0.7, 0.05))
    want = {0: (-5, 11, 0), 1: (-3, 5, 0), 2: (-2, 2, 0), 3: (-1, 1, 0)}
    for level, (x, y, z) in want.items():
        assert oracle_mod.vertex_key(cfg, v, level) == _join(level, 4, 10, x, y, z), level
    # a vertex outside the level-0 index range has no cell at any level
    far = vertex((4096.0, 0.0, 0.0))
    assert all(oracle_mod.vertex_key(cfg, far, level) is None for level in range(4))


@pytest.mark.parametrize("seed", [0, 1])
def test_coarse_cells_are_the_integer_regrouping_of_fine_cells(oracle_mod, seed):
    """Sums and counters of a level-l cell equal those of the level-0 cells whose signed
    indices floor-divide by 2^l onto it (integers, so exactly), after several iterations."""
    rng = np.random.default_rng(seed)
    q, levels = 3, 3
    o = oracle_mod.Oracle(pos_bits=q, dir_bits=1, levels=levels)
    for it in range(3):
        verts = random_vertices(rng, 400, q=q, cells_per_axis=6)
        verts[:, 0:3] -= np.float32(0.4)  # negative indices exercise the floor
        assert o.insert(verts) == 0
        rec = o.export()
        by_level = [rec[[_level(k) == l for k in rec["key"]]] for l in range(levels)]
        assert len(by_level[0]) > 2 * len(by_level[2]) > 0  # the regrouping merges cells
        for l in range(1, levels):
            groups = {}
            for r in by_level[0]:
                nb, dbin, x, y, z = _split(r["key"])
                g = groups.setdefault(_join(l, nb, dbin, x >> l, y >> l, z >> l), np.zeros(5, dtype=np.int64))
                g += np.array([*r["sum"], r["c_new"], r["c_old"]], dtype=np.int64)
            coarse = {int(r["key"]): np.array([*r["sum"], r["c_new"], r["c_old"]], dtype=np.int64)
                      for r in by_level[l]}
            assert coarse.keys() == groups.keys()
            for k, g in groups.items():
                assert np.array_equal(coarse[k], g), (it, l, hex(k))
        o.update()


def test_each_level_is_a_flat_table_at_the_coarser_resolution(oracle_mod):
    """Level l of a table at pos_bits q holds exactly what a flat table at pos_bits q - l
    holds, blended values included, over several insert/update iterations."""
    rng = np.random.default_rng(7)
    q, levels = 4, 3
    hier = oracle_mod.Oracle(pos_bits=q, dir_bits=2, levels=levels, alpha_min=0.05)
    flats = [oracle_mod.Oracle(pos_bits=q - l, dir_bits=2, alpha_min=0.05) for l in range(levels)]
    for it in range(4):
        verts = random_vertices(rng, 300, q=q, cells_per_axis=5)
        verts[:, 0:3] -= np.float32(0.25)
        hier.insert(verts)
        for f in flats:
            f.insert(verts)
        hier.update()
        for f in flats:
            f.update()
        rec = hier.export()
        for l, f in enumerate(flats):
            mine = rec[[_level(k) == l for k in rec["key"]]]
            ref = f.export()
            assert np.array_equal(mine["key"] & np.uint64((1 << 61) - 1), ref["key"]), (it, l)
            for field in REC_FIELDS:
                assert np.array_equal(mine[field], ref[field]), (it, l, field)


def test_one_level_is_the_flat_table(oracle_mod):
    rng = np.random.default_rng(3)
    verts = random_vertices(rng, 240, q=3, cells_per_axis=4)
    P, D = 80, 3
    a, b = oracle_mod.Oracle(pos_bits=3, levels=0), oracle_mod.Oracle(pos_bits=3, levels=1)
    for o in (a, b):
        o.insert(verts)
        o.update()
    assert a.export().tobytes() == b.export().tobytes()
    assert np.array_equal(a.query_cv(verts, P, D), b.query_cv(verts, P, D))


def _spread_path(D):
    """One path of depth D whose vertices sit in distinct cells at every level (q = 4 and
    up to 3 levels: cells at most 1/4 wide, vertices 1 apart)."""
    return stack([vertex((1.0 * j + 0.1, -0.6, 0.3), w=1.0, L=(0.2 * j, 0.1, 1.0 + j), t=(0.5, 0.25, 0.75))
                  for j in range(D)])


def _records(oracle_mod, cfg, verts, value_of):
    """Imported records: the cell of vertex j at level l holds value_of(j, l) (RGB)."""
    rec = np.zeros(0, dtype=oracle_mod.RECORD_DTYPE)
    out = []
    for j, v in enumerate(verts):
        for l in range(max(cfg.levels, 1)):
            r = np.zeros(1, dtype=oracle_mod.RECORD_DTYPE)
            r["key"] = oracle_mod.vertex_key(cfg, v, l)
            r["L"] = value_of(j, l)
            r["c_old"] = 1
            out.append(r)
    return np.concatenate(out) if out else rec


@pytest.mark.parametrize("levels", [2, 3])
def test_reads_take_level_min_j_top_and_reduce_to_a_flat_table(oracle_mod, levels):
    """Vertex j reads its cell at level min(j, levels - 1): the lookups return the value
    planted at that level, and the CV query, the biased query and the progressive insert
    give the same bits as a flat table whose level-0 cells hold those read values."""
    D, P = 5, 1
    verts = _spread_path(D)
    hier_cfg = oracle_mod.make_config(pos_bits=4, dir_bits=2, levels=levels, beta=0.75)
    flat_cfg = oracle_mod.make_config(pos_bits=4, dir_bits=2, levels=1, beta=0.75)

    def value(j, l):
        return (10.0 * l + j, 0.5 + l, 3.0 - 0.25 * j)

    top = levels - 1
    hier = oracle_mod.Oracle(hier_cfg)
    hier.import_records(_records(oracle_mod, hier_cfg, verts, value))
    flat = oracle_mod.Oracle(flat_cfg)
    flat.import_records(_records(oracle_mod, flat_cfg, verts, lambda j, l: value(j, min(j, top))))

    C = hier.lookup(verts, P, D)
    for j in range(D):
        assert np.array_equal(C[j], np.array(value(j, min(j, top)))), j
    assert np.array_equal(hier.query_cv(verts, P, D), flat.query_cv(verts, P, D))
    for gamma, jb, je in ((0.3, 0, D), (0.0, 1, 3)):
        assert np.array_equal(hier.query_biased(verts, P, D, gamma, jb, je), flat.query_biased(verts, P, D, gamma, jb, je))
    for field in (0, 1):
        h2, f2 = oracle_mod.Oracle(hier_cfg), oracle_mod.Oracle(flat_cfg)
        h2.import_records(_records(oracle_mod, hier_cfg, verts, value))
        f2.import_records(_records(oracle_mod, flat_cfg, verts, lambda j, l: value(j, min(j, top))))
        h2.insert_progressive(verts, P, D, field)
        f2.insert_progressive(verts, P, D, field)
        hr, fr = h2.export(), f2.export()
        for l in range(levels):  # the update values land in every level's cell
            mine = hr[[_level(k) == l for k in hr["key"]]]
            want = {oracle_mod.vertex_key(hier_cfg, v, l): oracle_mod.vertex_key(flat_cfg, v) for v in verts}
            fsum = {int(r["key"]): (tuple(r["sum"]), int(r["c_new"])) for r in fr}
            for r in mine:
                assert (tuple(r["sum"]), int(r["c_new"])) == fsum[want[int(r["key"])]], (field, l)
