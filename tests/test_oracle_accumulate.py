"""Pins for the oracle's accumulation (eq. 5-6), blend (eq. 10-11) and reset.

Each check compares the oracle with something other than itself: an O(n^2)
brute-force grouping, exact conservation sums, a hand-derived sequence, the
closed form of the blend recursion and a constant field."""

import json
import math
import os

import numpy as np
import pytest

from helpers import fixed, random_vertices, stack, vertex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_blend.json")


def _brute_force(oracle_mod, cfg, verts, frac_bits=24):
    """Group by full key with pairwise compares; returns {key: [sr, sg, sb, c]}."""
    groups = []  # list of (key, sums)
    for v in verts:
        key = oracle_mod.vertex_key(cfg, v)
        w = np.float32(v[3])
        prods = [np.float32(w * np.float32(v[12 + c])) for c in range(3)]
        if key is None or not (0.0 <= w <= 32768.0) or any((not np.isfinite(x)) or abs(x) > 32768.0 for x in prods):
            continue
        cw = int(fixed(w, frac_bits))
        if cw == 0:
            continue
        add = [int(fixed(x, frac_bits)) for x in prods] + [cw]
        for gk, gs in groups:
            if gk == key:
                for i in range(4):
                    gs[i] += add[i]
                break
        else:
            groups.append((key, add))
    return dict(groups)


@pytest.mark.parametrize("seed,frac_bits", [(0, 24), (1, 24), (2, 24), (3, 8), (4, 16), (5, 32)])
def test_brute_force_matches_map(oracle_mod, seed, frac_bits):
    rng = np.random.default_rng(seed)
    q, d = 2, 1
    verts = random_vertices(rng, 200, q=q, cells_per_axis=2, zero_weight_fraction=0.05)
    cfg = oracle_mod.make_config(pos_bits=q, dir_bits=d, frac_bits=frac_bits)
    o = oracle_mod.Oracle(cfg)
    assert o.insert(verts) == 0
    rec = o.export()
    bf = _brute_force(oracle_mod, cfg, verts, frac_bits)
    assert len(rec) == len(bf) and len(bf) < 120  # many vertices share a cell
    for r in rec:
        assert [int(r["sum"][0]), int(r["sum"][1]), int(r["sum"][2]), int(r["c_new"])] == bf[int(r["key"])]
    assert list(rec["key"]) == sorted(rec["key"])


def test_inserted_weight_equals_cell_weight(oracle_mod):
    """Sum over cells of the counters equals the sum over vertices, bit-exact (fixed point)."""
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    o = oracle_mod.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"])
    for it in range(3):
        v = iteration_vertices(w, it)
        assert o.insert(v) == 0
        rec = o.export()
        assert int(rec["c_new"].sum()) == int(fixed(v[:, 3]).sum())
        for c in range(3):
            assert int(rec["sum"][:, c].sum()) == int(fixed(v[:, 3] * v[:, 12 + c]).sum())
        o.update()
        rec = o.export()
        assert int(rec["c_new"].sum()) == 0 and int(np.abs(rec["sum"]).sum()) == 0
        assert int(rec["c_old"].sum()) == int(fixed(v[:, 3]).sum()) * (it + 1)


def test_range_rule_and_zero_weight(oracle_mod):
    cfg = oracle_mod.make_config(pos_bits=4, dir_bits=2)
    good = vertex((0.5, 0.5, 0.5), L=(1.0, 2.0, 3.0))
    bad = [
        vertex((0.5, 0.5, 0.5), L=(np.nan, 1.0, 1.0)),
        vertex((0.5, 0.5, 0.5), L=(1.0, np.inf, 1.0)),
        vertex((0.5, 0.5, 0.5), w=2.0, L=(1.0, 1.0, 20000.0)),  # |w L| > 2^15
        vertex((0.5, 0.5, 0.5), w=-0.5),
        vertex((0.5, 0.5, 0.5), w=40000.0),
        vertex((4096.0, 0.5, 0.5)),  # cell index out of the 16-bit range
        vertex((0.5, 0.5, 0.5), d=(0.0, 0.0, 0.0)),
    ]
    o = oracle_mod.Oracle(cfg)
    st = o.insert(stack([good] + bad + [vertex((0.5, 0.5, 0.5), w=2.0 ** -30)]))
    assert st == oracle_mod.STATUS_RANGE
    assert o.counters() == (len(bad), 1)
    rec = o.export()
    assert len(rec) == 1 and int(rec[0]["c_new"]) == 1 << 24
    # |w L| exactly 2^15 is still accepted
    o2 = oracle_mod.Oracle(cfg)
    assert o2.insert(stack([vertex((0.5, 0.5, 0.5), w=1.0, L=(32768.0, -32768.0, 0.0))])) == 0
    assert int(o2.export()[0]["sum"][0]) == 32768 << 24 and int(o2.export()[0]["sum"][1]) == -(32768 << 24)


def test_hand_derived_blend_sequence(oracle_mod):
    g = json.load(open(GOLDEN))
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2, alpha_min=g["alpha_min"])
    for it in g["iterations"]:
        if it["reset_before"]:
            o.reset()
        o.insert(stack([vertex((0.5, 0.5, 0.5), w=w, L=L) for w, L in it["vertices_wL"]]))
        r = o.export()
        assert len(r) == 1
        assert [int(x) for x in r[0]["sum"]] == it["after_insert"]["sum"]
        assert int(r[0]["c_new"]) == it["after_insert"]["c_new"]
        o.update()
        r = o.export()
        assert int(r[0]["c_old"]) == it["after_update"]["c_old"]
        np.testing.assert_allclose(r[0]["L"], it["after_update"]["L"], rtol=1e-15, atol=0)


def test_constant_field_reproduces_the_constant(oracle_mod):
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    o_nd = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    rng = np.random.default_rng(11)
    for it in range(4):
        v = iteration_vertices(w, it)
        v[:, 12:15] = 0.75  # dyadic constant with w = 1: every iteration's mean is exactly 0.75
        o.insert(v)
        o.update()
        # (1 - alpha) * 0.75 + alpha * 0.75 rounds by at most an ulp or two per step, and the
        # blend is a contraction, so the error stays at the level of a few ulps
        L = o.export()["L"]
        np.testing.assert_allclose(L, 0.75, rtol=1e-14)
        if it == 0:
            assert np.all(L == 0.75)  # first touch: alpha = 1, L = the exact mean
        v2 = v.copy()
        v2[:, 3] = rng.uniform(0.25, 2.0, size=len(v2)).astype(np.float32)
        v2[:, 12:15] = 0.3
        o_nd.insert(v2)
        o_nd.update()
        # error bound: one FP32 rounding of w*L (2^-24 relative) plus the fixed-point
        # rounding 0.5 / (w * 0.3 * 2^24) <= 4e-7 relative for w >= 0.25
        np.testing.assert_allclose(o_nd.export()["L"], float(np.float32(0.3)), rtol=5e-7)


def _blend_closed_form(xs, alphas):
    """L_k = sum_i alpha_i x_i prod_{m=i+1..k} (1 - alpha_m), with L_0 = 0."""
    k = len(xs)
    out = 0.0
    for i in range(k):
        prod = 1.0
        for m in range(i + 1, k):
            prod *= 1.0 - alphas[m]
        out += alphas[i] * xs[i] * prod
    return out


@pytest.mark.parametrize("alpha_min,mode", [(0.1, 0), (0.3, 0), (0.0, 0), (0.25, 1)])
def test_blend_matches_closed_form(oracle_mod, alpha_min, mode):
    """Constant weight per iteration: c_old = (k-1) c so alpha_k = max(k^-1/2, alpha_min)
    (eq. 11), or alpha_min in the constant-alpha mode; L_k follows the product formula."""
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2, alpha_min=alpha_min, blend_mode=mode)
    per_iter = 3
    xs, alphas = [], []
    for k in range(1, 41):
        x = float(k)  # x_k = k, exact in fixed point
        o.insert(stack([vertex((0.5, 0.5, 0.5), L=(x, 2 * x, 0.5 * x))] * per_iter))
        o.update()
        xs.append(x)
        alphas.append(max(k ** -0.5, alpha_min) if mode == 0 else alpha_min)
        r = o.export()[0]
        want = _blend_closed_form(xs, alphas)
        np.testing.assert_allclose(r["L"], [want, 2 * want, 0.5 * want], rtol=1e-12)
        assert int(r["c_old"]) == k * per_iter << 24
    if mode == 0 and alpha_min == 0.0:
        # without the floor the square-root schedule still reproduces a constant input exactly
        o2 = oracle_mod.Oracle(pos_bits=4, dir_bits=2, alpha_min=0.0)
        for _ in range(10):
            o2.insert(stack([vertex((0.5, 0.5, 0.5), L=(5.0, 5.0, 5.0))]))
            o2.update()
        np.testing.assert_allclose(o2.export()[0]["L"], 5.0, rtol=1e-15)


def test_untouched_cells_keep_their_state(oracle_mod):
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    a = vertex((0.1, 0.1, 0.1), L=(1.0, 1.0, 1.0))
    b = vertex((0.9, 0.9, 0.9), L=(3.0, 3.0, 3.0))
    o.insert(stack([a, b]))
    o.update()
    before = o.export()
    o.insert(stack([a]))
    o.update()
    after = o.export()
    kb = oracle_mod.vertex_key(o.cfg, b)
    rb0 = before[before["key"] == kb][0]
    rb1 = after[after["key"] == kb][0]
    assert rb0.tobytes() == rb1.tobytes()


def test_reset_clears_counters_only(oracle_mod):
    """The global counter reset (Section "Temporal averaging"): c_old := 0 everywhere, the
    approximant kept -- a query before the next update reads the same values, an untouched
    cell keeps its approximant, and a touched one takes alpha = 1 (its new mean)."""
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    a = vertex((0.1, 0.1, 0.1), L=(1.0, 2.0, 4.0))
    b = vertex((0.9, 0.9, 0.9), L=(3.0, 5.0, 7.0))
    path = stack([a, b])  # one path of depth 2: a's CV reads b's cell
    for _ in range(3):
        o.insert(path)
        o.update()
    before = o.export()
    q0 = o.query_cv(path, 1, 2)
    o.reset()
    mid = o.export()
    assert np.array_equal(mid["L"], before["L"]) and not np.any(mid["c_old"])
    assert np.array_equal(o.query_cv(path, 1, 2), q0)
    o.insert(stack([vertex((0.1, 0.1, 0.1), L=(8.0, 8.0, 8.0))]))
    o.update()
    after = o.export()
    kb = oracle_mod.vertex_key(o.cfg, b)
    assert np.array_equal(after[after["key"] == kb]["L"], before[before["key"] == kb]["L"])
    ka = oracle_mod.vertex_key(o.cfg, a)
    assert np.array_equal(after[after["key"] == ka]["L"][0], [8.0, 8.0, 8.0])


def test_counter_saturates(oracle_mod):
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    v = vertex((0.5, 0.5, 0.5))
    key = oracle_mod.vertex_key(o.cfg, v)
    rec = np.zeros(1, dtype=oracle_mod.RECORD_DTYPE)
    rec["key"] = key
    rec["c_old"] = np.iinfo(np.int64).max - 5
    rec["L"] = 2.0
    o.import_records(rec)
    o.insert(stack([v]))
    o.update()
    r = o.export()[0]
    assert int(r["c_old"]) == np.iinfo(np.int64).max
    assert math.isclose(float(r["L"][0]), 0.9 * 2.0 + 0.1 * 1.0, rel_tol=1e-12)  # alpha = alpha_min


@pytest.mark.parametrize("n,wraps", [(65535, False), (65536, True)])
def test_sum_range_rule_and_modular_sums(oracle_mod, n, wraps):
    """Sum range: with F = 32 every code is at most 2^47 in magnitude, so sums are exact while
    fewer than 2^(48-32) = 65536 vertices reach the table in one iteration; at that count the
    status bit is set, and sums that leave the int64 range wrap modulo 2^64 (two's complement).
    Here every vertex adds +2^47 (red), -2^47 (green) and 2^32 (weight) to one cell."""
    v = stack([vertex((0.3, 0.3, 0.3), w=1.0, L=(32768.0, -32768.0, 1.0))] * n)
    o = oracle_mod.Oracle(pos_bits=2, dir_bits=1, frac_bits=32)
    st = o.insert(v)
    assert bool(st & oracle_mod.STATUS_SUM_RANGE) == wraps
    r = o.export()[0]

    def as_int64(x):
        x %= 1 << 64
        return x - (1 << 64) if x >= 1 << 63 else x

    assert int(r["sum"][0]) == as_int64(n << 47)  # 2^63 wraps to -2^63
    assert int(r["sum"][1]) == as_int64(-(n << 47))  # -2^63 is still representable
    assert int(r["c_new"]) == n << 32
    o.update()
    assert o.insert(v[:1]) == 0  # the update starts a new count


def test_sum_range_counts_every_insert_of_the_iteration(oracle_mod):
    """The count covers all vertices handed to the inserts between two updates, dropped ones too."""
    bad = vertex((0.3, 0.3, 0.3), w=-1.0)  # dropped by the range rule, still counted
    good = vertex((0.3, 0.3, 0.3))
    o = oracle_mod.Oracle(pos_bits=2, dir_bits=1, frac_bits=32)
    assert o.insert(stack([bad] * 40000)) == oracle_mod.STATUS_RANGE
    assert o.insert(stack([good] * 25535)) == 0
    assert o.insert(stack([good])) == oracle_mod.STATUS_SUM_RANGE
