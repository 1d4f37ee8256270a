"""Pins for the oracle's cell keys (Section 'Basis functions and data structures:
spatio-directional hashing'): hand-derived keys, cell faces, normal bins, and the
octahedral direction grid checked through its inverse map."""

import json
import math
import os

import numpy as np
import pytest

from helpers import vertex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_keys.json")


def _fields(key, d):
    dbin = (key >> 48) & 0x3FF
    return dict(level=(key >> 61) & 3, nbin=(key >> 58) & 7, bu=dbin >> d, bv=dbin & ((1 << d) - 1),
                x=((key >> 32) & 0xFFFF) - 32768, y=((key >> 16) & 0xFFFF) - 32768, z=(key & 0xFFFF) - 32768)


def test_hand_derived_keys(oracle_mod):
    g = json.load(open(GOLDEN))
    for case in g["cases"]:
        cfg = oracle_mod.make_config(pos_bits=case["q"], dir_bits=case["d"], use_normal=case["use_normal"])
        assert oracle_mod.vertex_key(cfg, case["vertex"]) == int(case["key"], 16), case["derivation"]


def test_invalid_vertices_have_no_key(oracle_mod):
    g = json.load(open(GOLDEN))
    for case in g["invalid"]:
        cfg = oracle_mod.make_config(pos_bits=case["q"], dir_bits=case["d"])
        assert oracle_mod.vertex_key(cfg, case["vertex"]) is None, case["why"]


@pytest.mark.parametrize("q", [0, 3, 7, 12])
def test_cell_faces_belong_to_the_upper_cell(oracle_mod, q):
    cfg = oracle_mod.make_config(pos_bits=q, dir_bits=2)
    h = 2.0 ** -q
    for k in range(-5, 6):
        for p, want in [(k * h, k), ((k + 0.5) * h, k),
                        (float(np.nextafter(np.float32(k * h), np.float32(-np.inf))), k - 1)]:
            key = oracle_mod.vertex_key(cfg, vertex((p, p, p)))
            f = _fields(key, 2)
            assert (f["x"], f["y"], f["z"]) == (want, want, want), (q, k, p)


def test_normal_bins(oracle_mod):
    cfg = oracle_mod.make_config(pos_bits=2, dir_bits=2, use_normal=True)
    cases = {(1, 0, 0): 0, (-1, 0, 0): 1, (0, 1, 0): 2, (0, -1, 0): 3, (0, 0, 1): 4, (0, 0, -1): 5,
             (1, 1, 0): 0, (-1, 1, 0): 1, (0, 1, 1): 2, (0, -1, 1): 3, (1, 1, 1): 0, (0.2, -0.3, -0.9): 5,
             (0.0, -0.0, 0.0): 0}
    for n, want in cases.items():
        key = oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), n=n))
        assert _fields(key, 2)["nbin"] == want, n
    cfg0 = oracle_mod.make_config(pos_bits=2, dir_bits=2, use_normal=False)
    for n in cases:
        assert _fields(oracle_mod.vertex_key(cfg0, vertex((0.3, 0.3, 0.3), n=n)), 2)["nbin"] == 0


def _octahedral_decode(u, v):
    """Inverse of the octahedral map: a point of [-1,1]^2 back to a unit direction."""
    if abs(u) + abs(v) <= 1.0:
        w = np.array([u, v, 1.0 - abs(u) - abs(v)])
    else:
        su = 1.0 if u >= 0 else -1.0
        sv = 1.0 if v >= 0 else -1.0
        w = np.array([(1.0 - abs(v)) * su, (1.0 - abs(u)) * sv, 1.0 - abs(u) - abs(v)])
    return w / np.linalg.norm(w)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_octahedral_bin_centres_round_trip(oracle_mod, d):
    """Decoding the centre of every bin and encoding it again returns the same bin."""
    cfg = oracle_mod.make_config(pos_bits=2, dir_bits=d)
    n = 1 << d
    for bu in range(n):
        for bv in range(n):
            u = -1.0 + (bu + 0.5) * 2.0 / n
            v = -1.0 + (bv + 0.5) * 2.0 / n
            omega = _octahedral_decode(u, v)
            key = oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), d=tuple(-omega)))
            f = _fields(key, d)
            assert (f["bu"], f["bv"]) == (bu, bv), (d, bu, bv, omega)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_axis_directions(oracle_mod, d):
    cfg = oracle_mod.make_config(pos_bits=2, dir_bits=d)
    mid, top = 1 << (d - 1), (1 << d) - 1
    # omega_o -> expected (bu, bv); the vertex stores d = -omega_o
    cases = {(0, 0, 1): (mid, mid), (0, 0, -1): (top, top), (1, 0, 0): (top, mid), (-1, 0, 0): (0, mid),
             (0, 1, 0): (mid, top), (0, -1, 0): (mid, 0)}
    for omega, want in cases.items():
        key = oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), d=tuple(-float(c) for c in omega)))
        f = _fields(key, d)
        assert (f["bu"], f["bv"]) == want, (omega, f)


def test_direction_bins_are_scale_invariant_and_mirror(oracle_mod):
    """Bins depend only on the direction; mirroring x mirrors the u bin (away from bin edges)."""
    rng = np.random.default_rng(7)
    d = 3
    cfg = oracle_mod.make_config(pos_bits=2, dir_bits=d)
    n = 1 << d
    for _ in range(300):
        bu, bv = rng.integers(0, n, size=2)
        u = -1.0 + (bu + rng.uniform(0.2, 0.8)) * 2.0 / n
        v = -1.0 + (bv + rng.uniform(0.2, 0.8)) * 2.0 / n
        omega = _octahedral_decode(u, v)
        k1 = _fields(oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), d=tuple(-omega))), d)
        k2 = _fields(oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), d=tuple(-4.0 * omega))), d)
        mir = omega * np.array([-1.0, 1.0, 1.0])
        k3 = _fields(oracle_mod.vertex_key(cfg, vertex((0.3, 0.3, 0.3), d=tuple(-mir))), d)
        assert (k1["bu"], k1["bv"]) == (bu, bv)
        assert (k2["bu"], k2["bv"]) == (bu, bv)
        assert (k3["bu"], k3["bv"]) == (n - 1 - bu, bv)


def test_key_order_matches_tuple_order(oracle_mod):
    """Packed keys sort like the (level, normal, direction, x, y, z) tuple."""
    cfg = oracle_mod.make_config(pos_bits=3, dir_bits=2)
    rng = np.random.default_rng(3)
    keys = []
    for _ in range(200):
        p = rng.uniform(-2, 2, size=3)
        nrm = rng.standard_normal(3)
        dr = rng.standard_normal(3)
        k = oracle_mod.vertex_key(cfg, vertex(tuple(p), n=tuple(nrm), d=tuple(dr)))
        keys.append(k)
    tup = [tuple(_fields(k, 2)[f] for f in ("level", "nbin", "bu", "bv", "x", "y", "z")) for k in keys]
    assert sorted(range(200), key=lambda i: keys[i]) == sorted(range(200), key=lambda i: (tup[i], keys[i]))
    assert all(k < (1 << 63) for k in keys)
    assert not math.isnan(sum(keys))


def test_cell_index_range_edges(oracle_mod):
    """The index range is [-2^15, 2^15): at q = 0 the cell of x is floor(x) (float32 holds
    these values exactly), so 32767.5 and -32768.0 have cells and 32768.0 and -32768.5 do not;
    an accepted index is stored biased by 2^15 in 16 bits."""
    cfg = oracle_mod.make_config(pos_bits=0, dir_bits=1)
    inside = {32767.5: 65535, -32768.0: 0, 0.25: 32768, -0.25: 32767}
    for x, biased in inside.items():
        k = oracle_mod.vertex_key(cfg, vertex((x, 0.0, 0.0)))
        assert k is not None and (k >> 32) & 0xFFFF == biased, x
    for x in (32768.0, -32768.5):
        assert oracle_mod.vertex_key(cfg, vertex((x, 0.0, 0.0))) is None, x
