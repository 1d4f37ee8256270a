"""Host-side bookkeeping of the benchmark: the algorithmic bytes that the roofline divides by,
and the committed DRAM traffic, which applies only to the setup it was captured on."""

import json
import os

import pytest

import bench


def test_algorithmic_bytes_per_launch():
    V, C = 1000, 300
    a = bench.algorithmic_bytes(V, C, cache_fp16=False)
    assert a == {"k_insert": 64 * V + 72 * C, "k_update": 112 * C, "k_query": 76 * V + 24 * C}
    b = bench.algorithmic_bytes(V, C, cache_fp16=True, slot_cache=True)
    assert b == {"k_insert": 64 * V + 72 * C + 4 * V, "k_update": 120 * C, "k_query": 76 * V + 16 * C + 4 * V}


def test_committed_traffic_applies_to_its_own_setup_only():
    path = os.path.join(bench.ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        pytest.skip("no committed DRAM traffic")
    with open(path) as f:
        d = json.load(f)
    if d["kernel_source_hash"] != bench.kernel_source_hash():
        assert bench.load_traffic("k_insert", False, {}) is None  # stale counters are never used
        return
    cap = d["captures"][0]
    setup = {k: cap[k] for k in ("workload", "cache", "levels", "log2_capacity", "slot_cache", "key_layout")}
    got = bench.load_traffic("k_insert", False, setup)
    assert got == cap["kernels"]["k_insert"]["bytes_per_launch"] and got > 0
    for key, other in (("workload", "64x64_d3"), ("cache", "other"), ("levels", 7), ("log2_capacity", 3),
                       ("slot_cache", not setup["slot_cache"]),
                       ("key_layout", {"inline": "dense", "dense": "inline"}[setup["key_layout"]])):
        assert bench.load_traffic("k_insert", False, dict(setup, **{key: other})) is None, key
    # the staged insert is a different kernel: only its own capture counts
    assert bench.load_traffic("k_insert", True, setup) == cap["kernels"].get("k_insert_staged", {}).get("bytes_per_launch")


def test_sh_payload_bytes_per_launch():
    V, C = 1000, 300
    assert bench.algorithmic_bytes(V, C, cache_fp16=False, payload=1) == {
        "k_insert": 64 * V + 264 * C, "k_update": 320 * C, "k_query": 76 * V + 32 * C}


def test_oracle_sessions_aggregate_counts_every_vertex():
    """The batched line's CPU baseline runs every session once across spawned workers."""
    import bench

    ses = [dict(name=f"s{k}", width=w, height=(9 * w) // 16, depth=d, iterations=1, log2_capacity=16, pos_bits=6,
                dir_bits=3, alpha_min=0.1, radiance="glossy", seed=77 + k, camera_step=0.0, camera_x0=0.5,
                cache_fp16=True, vertices=w * ((9 * w) // 16) * d) for k, (w, d) in enumerate([(64, 2), (48, 3), (32, 4)])]
    r = bench.oracle_sessions_aggregate(ses, 2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert f"({sum(s['vertices'] for s in ses)} vertices)" in r["sample"]


def test_capture_with_its_own_sources_is_keyed_to_them(tmp_path, monkeypatch):
    """A capture of another kernel (the fused batched one) carries the hash of its own sources:
    it applies while they are unchanged, whatever the single-session kernels' hash says."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_text("kernel v1")
    setup = {"workload": "sessions_64", "slot_cache": True, "capacity_bits": 1,
             "batch_knobs": {"insert_mode": 0, "blocks_per_sm": 0}}
    d = {"kernel_source_hash": "stale", "captures": [
        dict(setup, sources=["k.cu"], source_hash=bench.kernel_source_hash(["k.cu"]),
             kernels={"k_batch": {"bytes_per_launch": 123.0}})]}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(d))
    assert bench.load_traffic("k_batch", False, setup) == 123.0
    assert bench.load_traffic("k_batch", False, dict(setup, capacity_bits=2)) is None
    assert bench.load_traffic("k_batch", False, dict(setup, batch_knobs={"insert_mode": 1, "blocks_per_sm": 0})) is None
    (tmp_path / "k.cu").write_text("kernel v2")
    assert bench.load_traffic("k_batch", False, setup) is None


def test_served_roofline_floors():
    """The served form's floor per tick: fused, the phase sums over the tick's sessions; plain,
    the sum of every launch's own floor (never below the fused one)."""
    a = dict(width=4, height=2, depth=2)  # V = 16
    b = dict(width=8, height=2, depth=1)  # V = 16
    stats = {(4, 2, 0): (10, 1000), (4, 2, 1): (12, 1000), (8, 1, 0): (6, 2), (8, 1, 1): (6, 2)}
    log = [{"ms": 2.0, "items": [(a, 0, 8), (b, 0, 8)]}, {"ms": 1.0, "items": [(a, 3, 8)]}]
    hbm, gp = 1e3, 1e3  # bytes/s, groups/s
    fused = bench.served_roofline(log, stats, 2, hbm, gp, True, True)
    plain = bench.served_roofline(log, stats, 2, hbm, gp, False, True)

    def ab(V, C):
        return bench.algorithmic_bytes(V, C, True, True)

    a0, b0, a1 = ab(16, 10), ab(16, 6), ab(16, 12)
    t0 = max((a0["k_insert"] + b0["k_insert"]) / hbm, 1002 / gp) + (a0["k_update"] + b0["k_update"] + a0["k_query"]
                                                                   + b0["k_query"]) / hbm
    t1 = max(a1["k_insert"] / hbm, 1000 / gp) + (a1["k_update"] + a1["k_query"]) / hbm
    assert fused["floor_ms"] == pytest.approx(1e3 * (t0 + t1))
    assert fused["frac"] == pytest.approx((t0 + t1) / 3e-3)
    p0 = (max(a0["k_insert"] / hbm, 1000 / gp) + (a0["k_update"] + a0["k_query"]) / hbm
          + max(b0["k_insert"] / hbm, 2 / gp) + (b0["k_update"] + b0["k_query"]) / hbm)
    assert plain["floor_ms"] == pytest.approx(1e3 * (p0 + t1))
    assert plain["floor_ms"] >= fused["floor_ms"]
    assert fused["groups"] == plain["groups"] == 2002 and fused["device_ms"] == 3.0
