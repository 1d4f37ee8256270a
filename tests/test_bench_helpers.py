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
                       ("slot_cache", not setup["slot_cache"])):
        assert bench.load_traffic("k_insert", False, dict(setup, **{key: other})) is None, key
    # the other key layout reads its own capture, if there is one
    other = {"inline": "dense", "dense": "inline"}[setup["key_layout"]]
    twin = [c for c in d["captures"] if c.get("key_layout") == other and c["workload"] == setup["workload"]]
    want = twin[0]["kernels"]["k_insert"]["bytes_per_launch"] if twin else None
    assert bench.load_traffic("k_insert", False, dict(setup, key_layout=other)) == want
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
    """The served form's floor per tick: the sum over the tick's sessions of each one's insert
    floor (bytes at the HBM rate or groups at the probe rate of its own footprint, whichever
    is larger) and its blend and query bytes at the HBM rate."""
    a = dict(width=4, height=2, depth=2)  # V = 16
    b = dict(width=8, height=2, depth=1)  # V = 16
    stats = {(4, 2, 0): (10, 1000), (4, 2, 1): (12, 1000), (8, 1, 0): (6, 2), (8, 1, 1): (6, 2)}
    log = [{"ms": 2.0, "items": [(a, 0, 8), (b, 0, 9)]}, {"ms": 1.0, "items": [(a, 3, 8)]}]
    hbm = 1e3  # bytes/s
    seen = []

    def rate_of(slot_bytes, touched, groups):
        seen.append((slot_bytes, touched, groups))
        return 1e3 if slot_bytes == 64 << 8 else 4e3

    r = bench.served_roofline(log, stats, 2, hbm, rate_of, True)

    def ab(V, C):
        return bench.algorithmic_bytes(V, C, True, True)

    def one(x, g, rate):
        return max(x["k_insert"] / hbm, g / rate) + (x["k_update"] + x["k_query"]) / hbm

    want = one(ab(16, 10), 1000, 1e3) + one(ab(16, 6), 2, 4e3) + one(ab(16, 12), 1000, 1e3)
    assert r["floor_ms"] == pytest.approx(1e3 * want)
    assert r["frac"] == pytest.approx(want / 3e-3)
    assert r["groups"] == 2002 and r["device_ms"] == 3.0 and r["ticks"] == 2
    assert seen == [(64 << 8, 10, 1000), (64 << 9, 6, 2), (64 << 8, 12, 1000)]


def test_group_rates_probe_each_footprint_once(monkeypatch):
    calls = []

    def fake_probe(modes, n_words, n_distinct, n_groups, reps):
        calls.append((n_words, n_distinct, n_groups))
        return {"insert_pattern_bulk32_1or": 5.0 * n_words}

    monkeypatch.setattr(bench, "atomic_probe_rates", fake_probe)
    rates = bench.GroupRates()
    assert rates(8 * 1024, 10.4, 5) == 1024.0
    assert rates(8 * 1024, 10.9, 7e6) == 1024.0  # same footprint: memoised
    assert rates(8 * 2048, 3, 5) == 2048.0
    assert calls == [(1024, 10, 1 << 22), (2048, 3, 1 << 22)]
