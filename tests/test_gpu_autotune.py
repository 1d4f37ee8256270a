"""The autotuner on the GPU: every candidate it times -- launch knobs of psf_step, the load
factor of a session, the batched kernel's knobs and the sessions' load factor -- leaves
the tables bit-identical (same cells, sums, counters and approximants), and the candidate it
returns is one of those it timed."""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _batches(name, n):
    import torch

    from synth.scene import iteration_vertices, make_scene, workload

    w = workload(name)
    scene = make_scene(w["seed"])
    return w, [torch.from_numpy(iteration_vertices(w, it, scene)).cuda() for it in range(n)]


@pytest.mark.parametrize("fp16", [False, True])
def test_every_table_candidate_gives_identical_tables(psf_mod, fp16):
    from paper_2005_07547_b300 import autotune

    w, batches = _batches("64x64_d3", 3)
    P, D = w["width"] * w["height"], w["depth"]
    cfg = psf_mod.make_config(log2_capacity=w["log2_capacity"], pos_bits=w["pos_bits"], dir_bits=w["dir_bits"],
                              alpha_min=w["alpha_min"], cache_fp16=fp16)
    res = autotune.tune_table(cfg, batches, P, D, warmup=2, iters=2, verify=True)
    n = int(np.prod([len(v) for v in autotune.TABLE_SPACE.values()]))
    assert res["verified"] == len(res["all"]) == n
    assert res["best"] in [{k: r[k] for k in autotune.TABLE_SPACE} for r in res["all"]]
    # the key layout is a table field: each candidate gets a table laid out its way
    res = autotune.tune_table(cfg, batches, P, D, space={"key_layout": (1, 2), "query_layout": (0, 1)}, warmup=2,
                              iters=2, verify=True, slot_cache=True)
    assert res["verified"] == len(res["all"]) == 4 and res["best"]["key_layout"] in (1, 2)
    cap = autotune.tune_capacity(cfg, batches, P, D, extra_bits=(1, 2, 3), verify=True)
    assert cap["verified"] == 3 and cap["best"] in [r["log2_capacity"] for r in cap["all"]]


def test_every_batch_candidate_gives_identical_tables(psf_mod):
    import torch

    from paper_2005_07547_b300 import autotune
    from synth.scene import config4_q_bits, iteration_vertices

    shapes = [(64, 3), (40, 2), (96, 6), (33, 4), (128, 5)]
    sessions = []
    for k, (wd, d) in enumerate(shapes):
        h = int(round(9 * wd / 16))
        cap = int(math.ceil(math.log2(wd * h * d))) + 1
        sessions.append(dict(width=wd, height=h, depth=d, pos_bits=config4_q_bits(cap, 3), dir_bits=3, alpha_min=0.1,
                             radiance="glossy", seed=6000 + k, camera_step=0.0, camera_x0=0.5, cache_fp16=bool(k % 2)))
    data = [torch.from_numpy(iteration_vertices(s, 0)).cuda() for s in sessions]
    outs = [torch.empty((d.shape[0], 3), device="cuda") for d in data]
    slots = [torch.empty(d.shape[0], dtype=torch.int32, device="cuda") for d in data]

    def make(capacity_bits=1, key_layout=0):
        tables = []
        for s in sessions:
            V = s["width"] * s["height"] * s["depth"]
            tables.append(psf_mod.Table(psf_mod.make_config(
                log2_capacity=int(math.ceil(math.log2(V))) + capacity_bits, pos_bits=s["pos_bits"],
                dir_bits=s["dir_bits"], alpha_min=s["alpha_min"], cache_fp16=s["cache_fp16"], key_layout=key_layout)))
        return [(tables[k], data[k], outs[k], s["width"] * s["height"], s["depth"], slots[k])
                for k, s in enumerate(sessions)]

    space = {**autotune.BATCH_SPACE, "capacity_bits": (1, 2)}
    res = autotune.tune_batch(make, len(sessions), space=space, verify=True)
    n = int(np.prod([len(v) for v in space.values()]))
    assert res["verified"] == len(res["all"]) == n
    assert all(math.isfinite(r["ms"]) for r in res["all"])
    assert "capacity_bits" in res["best"]
    # the key layout as a table field of the search, with the load factor
    space = {"capacity_bits": (1, 2), "key_layout": (1, 2)}
    res = autotune.tune_batch(make, len(sessions), space=space, verify=True)
    assert res["verified"] == len(res["all"]) == 4
    assert {(r["capacity_bits"], r["key_layout"]) for r in res["all"]} == {(1, 1), (1, 2), (2, 1), (2, 2)}
