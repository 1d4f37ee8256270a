"""The batched persistent kernel: every session's tables and CV outputs are the same,
bit for bit, alone and in the mix; graph capture and replay; the bounded barrier."""

import numpy as np
import pytest

from parity import check_after_update, check_cv

pytestmark = pytest.mark.gpu

# small uneven sessions (width, depth): 16:9 images, depth 2..6
SHAPES = [(64, 3), (40, 2), (96, 6), (33, 4), (128, 5), (72, 2), (50, 3)]


def _session(k, w, d):
    import math

    from synth.scene import config4_q_bits

    h = int(round(9 * w / 16))
    v = w * h * d
    log2cap = int(math.ceil(math.log2(v))) + 1
    levels = 3 if k % 4 == 1 else 1  # some tables have hierarchy levels (more cells: more capacity)
    return dict(name=f"s{k}", width=w, height=h, depth=d, log2_capacity=log2cap + (2 if levels > 1 else 0),
                pos_bits=config4_q_bits(log2cap, 3), dir_bits=3, alpha_min=0.1, radiance="glossy",
                seed=4000 + k, camera_step=0.0, camera_x0=0.5, cache_fp16=bool(k % 2),
                key_layout=2 if k % 3 == 2 else 0, levels=levels)  # some keep their keys in the slot records


def _data(sessions, iterations):
    from synth.scene import iteration_vertices, make_scene

    return [[iteration_vertices(s, it, make_scene(s["seed"])) for it in range(iterations)] for s in sessions]


def _table(psf, s):
    return psf.Table(psf.make_config(log2_capacity=s["log2_capacity"], pos_bits=s["pos_bits"], dir_bits=s["dir_bits"],
                                      alpha_min=s["alpha_min"], cache_fp16=s["cache_fp16"],
                                      key_layout=s.get("key_layout", 0), levels=s.get("levels", 1)))


@pytest.mark.parametrize("insert_mode", [0, 1])
def test_batch_matches_alone_and_oracle(psf_mod, oracle_mod, insert_mode):
    import torch

    sessions = [_session(k, w, d) for k, (w, d) in enumerate(SHAPES)]
    data = _data(sessions, 3)
    alone = [_table(psf_mod, s) for s in sessions]
    mixed = [_table(psf_mod, s) for s in sessions]
    oracles = [oracle_mod.Oracle(pos_bits=s["pos_bits"], dir_bits=s["dir_bits"],
                                 alpha_min=float(np.float32(s["alpha_min"])), levels=s["levels"]) for s in sessions]
    batch = psf_mod.Batch(len(sessions), insert_mode=insert_mode)
    # every other session carries a slot cache: the batched kernel notes and reads its slots
    slots = [torch.empty(s["width"] * s["height"] * s["depth"], dtype=torch.int32, device="cuda") if k % 2 == 0
             else None for k, s in enumerate(sessions)]
    for it in range(3):
        dev = [torch.from_numpy(data[k][it]).cuda() for k in range(len(sessions))]
        outs_b = [torch.empty((d.shape[0], 3), device="cuda") for d in dev]
        batch.step([(mixed[k], dev[k], outs_b[k], s["width"] * s["height"], s["depth"]) +
                    ((slots[k],) if slots[k] is not None else ()) for k, s in enumerate(sessions)])
        for k, s in enumerate(sessions):
            P, D = s["width"] * s["height"], s["depth"]
            out_a = alone[k].step(dev[k], P, D)
            ra, rb = alone[k].export(), mixed[k].export()
            assert ra.tobytes() == rb.tobytes(), f"session {k} table differs in the mix"
            assert np.array_equal(out_a.cpu().numpy(), outs_b[k].cpu().numpy()), f"session {k} output differs"
            o = oracles[k]
            o.insert(data[k][it])
            o.update()
            check_after_update(rb, o.export(), fp16=s["cache_fp16"])
            check_cv(outs_b[k].cpu().numpy(), o.query_cv(data[k][it], P, D), data[k][it], o.lookup(data[k][it], P, D), P, D,
                     1.0, 0xFFFFFFFF, o.export()["L"], fp16=s["cache_fp16"])
    assert batch.status() == 0
    for k, t in enumerate(mixed):
        st = t.stats()
        assert st["status"] == 0 and st["iterations"] == 3
        assert st["touched_cells"] == alone[k].stats()["touched_cells"]
    batch.close()


def test_batch_graph_capture_replay_and_membership_change(psf_mod):
    import torch

    sessions = [_session(k, w, d) for k, (w, d) in enumerate(SHAPES[:4])]
    data = _data(sessions, 3)
    static_in = [torch.empty((data[k][0].shape[0], 16), device="cuda") for k in range(len(sessions))]
    static_out = [torch.empty((data[k][0].shape[0], 3), device="cuda") for k in range(len(sessions))]
    graph_tables = [_table(psf_mod, s) for s in sessions]
    ref_tables = [_table(psf_mod, s) for s in sessions]
    batch = psf_mod.Batch(len(sessions))
    entries = [(graph_tables[k], static_in[k], static_out[k], s["width"] * s["height"], s["depth"])
               for k, s in enumerate(sessions)]
    batch.set(entries)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.launch()
    for it in range(3):
        # session 3 leaves after the first iteration: new descriptors, same graph
        live = list(range(len(sessions))) if it == 0 else [0, 1, 2]
        if it == 1:
            batch.set([entries[k] for k in live])
            torch.cuda.synchronize()
        for k in live:
            static_in[k].copy_(torch.from_numpy(data[k][it]))
        g.replay()
        for k in live:
            s = sessions[k]
            ref = ref_tables[k].step(torch.from_numpy(data[k][it]).cuda(), s["width"] * s["height"], s["depth"])
            assert np.array_equal(ref.cpu().numpy(), static_out[k].cpu().numpy()), (it, k)
            assert graph_tables[k].export().tobytes() == ref_tables[k].export().tobytes(), (it, k)
    assert graph_tables[3].stats()["iterations"] == 1
    batch.close()


def test_batch_barrier_timeout_is_reported_and_the_context_survives(psf_mod):
    """A barrier told to wait for a block that does not exist gives up after its bound."""
    import torch

    s = _session(0, 40, 2)
    data = _data([s], 1)[0][0]
    t = _table(psf_mod, s)
    dv = torch.from_numpy(data).cuda()
    out = torch.zeros((dv.shape[0], 3), device="cuda")
    bad = psf_mod.Batch(1, barrier_timeout_us=20000, test_phantom_blocks=1)
    bad.step([(t, dv, out, s["width"] * s["height"], s["depth"])])
    assert bad.status() & psf_mod.STATUS_TIMEOUT
    assert t.stats()["status"] & psf_mod.STATUS_TIMEOUT
    bad.close()
    # the device is still usable: a normal batch on a fresh table works
    t2 = _table(psf_mod, s)
    good = psf_mod.Batch(1)
    good.step([(t2, dv, out, s["width"] * s["height"], s["depth"])])
    assert good.status() == 0 and t2.stats()["status"] == 0
    ref = _table(psf_mod, s)
    assert np.array_equal(ref.step(dv, s["width"] * s["height"], s["depth"]).cpu().numpy(), out.cpu().numpy())
    good.close()


def test_batch_empty_and_zero_size_items(psf_mod):
    import torch

    s = _session(1, 40, 2)
    data = _data([s], 1)[0][0]
    t, t0 = _table(psf_mod, s), _table(psf_mod, s)
    b = psf_mod.Batch(4)
    b.step([])
    empty = torch.empty((0, 16), device="cuda")
    dv = torch.from_numpy(data).cuda()
    out = torch.empty((dv.shape[0], 3), device="cuda")
    b.step([(t0, empty, torch.empty((0, 3), device="cuda"), 0, 3), (t, dv, out, s["width"] * s["height"], s["depth"])])
    assert b.status() == 0
    assert t0.stats()["live_cells"] == 0 and t0.stats()["iterations"] == 1
    ref = _table(psf_mod, s)
    assert np.array_equal(ref.step(dv, s["width"] * s["height"], s["depth"]).cpu().numpy(), out.cpu().numpy())
    b.close()
