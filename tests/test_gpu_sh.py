"""Parity of the YCoCg two-band SH payload (Section "Basis functions and data structures:
spatio-directional hashing", last paragraph) with the SH oracle, through the C ABI, with
the bars of `sh_parity`."""

import numpy as np
import pytest

from helpers import random_vertices
from sh_parity import check_coef, check_cv_sh, check_sums, sh_pair, tol_sh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ridge", [0.01, 0.1])
@pytest.mark.parametrize("insert_mode", [0, 1])
def test_sh_payload_64x64_all_iterations(psf_mod, oracle_mod, ridge, insert_mode):
    import torch

    from synth.scene import iteration_vertices, make_scene, workload

    w = workload("64x64_d3")
    scene = make_scene(w["seed"])
    P, D = w["width"] * w["height"], w["depth"]
    _, table, ora = sh_pair(psf_mod, oracle_mod, w["log2_capacity"], w["pos_bits"], w["dir_bits"], ridge,
                            alpha_min=w["alpha_min"])
    table.set_launch(insert_mode=insert_mode)
    tol = tol_sh(ridge)
    worst = [0.0, 0.0]
    for it in range(w["iterations"]):
        v = iteration_vertices(w, it, scene)
        dv = torch.from_numpy(v).cuda()
        table.insert(dv)
        st = ora.insert(v)
        check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        worst[0] = max(worst[0], check_coef(table.export(), ora.export(), tol))
        out = table.query_cv(dv, P, D).cpu().numpy()
        worst[1] = max(worst[1], check_cv_sh(oracle_mod, ora, out, v, P, D, 1.0, tol))
        stats = table.stats()
        assert stats["status"] == st and (stats["dropped_vertices"], stats["zero_weight_vertices"]) == ora.counters()
        assert stats["live_cells"] == len(ora)
    # cells on the spheres and at the box's edges see several normals: band 1 is in use
    g = table.export()["coef"][:, 1:4]
    assert np.mean(np.any(g != 0.0, axis=1)) > 0.1
    print("worst err/bound (coefficients, cv):", worst)
    table.close()


@pytest.mark.parametrize("n", [1, 31, 33, 257, 4103, 70001])
def test_sh_payload_ragged_crowded_cells(psf_mod, oracle_mod, n):
    import torch

    rng = np.random.default_rng(100 + n)
    v = random_vertices(rng, n, q=3, cells_per_axis=3, zero_weight_fraction=0.02)
    D = next((d for d in (4, 3, 2) if n % d == 0), 1)
    P = n // D
    _, table, ora = sh_pair(psf_mod, oracle_mod, 14, 3, 2, 0.02, beta=0.75)
    tol = tol_sh(0.02)
    for it in range(3):
        vi = v if it % 2 == 0 else v[::-1].copy()
        dv = torch.from_numpy(vi).cuda()
        table.insert(dv)
        ora.insert(vi)
        check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        check_coef(table.export(), ora.export(), tol)
        out = table.query_cv(dv, P, D).cpu().numpy()
        check_cv_sh(oracle_mod, ora, out, vi, P, D, float(np.float32(0.75)), tol)
    table.close()


def test_sh_payload_reset_and_edge_vertices(psf_mod, oracle_mod):
    import torch

    from helpers import stack, vertex

    recs = [vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, 1.0)), vertex((0.3, 0.3, 0.3), n=(0.0, 1.0009765625, 0.0)),
            vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, -1.001)), vertex((0.3, 0.3, 0.3), w=2.0 ** -30),
            vertex((0.3, 0.3, 0.3), L=(1.0, np.nan, 1.0)), vertex((0.3, 0.3, 0.3), n=(0.6, 0.8, 0.0)),
            vertex((0.3, 0.3, 0.3), w=2.0, L=(16384.0, -16384.0, 0.0), n=(0.0, 0.6, 0.8))]
    v = stack(recs)
    _, table, ora = sh_pair(psf_mod, oracle_mod, 8, 2, 1, 0.01)
    for it in range(3):
        if it == 2:
            table.reset()
            ora.reset()
        table.insert(torch.from_numpy(v).cuda())
        st = ora.insert(v)
        check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        check_coef(table.export(), ora.export(), tol_sh(0.01))
    stats = table.stats()
    assert stats["status"] == st == psf_mod.STATUS_RANGE
    assert (stats["dropped_vertices"], stats["zero_weight_vertices"]) == ora.counters()
    table.close()


def test_sh_tables_are_rejected_where_the_payload_does_not_apply(psf_mod):
    import ctypes

    import torch

    from paper_2005_07547_b300 import _abi

    lib = _abi.load()
    t = psf_mod.Table(psf_mod.make_config(log2_capacity=10, payload=1))
    dv = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bad = _abi.PSF_ERR_INVALID_ARG
    assert lib.psf_insert_progressive(t.handle, dv.data_ptr(), 4, 1, 0, s) == bad
    n = ctypes.c_size_t()
    assert lib.psf_export(t.handle, None, 0, ctypes.byref(n), s) == bad
    items = (_abi.BatchItem * 1)(_abi.BatchItem(t.handle, dv.data_ptr(), out.data_ptr(), 4, 1, None))
    assert lib.psf_batch_step_noalloc(items, 1, None, s) == bad
    b = psf_mod.Batch(1)
    with pytest.raises(RuntimeError):
        b.set([(t, dv, out, 4, 1)])
    b.close()
    rgb = psf_mod.Table(psf_mod.make_config(log2_capacity=10))
    assert lib.psf_export_sh(rgb.handle, None, 0, ctypes.byref(n), s) == bad
    rgb.close()
    t.close()


@pytest.mark.parametrize("insert_mode", [0, 1])
def test_sh_slot_cache_gives_the_same_tables_and_outputs(psf_mod, insert_mode):
    """The slot-cache insert leaves the same table as the plain insert, and the query that reads
    each vertex's fit at its noted slot returns the probing query's outputs bit for bit
    (vertices that were not added -- range rule, zero weight -- fall back to probing)."""
    import torch

    rng = np.random.default_rng(7)
    P, D = 3001, 3
    v = random_vertices(rng, P * D, q=3, cells_per_axis=4, zero_weight_fraction=0.05)
    v[::97, 4] = 2.0  # a few normals outside the unit-normal range rule
    dv = torch.from_numpy(v).cuda()
    cfg = psf_mod.make_config(log2_capacity=14, pos_bits=3, dir_bits=2, use_normal=False, payload=1, sh_ridge=0.02)
    a, b = psf_mod.Table(cfg), psf_mod.Table(cfg)
    a.set_launch(insert_mode=insert_mode)
    b.set_launch(insert_mode=insert_mode)
    for it in range(3):
        a.insert(dv)
        slots = b.insert_slots(dv, P, D)
        assert a.export().tobytes() == b.export().tobytes()
        a.update()
        b.update()
        want = a.query_cv(dv, P, D).cpu().numpy()
        got = b.query_cv_slots(dv, slots, P, D).cpu().numpy()
        assert np.array_equal(want, got, equal_nan=True), it
        assert (slots.cpu().numpy() == -1).sum() > 0  # some vertices were not added
    assert a.stats()["status"] == b.stats()["status"] == psf_mod.STATUS_RANGE
    a.close()
    b.close()
