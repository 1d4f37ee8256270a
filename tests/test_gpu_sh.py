"""Parity of the YCoCg two-band SH payload (Section "Basis functions and data structures:
spatio-directional hashing", last paragraph) with the SH oracle, through the C ABI.

Bars:
  * keys, the sixteen fixed-point sums and c_old: bit-exact;
  * the six coefficients (a, g, Co, Cg) after each blend: norm-wise per cell,
      |x - ref| <= TOL_SH * (|a| + |g|_1 + |Co| + |Cg| + floor);
  * control-variate outputs: norm-wise, with each cell value bounded by its coefficient norm
      |out - ref| <= TOL_SH * (|L| + beta |t| (3 K_{j+1} + floor) + beta (3 K_j + floor)),
    K the cell's |a| + |g . n| + |Co| + |Cg| (each RGB channel adds three of them).
TOL_SH: the GPU solves the 3x3 regularised normal equations in FP32 (moments rounded once
from exact 128-bit integers, a Cholesky factorisation), so its relative error is a few units
of 2^-24 times the system's condition number, at most 1 + 1/ridge for unit normals (the
centred second moments of unit vectors have eigenvalues at most 1):
    TOL_SH = 1e-5 + 16 * 2^-24 * (1 + 1/ridge).
"""

import numpy as np
import pytest

from helpers import random_vertices

pytestmark = pytest.mark.gpu


def _tol(ridge):
    return 1e-5 + 16 * 2.0 ** -24 * (1.0 + 1.0 / ridge)


def _pair(psf, oracle_mod, log2cap, q, d, ridge, **kw):
    cfg = psf.make_config(log2_capacity=log2cap, pos_bits=q, dir_bits=d, use_normal=False, payload=1, sh_ridge=ridge,
                          **kw)
    ora = oracle_mod.ShOracle(pos_bits=q, dir_bits=d, use_normal=False, ridge=float(np.float32(ridge)),
                              alpha_min=float(np.float32(cfg.alpha_min)), beta=float(np.float32(cfg.beta)),
                              cv_max_depth=cfg.cv_max_depth, frac_bits=cfg.frac_bits, blend_mode=cfg.blend_mode)
    return cfg, psf.Table(cfg), ora


def _check_sums(g, r):
    assert g.shape[0] == r.shape[0], (g.shape, r.shape)
    assert np.array_equal(g["key"], r["key"])
    assert np.array_equal(g["sum"], r["sum"])
    assert np.array_equal(g["c_old"], r["c_old"])


def _coef_scale(coef):
    return np.abs(coef[:, 0]) + np.abs(coef[:, 1:4]).sum(axis=1) + np.abs(coef[:, 4:]).sum(axis=1)


def _check_coef(g, r, tol):
    assert g.shape[0] == r.shape[0], (g.shape, r.shape)
    assert np.array_equal(g["key"], r["key"]) and np.array_equal(g["c_old"], r["c_old"])
    assert not np.any(g["sum"])
    scale = _coef_scale(r["coef"])
    fl = 2.0 ** -14 * (float(np.max(scale)) if scale.size else 0.0)
    err = np.abs(g["coef"].astype(np.float64) - r["coef"])
    bound = tol * (scale + fl)[:, None]
    bad = err > bound
    assert not np.any(bad), (np.argwhere(bad)[:5], g["coef"][np.any(bad, axis=1)][:3], r["coef"][np.any(bad, axis=1)][:3])
    return float(np.max(err / bound)) if err.size else 0.0


def _cell_norm(oracle_mod, ora, v):
    """K per vertex: |a| + |g . n| + |Co| + |Cg| of its cell at its normal (0 if absent)."""
    rec = ora.export()
    by_key = {int(k): c for k, c in zip(rec["key"], rec["coef"])}
    K = np.zeros(v.shape[0])
    for i in range(v.shape[0]):
        k = oracle_mod.vertex_key(ora.cfg, v[i])
        c = by_key.get(k) if k is not None else None
        if c is not None:
            K[i] = abs(c[0]) + abs(float(c[1:4] @ v[i, 4:7].astype(np.float64))) + abs(c[4]) + abs(c[5])
    return K


def _check_cv(oracle_mod, ora, out_gpu, v, P, D, beta, tol):
    ref = ora.query_cv(v, P, D)
    K = _cell_norm(oracle_mod, ora, v).reshape(D, P)
    Kn = np.zeros_like(K)
    Kn[:-1] = K[1:]
    fl = 2.0 ** -14 * float(np.max(K)) if K.size else 0.0
    on = (np.arange(D)[:, None] + 1 < D).repeat(P, axis=1).reshape(-1, 1)
    L = v[:, 12:15].astype(np.float64)
    t = v[:, [7, 11, 15]].astype(np.float64)
    bound = tol * (np.abs(L) + on * (beta * np.abs(t) * (3 * Kn.reshape(-1, 1) + fl) + beta * (3 * K.reshape(-1, 1) + fl)))
    out = np.asarray(out_gpu, dtype=np.float64)
    err = np.abs(out - ref)
    bad = err > bound
    assert not np.any(bad), (np.argwhere(bad)[:5], out[bad][:5], ref[bad][:5])
    assert np.array_equal(out[~on[:, 0]], L[~on[:, 0]].astype(np.float32).astype(np.float64))
    return float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0


@pytest.mark.parametrize("ridge", [0.01, 0.1])
@pytest.mark.parametrize("insert_mode", [0, 1])
def test_sh_payload_64x64_all_iterations(psf_mod, oracle_mod, ridge, insert_mode):
    import torch

    from synth.scene import iteration_vertices, make_scene, workload

    w = workload("64x64_d3")
    scene = make_scene(w["seed"])
    P, D = w["width"] * w["height"], w["depth"]
    cfg, table, ora = _pair(psf_mod, oracle_mod, w["log2_capacity"], w["pos_bits"], w["dir_bits"], ridge,
                            alpha_min=w["alpha_min"])
    table.set_launch(insert_mode=insert_mode)
    tol = _tol(ridge)
    worst = [0.0, 0.0]
    for it in range(w["iterations"]):
        v = iteration_vertices(w, it, scene)
        dv = torch.from_numpy(v).cuda()
        table.insert(dv)
        st = ora.insert(v)
        _check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        worst[0] = max(worst[0], _check_coef(table.export(), ora.export(), tol))
        out = table.query_cv(dv, P, D).cpu().numpy()
        worst[1] = max(worst[1], _check_cv(oracle_mod, ora, out, v, P, D, 1.0, tol))
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
    cfg, table, ora = _pair(psf_mod, oracle_mod, 14, 3, 2, 0.02, beta=0.75)
    tol = _tol(0.02)
    for it in range(3):
        vi = v if it % 2 == 0 else v[::-1].copy()
        dv = torch.from_numpy(vi).cuda()
        table.insert(dv)
        ora.insert(vi)
        _check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        _check_coef(table.export(), ora.export(), tol)
        out = table.query_cv(dv, P, D).cpu().numpy()
        _check_cv(oracle_mod, ora, out, vi, P, D, float(np.float32(0.75)), tol)
    table.close()


def test_sh_payload_reset_and_edge_vertices(psf_mod, oracle_mod):
    import torch

    from helpers import stack, vertex

    recs = [vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, 1.0)), vertex((0.3, 0.3, 0.3), n=(0.0, 1.0009765625, 0.0)),
            vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, -1.001)), vertex((0.3, 0.3, 0.3), w=2.0 ** -30),
            vertex((0.3, 0.3, 0.3), L=(1.0, np.nan, 1.0)), vertex((0.3, 0.3, 0.3), n=(0.6, 0.8, 0.0)),
            vertex((0.3, 0.3, 0.3), w=2.0, L=(16384.0, -16384.0, 0.0), n=(0.0, 0.6, 0.8))]
    v = stack(recs)
    cfg, table, ora = _pair(psf_mod, oracle_mod, 8, 2, 1, 0.01)
    for it in range(3):
        if it == 2:
            table.reset()
            ora.reset()
        table.insert(torch.from_numpy(v).cuda())
        st = ora.insert(v)
        _check_sums(table.export(), ora.export())
        table.update()
        ora.update()
        _check_coef(table.export(), ora.export(), _tol(0.01))
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
    slots = torch.zeros(4, dtype=torch.int32, device="cuda")
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
