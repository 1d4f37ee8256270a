"""Comparators of the YCoCg two-band SH payload against the SH oracle, shared by the SH
parity tests.

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


def tol_sh(ridge):
    return 1e-5 + 16 * 2.0 ** -24 * (1.0 + 1.0 / ridge)


def sh_pair(psf, oracle_mod, log2cap, q, d, ridge, **kw):
    cfg = psf.make_config(log2_capacity=log2cap, pos_bits=q, dir_bits=d, use_normal=False, payload=1, sh_ridge=ridge,
                          **kw)
    ora = oracle_mod.ShOracle(pos_bits=q, dir_bits=d, use_normal=False, ridge=float(np.float32(ridge)),
                              alpha_min=float(np.float32(cfg.alpha_min)), beta=float(np.float32(cfg.beta)),
                              cv_max_depth=cfg.cv_max_depth, frac_bits=cfg.frac_bits, blend_mode=cfg.blend_mode)
    return cfg, psf.Table(cfg), ora


def check_sums(g, r):
    assert g.shape[0] == r.shape[0], (g.shape, r.shape)
    assert np.array_equal(g["key"], r["key"])
    assert np.array_equal(g["sum"], r["sum"])
    assert np.array_equal(g["c_old"], r["c_old"])


def coef_scale(coef):
    return np.abs(coef[:, 0]) + np.abs(coef[:, 1:4]).sum(axis=1) + np.abs(coef[:, 4:]).sum(axis=1)


def check_coef(g, r, tol):
    assert g.shape[0] == r.shape[0], (g.shape, r.shape)
    assert np.array_equal(g["key"], r["key"]) and np.array_equal(g["c_old"], r["c_old"])
    assert not np.any(g["sum"])
    scale = coef_scale(r["coef"])
    fl = 2.0 ** -14 * (float(np.max(scale)) if scale.size else 0.0)
    err = np.abs(g["coef"].astype(np.float64) - r["coef"])
    bound = tol * (scale + fl)[:, None]
    bad = err > bound
    assert not np.any(bad), (np.argwhere(bad)[:5], g["coef"][np.any(bad, axis=1)][:3], r["coef"][np.any(bad, axis=1)][:3])
    return float(np.max(err / bound)) if err.size else 0.0


def cell_norm(oracle_mod, ora, v):
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


def check_cv_sh(oracle_mod, ora, out_gpu, v, P, D, beta, tol):
    ref = ora.query_cv(v, P, D)
    K = cell_norm(oracle_mod, ora, v).reshape(D, P)
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
