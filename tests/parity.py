"""Element-by-element comparison of the CUDA path's tables and CV outputs with the oracle.

Bars:
  * keys, fixed-point sums, c_new and c_old: bit-exact (integer work);
  * approximant L~ (FP32 blend): |x - ref| <= 1e-5 * max(|ref|, 2^-14 * max|ref|);
  * FP16 copy of L~: the same with 2e-3 (binary16 has an 11-bit significand);
  * estimator outputs out = a L - b t C_next + c C (norm-wise, the formula can cancel):
      |out - ref| <= tol * (|a||L| + |b||t|(|C_next| + floor) + |c|(|C| + floor))
    with floor = 2^-14 * max|ref L~| and tol = 1e-5 (FP32 cache) or 2e-3 (FP16 cache);
    the control variate is a = 1, b = c = beta, the biased estimator a = b = gamma, c = 1.
The floor covers values below binary16's normal range; for FP32 it is never the
binding term on these workloads.
"""

import numpy as np

TOL_FP32 = 1e-5
TOL_FP16 = 2e-3
FLOOR_REL = 2.0 ** -14


def _floor(ref_L):
    return FLOOR_REL * float(np.max(np.abs(ref_L))) if ref_L.size else 0.0


def check_after_insert(gpu, ora):
    assert gpu.shape[0] == ora.shape[0], (gpu.shape, ora.shape)
    assert np.array_equal(gpu["key"], ora["key"])
    assert np.array_equal(gpu["sum"], ora["sum"])
    assert np.array_equal(gpu["c_new"], ora["c_new"])
    assert np.array_equal(gpu["c_old"], ora["c_old"])


def check_after_update(gpu, ora, fp16=False):
    """Returns the worst relative errors (fp32, fp16) seen, for reporting."""
    assert gpu.shape[0] == ora.shape[0], (gpu.shape, ora.shape)
    assert np.array_equal(gpu["key"], ora["key"])
    assert not np.any(gpu["sum"]) and not np.any(gpu["c_new"])
    assert np.array_equal(gpu["c_old"], ora["c_old"])
    ref = ora["L"]
    fl = _floor(ref)
    scale = np.maximum(np.abs(ref), fl)
    err32 = np.abs(gpu["L"].astype(np.float64) - ref)
    bad = err32 > TOL_FP32 * scale
    assert not np.any(bad), (np.argwhere(bad)[:5], gpu["L"][bad][:5], ref[bad][:5])
    rel32 = float(np.max(err32 / np.where(scale > 0, scale, 1.0))) if ref.size else 0.0
    rel16 = None
    if fp16:
        h = gpu["L_fp16"].astype(np.uint16).view(np.float16).astype(np.float64)
        err16 = np.abs(h - ref)
        bad = err16 > TOL_FP16 * scale
        assert not np.any(bad), (np.argwhere(bad)[:5], h[bad][:5], ref[bad][:5])
        rel16 = float(np.max(err16 / np.where(scale > 0, scale, 1.0))) if ref.size else 0.0
    return rel32, rel16


def check_estimator(out_gpu, out_ref, verts, C_ref, P, D, a, b, c, j_begin, j_end, ref_L_all, fp16=False):
    """Norm-wise comparison of out_j = a L_j - b t_j C_{j+1} + c C_j (vertices j_begin <= j < j_end
    with a successor; others must be L_j exactly).  Returns the worst ratio err / bound."""
    tol = TOL_FP16 if fp16 else TOL_FP32
    out_gpu = np.asarray(out_gpu, dtype=np.float64).reshape(D * P, 3)
    L = verts[:, 12:15].astype(np.float64)
    t = verts[:, [7, 11, 15]].astype(np.float64)
    C = C_ref.reshape(D, P, 3)
    C_next = np.zeros_like(C)
    C_next[:-1] = C[1:]
    j = np.repeat(np.arange(D), P)
    on = ((j + 1 < D) & (j >= j_begin) & (j < j_end))[:, None]
    fl = _floor(ref_L_all)
    bound = tol * (np.where(on, abs(a), 1.0) * np.abs(L)
                   + on * (abs(b) * np.abs(t) * (np.abs(C_next.reshape(-1, 3)) + fl) + abs(c) * (np.abs(C_ref) + fl)))
    # non-finite inputs propagate identically on both sides: NaN where the oracle has NaN, and
    # the same signed infinity where it has one
    assert np.array_equal(np.isnan(out_gpu), np.isnan(out_ref))
    assert np.array_equal(np.isinf(out_gpu), np.isinf(out_ref))
    inf = np.isinf(out_ref)
    assert np.array_equal(out_gpu[inf], out_ref[inf])
    err = np.abs(out_gpu - out_ref)
    err[np.isnan(out_ref) | inf] = 0.0
    bad = err > bound
    assert not np.any(bad), (np.argwhere(bad)[:5], out_gpu[bad][:5], out_ref[bad][:5])
    # vertices without an estimator are copied exactly
    off = ~on[:, 0]
    assert np.array_equal(out_gpu[off], L[off].astype(np.float32).astype(np.float64), equal_nan=True)
    return float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0


def check_cv(out_gpu, out_ref, verts, C_ref, P, D, beta, cv_max_depth, ref_L_all, fp16=False):
    """The control variate: a = 1, b = c = beta on vertices j < cv_max_depth."""
    return check_estimator(out_gpu, out_ref, verts, C_ref, P, D, 1.0, beta, beta, 0, cv_max_depth, ref_L_all, fp16)
