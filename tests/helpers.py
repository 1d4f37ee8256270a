"""Small input builders shared by the tests (no method arithmetic here)."""

import numpy as np


def vertex(p, n=(0.0, 0.0, 1.0), d=(0.0, 0.0, -1.0), w=1.0, L=(1.0, 1.0, 1.0), t=(0.5, 0.5, 0.5)):
    """One 16-float vertex record: v0=(p,w) v1=(n,tr) v2=(d,tg) v3=(L,tb)."""
    return np.array([p[0], p[1], p[2], w, n[0], n[1], n[2], t[0], d[0], d[1], d[2], t[1],
                     L[0], L[1], L[2], t[2]], dtype=np.float32)


def stack(records):
    return np.ascontiguousarray(np.stack(records).astype(np.float32))


def fixed(x, frac_bits=24):
    """round-to-nearest-even(x * 2^F) of float32 values, as int64."""
    return np.rint(np.asarray(x, dtype=np.float32).astype(np.float64) * float(2 ** frac_bits)).astype(np.int64)


def random_vertices(rng, n, *, q, cells_per_axis=3, n_dirs=4, face_fraction=0.2, zero_weight_fraction=0.0):
    """Vertices crowded into a few cells and directions so that many share a key."""
    h = 2.0 ** -q
    cell = rng.integers(0, cells_per_axis, size=(n, 3))
    frac = rng.random((n, 3))
    on_face = rng.random((n, 3)) < face_fraction
    frac[on_face] = 0.0
    p = (cell + frac) * h
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    nrm = axes[rng.integers(0, 6, size=n)] + 0.3 * rng.standard_normal((n, 3)) * (rng.random((n, 1)) < 0.5)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dir_set = rng.standard_normal((n_dirs, 3))
    dir_set /= np.linalg.norm(dir_set, axis=1, keepdims=True)
    d = dir_set[rng.integers(0, n_dirs, size=n)] + 0.05 * rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w = rng.uniform(0.0, 2.0, size=n)
    w[rng.random(n) < zero_weight_fraction] = 2.0 ** -30
    L = rng.lognormal(0.0, 1.0, size=(n, 3))
    t = rng.uniform(0.1, 0.9, size=(n, 3))
    out = np.empty((n, 16), dtype=np.float32)
    out[:, 0:3], out[:, 3] = p, w
    out[:, 4:7], out[:, 7] = nrm, t[:, 0]
    out[:, 8:11], out[:, 11] = d, t[:, 1]
    out[:, 12:15], out[:, 15] = L, t[:, 2]
    return out
