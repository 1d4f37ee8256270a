"""Pins for the oracle's YCoCg two-band SH payload (Section "Basis functions and data
structures: spatio-directional hashing", last paragraph: luminance in two spherical-
harmonics bands over the normal, chroma per cell).

The oracle fits each cell's luminance per iteration by weighted least squares over the two
SH bands (span {1, n_x, n_y, n_z}: Y(n) ~ a + g . n) with a ridge on band 1, from exact
integer moments, and blends the six coefficients (a, g, Co, Cg) with eq. (10)-(11).  These
pins hold it to things fixed outside its own code: numpy's least-squares solver on the
textbook weighted ridge problem built from the raw samples; exact reproduction of a
luminance that is linear in the normal; the already-pinned RGB oracle, which a cell with a
single normal or an overwhelming ridge must reproduce; YCoCg's published inverse; the blend's
closed form; and brute-force fixed-point sums."""

import math

import numpy as np
import pytest

from helpers import stack, vertex

F = 24


def _ycocg(rgb):
    r, g, b = rgb[..., 0], rgb[..., 1], rgb[..., 2]
    return np.stack([r / 4 + g / 2 + b / 4, r / 2 - b / 2, g / 2 - r / 4 - b / 4], axis=-1)


def _unit(rng, n, spread, axis=(0.0, 0.0, 1.0)):
    v = np.asarray(axis)[None, :] + spread * rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _cell_vertices(rng, n, normals, rgb, w, pos=(0.53, 0.53, 0.53)):
    """n vertices in one cell (same position and direction), given normals, RGB and weights."""
    return stack([vertex(pos, n=tuple(normals[i]), d=(0.1, 0.2, -1.0), w=float(w[i]), L=tuple(rgb[i]))
                  for i in range(n)])


def _textbook_fit(v, ridge):
    """argmin sum w (Y - a - g.n)^2 + ridge * W |g|^2 by numpy's least squares on the raw
    samples (float64 of the float32 inputs), and the weighted chroma means."""
    w = v[:, 3].astype(np.float64)
    n = v[:, 4:7].astype(np.float64)
    ycc = _ycocg(v[:, 12:15].astype(np.float64))
    sw = np.sqrt(w)[:, None]
    A = np.hstack([np.ones((len(w), 1)), n]) * sw
    b = ycc[:, 0] * sw[:, 0]
    if ridge > 0:
        A = np.vstack([A, np.hstack([np.zeros((3, 1)), math.sqrt(ridge * w.sum()) * np.eye(3)])])
        b = np.concatenate([b, np.zeros(3)])
    sol = np.linalg.lstsq(A, b, rcond=None)[0]
    co = float(np.sum(w * ycc[:, 1]) / w.sum())
    cg = float(np.sum(w * ycc[:, 2]) / w.sum())
    return np.array([sol[0], sol[1], sol[2], sol[3], co, cg])


def _one_cell(oracle_mod, v, ridge, **kw):
    o = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=ridge, use_normal=False, **kw)
    o.insert(v)
    o.update()
    rec = o.export()
    assert len(rec) == 1
    return o, rec[0]


@pytest.mark.parametrize("ridge", [0.0, 1e-3, 0.01, 0.3])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_first_fit_equals_textbook_weighted_ridge_regression(oracle_mod, ridge, seed):
    rng = np.random.default_rng(seed)
    n = 40
    normals = _unit(rng, n, 0.6)
    v = _cell_vertices(rng, n, normals, rng.lognormal(0.0, 1.0, (n, 3)), rng.uniform(0.2, 2.0, n))
    _, rec = _one_cell(oracle_mod, v, ridge)  # first touch: alpha = 1, the approximant is the fit
    want = _textbook_fit(v, ridge)
    scale = np.abs(want[0]) + np.abs(want[1:4]).sum() + np.abs(want[4:]).sum()
    assert np.all(np.abs(rec["coef"] - want) <= 1e-6 * scale), (rec["coef"], want)


def test_linear_luminance_in_the_normal_is_reproduced(oracle_mod):
    rng = np.random.default_rng(7)
    n = 30
    normals = _unit(rng, n, 0.8)
    a0, g0 = 2.0, np.array([0.5, -0.25, 0.75])
    Y = a0 + normals @ g0
    v = _cell_vertices(rng, n, normals, np.repeat(Y[:, None], 3, axis=1), rng.uniform(0.5, 1.5, n))
    _, rec = _one_cell(oracle_mod, v, 0.0)
    assert np.allclose(rec["coef"][:4], [a0, *g0], rtol=0, atol=2e-6)
    assert np.allclose(rec["coef"][4:], 0.0, atol=1e-7)  # grey: no chroma


def test_ridge_shrinks_a_linear_gradient_by_its_closed_form(oracle_mod):
    """For Y = a0 + g0 . n the ridge solution is g = (S + ridge I)^-1 S g0 with S the weighted
    covariance of the normals, and a = mean(Y) - g . mean(n)."""
    rng = np.random.default_rng(8)
    n, ridge = 50, 0.05
    normals = _unit(rng, n, 0.5)
    w = rng.uniform(0.5, 1.5, n)
    a0, g0 = 1.0, np.array([0.3, 0.2, -0.4])
    Y = a0 + normals @ g0
    v = _cell_vertices(rng, n, normals, np.repeat(Y[:, None], 3, axis=1), w)
    _, rec = _one_cell(oracle_mod, v, ridge)
    wn = v[:, 3].astype(np.float64)
    nn = v[:, 4:7].astype(np.float64)
    S = np.cov(nn.T, aweights=wn, bias=True)
    g = np.linalg.solve(S + ridge * np.eye(3), S @ g0)
    Yv = a0 + nn @ g0
    a = np.average(Yv, weights=wn) - g @ np.average(nn, axis=0, weights=wn)
    assert np.allclose(rec["coef"][:4], [a, *g], rtol=0, atol=5e-6)


@pytest.mark.parametrize("normal", [(0.0, 0.0, 1.0), (-1.0, 0.0, 0.0), (0.0, 1.0, 0.0)])
def test_single_axis_normal_cell_equals_the_rgb_oracle(oracle_mod, normal):
    """All normals equal (a wall): the normal moments have no spread, band 1 is exactly 0 and
    the cell's RGB at any normal is the RGB oracle's weighted mean (up to the FP32 rounding of
    the YCoCg codes), over several iterations."""
    rng = np.random.default_rng(11)
    sh = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=0.01, use_normal=False)
    rgb = oracle_mod.Oracle(pos_bits=2, dir_bits=1, use_normal=False)
    for it in range(4):
        n = 25
        normals = np.tile(normal, (n, 1))
        v = _cell_vertices(rng, n, normals, rng.lognormal(0, 1, (n, 3)), np.ones(n))
        sh.insert(v)
        rgb.insert(v)
        sh.update()
        rgb.update()
        rec = sh.export()[0]
        assert np.all(rec["coef"][1:4] == 0.0)
        probe = stack([vertex((0.53, 0.53, 0.53), n=tuple(_unit(rng, 1, 1.0)[0]), d=(0.1, 0.2, -1.0))])
        # the luminance and chroma codes are rounded once in FP32 before fixed point
        assert np.allclose(sh.lookup(probe)[0], rgb.export()[0]["L"], rtol=0, atol=4e-7 * np.max(rgb.export()[0]["L"]))
        assert rec["c_old"] == rgb.export()[0]["c_old"]


def test_overwhelming_ridge_reduces_to_the_rgb_oracle_everywhere(oracle_mod):
    """With band 1 suppressed the payload is eq. (6)'s mean in YCoCg: on a whole synthetic
    iteration sequence every cell's RGB equals the RGB oracle's, keys and counters included."""
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    sh = oracle_mod.ShOracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], ridge=1e15,
                             alpha_min=float(np.float32(0.1)))
    rgb = oracle_mod.Oracle(pos_bits=w["pos_bits"], dir_bits=w["dir_bits"], alpha_min=float(np.float32(0.1)))
    for it in range(3):
        v = iteration_vertices(w, it)
        assert sh.insert(v) == rgb.insert(v)
        sh.update()
        rgb.update()
    a, b = sh.export(), rgb.export()
    assert np.array_equal(a["key"], b["key"]) and np.array_equal(a["c_old"], b["c_old"])
    assert np.max(np.abs(a["coef"][:, 1:4])) < 1e-9 * np.max(np.abs(a["coef"][:, 0]))
    got = sh.lookup(v)
    want = rgb.lookup(v)
    # Y, Co and Cg are each rounded once in FP32 (relative 2^-24 of at most max|RGB|) before
    # fixed point, and each output channel adds three of them
    row = np.max(np.abs(want), axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= 4e-7 * row)


def test_ycocg_inverse_on_the_lookup(oracle_mod):
    """A grey-free cell: the lookup turns (Y, Co, Cg) back into the input colour exactly
    (R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg)."""
    rng = np.random.default_rng(3)
    n = 10
    rgb = np.tile([[0.9, 0.2, 0.4]], (n, 1))
    v = _cell_vertices(rng, n, np.tile((0.0, 1.0, 0.0), (n, 1)), rgb, np.ones(n))
    o, rec = _one_cell(oracle_mod, v, 0.01)
    assert np.allclose(o.lookup(v[:1])[0], np.float32(rgb[0]).astype(np.float64), rtol=1e-6)
    assert np.allclose(rec["coef"][[0, 4, 5]], _ycocg(np.float32(rgb[0]).astype(np.float64)), rtol=1e-6)


def test_fixed_point_sums_brute_force(oracle_mod):
    """Every sum is, exactly, the cell's sum of each vertex's code round(x * 2^F), x taken in
    FP32 in the stated order; grouped here by brute force over vertex pairs."""
    rng = np.random.default_rng(4)
    n = 120
    cells = rng.integers(0, 3, n)
    pos = np.stack([(cells + 0.5) / 4.0, np.full(n, 0.3), np.full(n, 0.6)], axis=1)
    normals = _unit(rng, n, 0.7)
    rgb = rng.lognormal(0, 1, (n, 3)).astype(np.float32)
    w = rng.uniform(0.0, 2.0, n).astype(np.float32)
    v = stack([vertex(tuple(pos[i]), n=tuple(normals[i]), d=(0.3, -0.2, -1.0), w=float(w[i]), L=tuple(rgb[i]))
               for i in range(n)])
    o = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=0.01, use_normal=False)
    o.insert(v)
    rec = o.export()
    f32 = np.float32
    codes = np.zeros((n, 16), dtype=np.int64)
    for i in range(n):
        wi, nr = v[i, 3], v[i, 4:7]
        p = [f32(wi * v[i, 12 + c]) for c in range(3)]
        wY = f32(f32(f32(0.25) * p[0] + f32(0.5) * p[1]) + f32(0.25) * p[2])
        wCo = f32(f32(0.5) * p[0] - f32(0.5) * p[2])
        wCg = f32(f32(f32(0.5) * p[1] - f32(0.25) * p[0]) - f32(0.25) * p[2])
        m = [f32(wi * nr[k]) for k in range(3)]
        vals = [wY, wCo, wCg, wi, *m, *[f32(wY * nr[k]) for k in range(3)],
                f32(m[0] * nr[0]), f32(m[0] * nr[1]), f32(m[0] * nr[2]), f32(m[1] * nr[1]), f32(m[1] * nr[2]),
                f32(m[2] * nr[2])]
        codes[i] = [int(np.rint(float(x) * 2.0 ** F)) for x in vals]
    assert len(rec) == len(set(cells.tolist()))
    for r in rec:
        cell = int((r["key"] >> 32) & 0xFFFF) - 32768
        members = [i for i in range(n) if int(np.floor(pos[i, 0] * 4)) == cell]
        want = sum((codes[i] for i in members), np.zeros(16, dtype=np.int64))
        assert np.array_equal(r["sum"], want), (cell, r["sum"] - want)


def test_blend_follows_the_closed_form_per_coefficient(oracle_mod):
    """Equal per-iteration weight: alpha_k = max(k^-1/2, alpha_min); each coefficient follows
    L_k = (1 - alpha_k) L_{k-1} + alpha_k x_k with x_k the textbook fit of iteration k."""
    rng = np.random.default_rng(9)
    o = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=0.02, alpha_min=0.2, use_normal=False)
    L = np.zeros(6)
    for k in range(1, 9):
        n = 16
        v = _cell_vertices(rng, n, _unit(rng, n, 0.5), rng.lognormal(0, 1, (n, 3)), np.ones(n))
        o.insert(v)
        o.update()
        alpha = max(1.0 / math.sqrt(k), 0.2)
        L = (1 - alpha) * L + alpha * _textbook_fit(v, 0.02)
        got = o.export()[0]["coef"]
        assert np.all(np.abs(got - L) <= 1e-6 * (np.abs(L).sum())), (k, got, L)


def test_cv_reads_each_vertex_at_its_own_normal(oracle_mod):
    """out_j = L_j - beta t_j C(x_{j+1}, n_{j+1}) + beta C(x_j, n_j), with C the cell fit at the
    named vertex's normal, rebuilt here from the exported coefficients."""
    rng = np.random.default_rng(12)
    n = 60
    cells = rng.integers(0, 2, n)
    normals = _unit(rng, n, 0.7)
    recs = [vertex(((cells[i] + 0.5) / 4, 0.3, 0.3), n=tuple(normals[i]), d=(0.2, 0.1, -1.0), w=1.0,
                   L=tuple(rng.lognormal(0, 1, 3))) for i in range(n)]
    o = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=0.01, beta=0.75, use_normal=False)
    o.insert(stack(recs))
    o.update()
    coef = {int((r["key"] >> 32) & 0xFFFF) - 32768: r["coef"] for r in o.export()}
    P, D = 20, 3
    q_norm = _unit(rng, P * D, 0.9)
    q_cell = rng.integers(0, 3, P * D)  # cell 2 is absent
    v = stack([vertex(((q_cell[i] + 0.5) / 4, 0.3, 0.3), n=tuple(q_norm[i]), d=(0.2, 0.1, -1.0),
                      L=tuple(rng.lognormal(0, 1, 3)), t=tuple(rng.uniform(0.1, 0.9, 3))) for i in range(P * D)])

    def C(i):
        c = coef.get(int(q_cell[i]))
        if c is None:
            return np.zeros(3)
        Y = c[0] + c[1:4] @ v[i, 4:7].astype(np.float64)
        return np.array([Y + c[4] - c[5], Y + c[5], Y - c[4] - c[5]])

    out = o.query_cv(v, P, D)
    for j in range(D):
        for p in range(P):
            i = j * P + p
            L = v[i, 12:15].astype(np.float64)
            t = v[i, [7, 11, 15]].astype(np.float64)
            want = L - 0.75 * t * C(i + P) + 0.75 * C(i) if j + 1 < D else L
            assert np.allclose(out[i], want, rtol=1e-12, atol=1e-12), (j, p)
    assert np.allclose(o.lookup(v), np.stack([C(i) for i in range(P * D)]), rtol=1e-12, atol=1e-12)


def test_range_rule_on_the_normal_and_counters(oracle_mod):
    recs = [vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, 1.0)), vertex((0.3, 0.3, 0.3), n=(0.0, 1.0009765625, 0.0)),
            vertex((0.3, 0.3, 0.3), n=(0.0, 0.0, -1.001)), vertex((0.3, 0.3, 0.3), w=2.0 ** -30),
            vertex((0.3, 0.3, 0.3), L=(1.0, np.nan, 1.0))]
    o = oracle_mod.ShOracle(pos_bits=2, dir_bits=1, ridge=0.01, use_normal=False)
    st = o.insert(stack(recs))
    assert st == oracle_mod.STATUS_RANGE
    assert o.counters() == (2, 1)
    assert o.export()[0]["sum"][3] == 2 << F  # the two accepted vertices
