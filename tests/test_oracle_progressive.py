"""Pins for the oracle's progressive update values (Section "Progressive solver", eq. (9);
Alg. 1 for L~_o, Alg. 2 for L~_{o\\e}).

Paths form a fixed chain of cells A -> B -> C where only the last cell emits E.  The
progressive solver transports one more bounce per iteration (a Jacobi iteration), so each
cell sees a piecewise-constant input sequence whose blended value has the closed form of
the blend recursion (eq. 10-11) with alpha_k = max(k^-1/2, alpha_min)."""

import numpy as np
import pytest

from helpers import vertex

T = 0.5
E = 3.0
CELLS = [(0.1, 0.1, 0.1), (0.5, 0.5, 0.5), (0.9, 0.9, 0.9)]


def _closed_form(xs, alpha_min):
    """L_k = sum_i alpha_i x_i prod_{m>i} (1 - alpha_m)."""
    alphas = [max((k + 1) ** -0.5, alpha_min) for k in range(len(xs))]
    out = 0.0
    for i, x in enumerate(xs):
        prod = 1.0
        for m in range(i + 1, len(xs)):
            prod *= 1.0 - alphas[m]
        out += alphas[i] * x * prod
    return out


def _chain(P, depth):
    """P identical paths visiting CELLS[3-depth:] in order; only the last vertex emits."""
    cells = CELLS[3 - depth:]
    v = np.empty((depth * P, 16), dtype=np.float32)
    for j, c in enumerate(cells):
        Le = E if j == depth - 1 else 0.0
        for p in range(P):
            v[j * P + p] = vertex(c, L=(Le, 2 * Le, 0.5 * Le), t=(T, T, T))
    return v


def _cell_L(o, pos):
    key = [r for r in o.export() if r["key"] == __import__("oracle").vertex_key(o.cfg, vertex(pos))][0]
    return key["L"]


@pytest.mark.parametrize("alpha_min", [0.1, 0.0])
def test_alg1_transports_one_bounce_per_iteration(oracle_mod, alpha_min):
    P, D = 4, 3
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2, alpha_min=alpha_min)
    v = _chain(P, D)
    xs = {0: [], 1: [], 2: []}  # per cell: the sequence of this-iteration means
    for k in range(8):
        # what eq. (9) feeds each cell at iteration k (old approximants of the next cell)
        L_old = {j: (_cell_L(o, CELLS[j]) if k > 0 else np.zeros(3)) for j in range(3)}
        # each input enters through 24-bit fixed point (all vertices of a cell agree, so the
        # cell mean is exactly the quantised value)
        def q(x):
            return float(np.rint(x * 2.0 ** 24) / 2.0 ** 24)

        xs[2].append(q(E))
        xs[1].append(q(T * L_old[2][0]))
        xs[0].append(q(T * L_old[1][0]))
        o.insert_progressive(v, P, D, field=0)
        o.update()
        for j in range(3):
            np.testing.assert_allclose(_cell_L(o, CELLS[j])[0], _closed_form(xs[j], alpha_min), rtol=1e-12)
        np.testing.assert_allclose(_cell_L(o, CELLS[2]), [E, 2 * E, 0.5 * E], rtol=1e-15)
    # C holds E from the first iteration, so B's input is T E from the second one; A's input
    # lags one more iteration and rises towards T^2 E as B's approximant converges
    assert xs[1][0] == 0.0 and xs[1][1:] == [T * E] * 7
    assert xs[0][:2] == [0.0, 0.0] and all(0.0 < a < b <= T * T * E for a, b in zip(xs[0][2:], xs[0][3:]))


def test_alg2_excludes_emission_and_shifts_by_one_vertex(oracle_mod):
    """L~_{o\\e}: the emitter's own cell holds 0 (it has no successor and emission is
    excluded); the cell before it receives t * (L_e + 0) = T E from the first iteration."""
    P, D = 3, 3
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2, alpha_min=0.1)
    v = _chain(P, D)
    for k in range(6):
        o.insert_progressive(v, P, D, field=1)
        o.update()
        np.testing.assert_allclose(_cell_L(o, CELLS[2]), 0.0, atol=0)
        np.testing.assert_allclose(_cell_L(o, CELLS[1]), [T * E, 2 * T * E, 0.5 * T * E], rtol=1e-15)
    # A receives t * (L_e(B) + L~_{o\\e}(B)) = T * (0 + T E) from the second iteration on
    np.testing.assert_allclose(_cell_L(o, CELLS[0])[0], _closed_form([0.0] + [T * T * E] * 5, 0.1), rtol=1e-12)


def test_progressive_counters_match_plain_insert(oracle_mod):
    """Only the values change: cells and counters are those of a plain insert."""
    from synth.scene import iteration_vertices, workload

    w = workload("64x64_d3")
    v = iteration_vertices(w, 0)
    P, D = w["width"] * w["height"], w["depth"]
    a = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    b = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    a.insert(v)
    b.insert_progressive(v, P, D, field=0)
    ra, rb = a.export(), b.export()
    assert np.array_equal(ra["key"], rb["key"]) and np.array_equal(ra["c_new"], rb["c_new"])
    # with an empty table the Alg. 1 value of every vertex is its own L_e
    np.testing.assert_allclose(rb["sum"], ra["sum"], rtol=0, atol=1)


def test_progressive_weight_range_edges(oracle_mod):
    """The progressive insert applies the range rule to the vertex's own record: w = 2^15 with an
    emission of 1 is accepted, w just above 2^15 is dropped (a one-vertex path: the Alg. 1 value
    is the vertex's own emission)."""
    for w, accepted in ((32768.0, True), (32768.0078125, False), (0.0, True)):
        o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
        v = vertex((0.3, 0.3, 0.3), w=w, L=(1.0, 1.0, 1.0))[None, :]
        status = o.insert_progressive(v, 1, 1, field=0)
        dropped, zero_w = o.counters()
        if accepted and w > 0:
            assert status == 0 and len(o) == 1 and int(o.export()[0]["c_new"]) == int(w * 2 ** 24)
        elif accepted:
            assert status == 0 and zero_w == 1 and len(o) == 0
        else:
            assert status != 0 and dropped == 1 and len(o) == 0


def _two_cell_path(oracle_mod, C_next, Le0, t0, w0=1.0, Le1=0.0):
    """An oracle whose cell B holds the approximant C_next, and one path A -> B."""
    o = oracle_mod.Oracle(pos_bits=4, dir_bits=2)
    o.insert(vertex(CELLS[1], L=(C_next, C_next, C_next))[None, :])
    o.update()
    v = np.stack([vertex(CELLS[0], w=w0, L=(Le0, Le0, Le0), t=(t0, t0, t0)),
                  vertex(CELLS[1], L=(Le1, Le1, Le1))]).astype(np.float32)
    return o, v


def _cell_A(o):
    return [r for r in o.export() if r["key"] == __import__("oracle").vertex_key(o.cfg, vertex(CELLS[0]))]


@pytest.mark.parametrize("field", [0, 1])
@pytest.mark.parametrize("t0", [1.0, 2.0, 1e30])
def test_progressive_value_saturates_at_the_bound(oracle_mod, field, t0):
    """A progressive value past |w * value| = 2^15 is saturated there, not dropped: with
    C(B) = 32767 and L_e = 1 (field 0) the value 1 + t * 32767 is 32768 at t = 1 (exactly the
    bound) and beyond it for larger t; field 1's t * (0 + 32767) likewise.  The vertex keeps
    its weight in c_new and nothing is counted as dropped."""
    o, v = _two_cell_path(oracle_mod, 32767.0, 1.0 if field == 0 else 0.0, t0)
    st = o.insert_progressive(v, 1, 2, field=field)
    assert st == 0 and o.counters() == (0, 0)
    a = _cell_A(o)[0]
    want = min(32768.0, (1.0 if field == 0 else 0.0) + t0 * 32767.0)
    assert int(a["sum"][0]) == int(round(want * 2 ** 24)) and int(a["c_new"]) == 1 << 24


def test_progressive_drops_by_the_record_not_by_the_value(oracle_mod):
    """A record that fails the plain range rule is dropped even if its progressive value is
    small (field 1 does not contain the vertex's own emission); a NaN throughput drops too."""
    o, v = _two_cell_path(oracle_mod, 1.0, 40000.0, 0.5)
    assert o.insert_progressive(v, 1, 2, field=1) == oracle_mod.STATUS_RANGE
    assert o.counters()[0] == 1 and not _cell_A(o)
    o, v = _two_cell_path(oracle_mod, 1.0, 1.0, float("nan"))
    assert o.insert_progressive(v, 1, 2, field=0) == oracle_mod.STATUS_RANGE
    assert o.counters()[0] == 1 and not _cell_A(o)
