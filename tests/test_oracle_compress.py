"""Pins for the oracle's compression (Sec. 2.2, last paragraph: merging adjacent
visibilities that share a point of the oversampled grid).

Each pin is independent of the routine under test:
  - run boundaries against exact rational rounding of the positions (Fraction);
  - the weighted sums against a plain Python loop in the same order;
  - the defining property: gridding the merged records with unit weights gives
    the grid of the original weighted records (through oracle.grid, pinned in
    test_oracle.py), to FP64 rounding;
  - degridding the merged records and expanding by run_of gives the original
    records' degridded values exactly (same cell, same table row);
  - hand-built special cases: stationary track, alternation, equal cell with a
    different table row, non-finite coordinates, empty input.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1605_07023_gb300 import synth


def exact_fine(u: float, O: int):
    """floor(u*O + 1/2) in exact rational arithmetic, or None for a non-finite u."""
    if not math.isfinite(u):
        return None
    return math.floor(Fraction(u) * O + Fraction(1, 2))


def expected_runs(uv, O):
    keys = []
    for u, v in uv:
        fu, fv = exact_fine(u, O), exact_fine(v, O)
        keys.append(None if fu is None or fv is None else (fu, fv))
    run_of, m = [], 0
    for k, key in enumerate(keys):
        if k == 0 or key is None or keys[k - 1] is None or key != keys[k - 1]:
            m += 1
        run_of.append(m - 1)
    return np.array(run_of, np.int64), m


def walk(n, O, rng):
    """A track whose steps are often zero or below half a fine step, with some positions on rounding ties."""
    uv = np.empty((n, 2))
    x = np.array([10.0, -7.0])
    for k in range(n):
        c = rng.integers(0, 5)
        if c == 0:
            pass                                                     # stationary
        elif c == 1:
            x = x + rng.uniform(-0.2, 0.2, 2) / O                    # usually the same fine position
        elif c == 2:
            x = np.round(x * O) / O + 0.5 / O                        # exactly on a tie: rounds up
        elif c == 3:
            x = x + rng.uniform(-3, 3, 2) / O                        # a few fine steps away
        else:
            x = x + rng.uniform(-0.6, 0.6, 2) / O
        uv[k] = x
    return uv


@pytest.mark.parametrize("O", [1, 8, 16])
def test_runs_and_sums_match_exact_definition(O):
    rng = np.random.default_rng(O)
    n, P = 400, 2
    uv = walk(n, O, rng)
    vis = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    w = rng.uniform(0.1, 2.0, n)
    uv_c, vis_c, run_of = oracle.compress(O, uv, vis, w)
    want_run_of, m = expected_runs(uv, O)
    assert 1 < m < n
    assert np.array_equal(run_of, want_run_of)
    assert uv_c.shape == (m, 2) and vis_c.shape == (m, P)
    # merged record = first member's uv; value = sum of w*V in input order (plain FP64 loop)
    for r in range(m):
        members = np.flatnonzero(want_run_of == r)
        assert np.array_equal(uv_c[r], uv[members[0]])
        for p in range(P):
            re = im = 0.0
            for k in members:
                re += w[k] * vis[k, p].real
                im += w[k] * vis[k, p].imag
            assert vis_c[r, p].real == re and vis_c[r, p].imag == im


def test_compressed_grid_equals_original_grid():
    w = synth.scaled_down(synth.cored_quad_pol(), 60_000)  # core-core baselines come first: many merges
    rng = np.random.default_rng(5)
    weights = rng.uniform(0.2, 2.0, w.n_vis)
    table = oracle.kb_table(w.S, w.oversample, w.beta)
    uv_c, vis_c, run_of = oracle.compress(w.oversample, w.uv, w.vis, weights)
    assert len(uv_c) < 0.6 * w.n_vis
    g0, s0 = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, weights, table)
    g1, s1 = oracle.grid(w.G, w.S, w.oversample, uv_c, vis_c, None, table)
    assert s0 == s1 == 0
    for p in range(w.npol):
        assert np.linalg.norm(g1[p] - g0[p]) <= 1e-12 * np.linalg.norm(g0[p])
    # dropping the weights must break the identity (the pin sees the weights)
    uv_u, vis_u, _ = oracle.compress(w.oversample, w.uv, w.vis, None)
    g2, _ = oracle.grid(w.G, w.S, w.oversample, uv_u, vis_u, None, table)
    assert np.linalg.norm(g2[0] - g0[0]) > 1e-3 * np.linalg.norm(g0[0])


def test_degrid_of_merged_records_expands_exactly():
    w = synth.scaled_down(synth.cored_quad_pol(), 20_000)
    rng = np.random.default_rng(6)
    g = rng.standard_normal((w.npol, w.G, w.G)) + 1j * rng.standard_normal((w.npol, w.G, w.G))
    table = oracle.kb_table(w.S, w.oversample, w.beta)
    uv_c, _, run_of = oracle.compress(w.oversample, w.uv, w.vis, None)
    d0, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g, table)
    d1, _ = oracle.degrid(w.G, w.S, w.oversample, uv_c, g, table)
    assert np.array_equal(d1[run_of], d0)


def test_special_cases():
    O = 8
    v1 = np.ones((1, 1), complex)
    # stationary: one run, first uv kept
    uv = np.array([[3.0, 4.0]] * 5 + [[3.0 + 0.25 / O, 4.0 - 0.25 / O]])
    uv_c, vis_c, run_of = oracle.compress(O, uv, np.ones((6, 1)), None)
    assert len(uv_c) == 1 and np.array_equal(uv_c[0], uv[0]) and vis_c[0, 0] == 6 and list(run_of) == [0] * 6
    # alternating positions: nothing adjacent matches
    uv = np.array([[3.0, 4.0], [5.0, 4.0]] * 3)
    assert len(oracle.compress(O, uv, np.ones((6, 1)))[0]) == 6
    # same cell, different GCF row: not merged
    uv = np.array([[10.0, 0.0], [10.0 + 1.0 / O, 0.0]])
    assert oracle.indices(64, 7, O, uv)[0][0][0] == oracle.indices(64, 7, O, uv)[0][1][0]
    assert len(oracle.compress(O, uv, np.ones((2, 1)))[0]) == 2
    # non-finite coordinates: runs of their own, and the next record starts a new run
    uv = np.array([[1.0, 1.0], [np.nan, 1.0], [np.nan, 1.0], [1.0, 1.0], [1.0, np.inf], [1.0, 1.0], [1.0, 1.0]])
    _, _, run_of = oracle.compress(O, uv, np.ones((7, 1)))
    assert list(run_of) == [0, 1, 2, 3, 4, 5, 5]
    # empty
    uv_c, vis_c, run_of = oracle.compress(O, np.zeros((0, 2)), np.zeros((0, 1)))
    assert len(uv_c) == 0 and len(run_of) == 0
    del v1
