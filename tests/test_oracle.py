"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Every check here could fail on a plausible mistake in the oracle:
  - exact rational arithmetic for the index rounding rule (a wrong tie or
    floor, or an FP64 rounding slip);
  - scipy's independent I0 for the Kaiser-Bessel table;
  - the table's mirror symmetry and its unit peak (a wrong sub-offset
    mapping);
  - a unit visibility reproducing the table's outer product at the right
    cells (Sec. 2.2; a transposed axis, wrong row or wrong half-width);
  - nearest-cell binning (np.add.at) as the S=1, O=1 special case;
  - linearity, weights, and P=4 as four P=1 problems (Sec. 4);
  - the adjoint identity for degridding;
  - imaging by FFT with grid correction matching a direct DFT (Sec. 2.2:
    convolution in uv is multiplication in the image). The KB transform pair
    used there is checked by quadrature first.
"""
from fractions import Fraction
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_1605_07023_gb300 import synth


def exact_fine(u: float, O: int) -> int:
    """floor(u*O + 1/2) in exact rational arithmetic."""
    return math.floor(Fraction(u) * O + Fraction(1, 2))


def exact_axis(u: float, G: int, S: int, O: int):
    """Independent restatement of the index rule in exact integers. Returns (C, row) or None."""
    if not math.isfinite(u):
        return None
    f = exact_fine(u, O)
    c = (f + O // 2) // O          # Python // is floor division
    s = f - c * O
    assert 0 <= s + O // 2 < O
    h = (S - 1) // 2
    C = c + G // 2
    if C - h < 0 or C - h + S > G:
        return None
    return C, s + O // 2


# ---------------------------------------------------------------- indices

def _edge_values(O: int, rng):
    vals = []
    for k in range(-40, 41):
        for frac in (0.0, 0.5, -0.5, 0.25):
            x = (k + frac) / O
            vals += [x, np.nextafter(x, np.inf), np.nextafter(x, -np.inf)]
    vals += list(rng.uniform(-50, 50, 300))
    vals += [0.0, -0.0, 1e-300, -1e-300, 0.5 / O - 2.0 ** -60, -0.5 / O + 2.0 ** -60,
             0.25 / O + 2.0 ** -56, -0.25 / O - 2.0 ** -56]
    return vals


@pytest.mark.parametrize("O", [1, 2, 8, 16, 64])
def test_fine_position_matches_exact_rationals(oracle_mod, O):
    rng = np.random.default_rng(O)
    for u in _edge_values(O, rng):
        assert oracle_mod.fine_position(u, O) == exact_fine(u, O), (u, O)


def test_fine_position_rejects_nonfinite(oracle_mod):
    for u in (np.inf, -np.inf, np.nan, 1e300):
        with pytest.raises(ValueError):
            oracle_mod.fine_position(u, 8)


@pytest.mark.parametrize("G,S,O", [(32, 7, 8), (64, 15, 16), (16, 1, 1), (20, 5, 4), (32, 8, 8)])
def test_indices_bruteforce(oracle_mod, G, S, O):
    rng = np.random.default_rng(G + S + O)
    us = np.array(_edge_values(O, rng))
    us = us[np.abs(us) < G]
    pairs = np.stack([us, rng.permutation(us)], axis=1)
    pairs = np.concatenate([pairs, [[np.nan, 0.0], [0.0, np.inf]]])
    cell, sub, skipped = oracle_mod.indices(G, S, O, pairs)
    n_bad = 0
    for k, (u, v) in enumerate(pairs):
        a, b = exact_axis(u, G, S, O), exact_axis(v, G, S, O)
        if a is None or b is None:
            n_bad += 1
            assert tuple(cell[k]) == (-1, -1) and tuple(sub[k]) == (-1, -1)
        else:
            assert tuple(cell[k]) == (a[0], b[0]) and tuple(sub[k]) == (a[1], b[1]), (u, v)
    assert skipped == n_bad


def test_indices_geometry(oracle_mod):
    """A visibility at u = k + s/O sits s/O of a cell right of cell centre k, so its table row is s + O/2."""
    G, S, O = 64, 7, 8
    for k in (-20, -1, 0, 3, 21):
        for s in range(-O // 2, O // 2):
            cell, sub, _ = oracle_mod.indices(G, S, O, np.array([[k + s / O, 0.0]]))
            assert cell[0, 0] == k + G // 2 and sub[0, 0] == s + O // 2
            assert cell[0, 1] == G // 2 and sub[0, 1] == O // 2


def test_edges_skipped_exactly_at_boundary(oracle_mod):
    G, S, O = 32, 7, 8
    h = 3
    lo = float(h - G // 2)            # C - h == 0: valid
    hi = float(G // 2 - h - 1)        # C - h + S == G: valid
    uv = np.array([[lo, 0], [lo - 1, 0], [hi, 0], [hi + 1, 0], [0, lo], [0, lo - 1], [0, hi], [0, hi + 1],
                   [lo - 0.5, 0], [lo - 0.5 - 1 / 16, 0], [lo - 0.5 - 1 / 8, 0]])
    cell, sub, skipped = oracle_mod.indices(G, S, O, uv)
    valid = cell[:, 0] >= 0
    # u = lo - 0.5 rounds up (ties toward +inf) to cell lo: still valid. So does lo - 0.5 - 1/16,
    # a tie on the 1/8 fine grid, which rounds up to fine position -4. An eighth lower is not.
    assert list(valid) == [True, False, True, False, True, False, True, False, True, True, False]
    assert skipped == 5


# ---------------------------------------------------------------- Kaiser-Bessel table

def test_bessel_i0_against_scipy(oracle_mod):
    for x in [0.0, 1e-8, 0.3, 1.0, 2.5, 7.3, 16.38, 35.1, 80.0, 140.0]:
        assert oracle_mod.bessel_i0(x) == pytest.approx(float(special.i0(x)), rel=2e-14, abs=0)


@pytest.mark.parametrize("S,O", [(7, 8), (15, 16), (9, 8), (8, 8)])
def test_kb_table_against_scipy(oracle_mod, S, O):
    beta = 2.34 * S
    t = oracle_mod.kb_table(S, O, beta)
    h = (S - 1) // 2
    for r in range(O):
        for i in range(S):
            d = (i - h) - (r - O / 2) / O
            x = 2 * d / S
            ref = special.i0(beta * np.sqrt(1 - x * x)) / special.i0(beta) if abs(x) <= 1 else 0.0
            assert t[r, i] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_kb_table_symmetry_and_peak(oracle_mod):
    S, O = 7, 8
    t = oracle_mod.kb_table(S, O, 2.34 * S)
    h = (S - 1) // 2
    assert t[O // 2, h] == 1.0                              # d = 0 at the centre row
    assert np.argmax(t[O // 2]) == h
    np.testing.assert_allclose(t[O // 2], t[O // 2][::-1], rtol=0, atol=0)
    for r in range(1, O):                                   # mirror: d(r, i) = -d(O-r, S-1-i)
        np.testing.assert_allclose(t[r], t[O - r][::-1], rtol=1e-15, atol=0)
    # Row r = 0 (s = -O/2) is the visibility half a cell left of centre:
    # its peak taps are at i = h-1 and h, equal.
    assert t[0, h] == pytest.approx(t[0, h - 1], rel=1e-15)
    assert np.all(t > 0) and np.all(t <= 1.0)


# ---------------------------------------------------------------- gridding definition pins

def test_single_visibility_footprint(oracle_mod):
    """Sec. 2.2: a unit delta convolved with the GCF, sampled on the grid."""
    G, S, O = 32, 5, 4
    rng = np.random.default_rng(1)
    table = rng.uniform(0.1, 1.0, (O, S))       # distinct values catch index mistakes
    h = (S - 1) // 2
    for (ku, su, kv, sv) in [(3, -2, -5, 1), (0, 0, 0, 0), (-7, 1, 9, -1), (10, -1, -10, -2)]:
        u, v = ku + su / O, kv + sv / O
        g, sk = oracle_mod.grid(G, S, O, [[u, v]], np.array([[1.0 + 0j]]), None, table)
        assert sk == 0
        expect = np.zeros((G, G), complex)
        Cu, Cv = ku + G // 2, kv + G // 2
        expect[Cv - h:Cv - h + S, Cu - h:Cu - h + S] = np.outer(table[sv + O // 2], table[su + O // 2])
        np.testing.assert_array_equal(g[0], expect)


def test_nearest_cell_binning_special_case(oracle_mod):
    """S = 1, O = 1 reduces gridding to nearest-cell binning, as np.add.at computes it."""
    G = 16
    rng = np.random.default_rng(2)
    n = 500
    uv = rng.uniform(-G / 2 + 0.5, G / 2 - 1.5, (n, 2))
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = rng.uniform(0.5, 2.0, n)
    table = np.array([[0.75]])
    g, sk = oracle_mod.grid(G, 1, 1, uv, vis[:, None], w, table)
    assert sk == 0
    ref = np.zeros((G, G), complex)
    cu = np.floor(uv[:, 0] + 0.5).astype(int) + G // 2
    cv = np.floor(uv[:, 1] + 0.5).astype(int) + G // 2
    np.add.at(ref, (cv, cu), 0.75 * 0.75 * w * vis)   # separable: tap_u * tap_v
    np.testing.assert_allclose(g[0], ref, rtol=1e-13, atol=1e-13)


def test_linearity_weights_and_polarizations(oracle_mod):
    w = synth.random_uniform(48, 7, 8, 4, 300, seed=3)
    table = oracle_mod.kb_table(7, 8, 2.34 * 7)
    rng = np.random.default_rng(4)
    v1 = w.vis.astype(complex)
    v2 = rng.standard_normal(v1.shape) + 1j * rng.standard_normal(v1.shape)
    wt = rng.uniform(0.1, 3.0, w.n_vis)
    a, b = 0.7 - 0.2j, -1.3
    g12, _ = oracle_mod.grid(48, 7, 8, w.uv, a * v1 + b * v2, None, table)
    g1, _ = oracle_mod.grid(48, 7, 8, w.uv, v1, None, table)
    g2, _ = oracle_mod.grid(48, 7, 8, w.uv, v2, None, table)
    np.testing.assert_allclose(g12, a * g1 + b * g2, rtol=1e-12, atol=1e-12)
    gw, _ = oracle_mod.grid(48, 7, 8, w.uv, v1, wt, table)
    gw2, _ = oracle_mod.grid(48, 7, 8, w.uv, v1 * wt[:, None], None, table)
    np.testing.assert_allclose(gw, gw2, rtol=1e-13, atol=1e-13)
    for p in range(4):
        gp, _ = oracle_mod.grid(48, 7, 8, w.uv, v1[:, p:p + 1], wt, table)
        np.testing.assert_array_equal(gp[0], gw[p])


def test_adjoint_identity(oracle_mod):
    """<grid(v), g> = <v, degrid(g)> with unit weights, to 1e-12 relative."""
    G, S, O, P = 40, 7, 8, 4
    w = synth.random_uniform(G, S, O, P, 400, seed=5)
    table = oracle_mod.kb_table(S, O, 2.34 * S)
    rng = np.random.default_rng(6)
    g = rng.standard_normal((P, G, G)) + 1j * rng.standard_normal((P, G, G))
    v = w.vis.astype(complex)
    gv, _ = oracle_mod.grid(G, S, O, w.uv, v, None, table)
    dg, _ = oracle_mod.degrid(G, S, O, w.uv, g, table)
    lhs = np.vdot(gv, g)
    rhs = np.vdot(v, dg)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_degrid_single_cell(oracle_mod):
    G, S, O = 32, 5, 4
    rng = np.random.default_rng(7)
    table = rng.uniform(0.1, 1.0, (O, S))
    g = np.zeros((1, G, G), complex)
    g[0, 20, 11] = 2.0 - 1.0j                    # row v = 20, column u = 11
    # a visibility at cell (u, v) = (12, 19) absolute with sub rows (1, 3):
    # taps i = 11 - 12 + 2 = 1 and j = 20 - 19 + 2 = 3
    u, v = 12 - G // 2 + (1 - O // 2) / O, 19 - G // 2 + (3 - O // 2) / O
    out, _ = oracle_mod.degrid(G, S, O, [[u, v]], g, table)
    assert out[0, 0] == pytest.approx((2.0 - 1.0j) * table[1, 1] * table[3, 3], rel=1e-15)


def test_skipped_visibilities_do_not_grid(oracle_mod):
    G, S, O = 32, 7, 8
    table = oracle_mod.kb_table(S, O, 2.34 * S)
    uv = np.array([[0.0, 0.0], [15.9, 0.0], [np.nan, 1.0], [-16.0, 0.0]])
    g, sk = oracle_mod.grid(G, S, O, uv, np.ones((4, 1)), None, table)
    g1, _ = oracle_mod.grid(G, S, O, uv[:1], np.ones((1, 1)), None, table)
    assert sk == 3
    np.testing.assert_array_equal(g, g1)
    d, skd = oracle_mod.degrid(G, S, O, uv, g, table)
    assert skd == 3 and np.all(d[1:] == 0)


# ---------------------------------------------------------------- imaging check (FFT + grid correction vs DFT)

def kb_transform(nu, S, beta):
    """Closed-form Fourier transform of I0(beta*sqrt(1-(2x/S)^2))/I0(beta) on |x| <= S/2."""
    nu = np.asarray(nu, dtype=np.float64)
    z2 = beta * beta - (np.pi * S * nu) ** 2
    z = np.sqrt(np.abs(z2))
    core = np.ones_like(z)
    pos = (z2 > 0) & (z > 0)
    neg = (z2 < 0)
    core[pos] = np.sinh(z[pos]) / z[pos]
    core[neg] = np.sin(z[neg]) / z[neg]
    return S * core / special.i0(beta)


def test_kb_transform_closed_form_by_quadrature():
    S, beta = 7, 2.34 * 7
    for nu in [0.0, 0.05, 0.11, 0.25, 0.5, 0.8, 1.3]:
        f = lambda x: special.i0(beta * np.sqrt(max(0.0, 1 - (2 * x / S) ** 2))) / special.i0(beta) * np.cos(2 * np.pi * nu * x)
        q, _ = integrate.quad(f, -S / 2, S / 2, limit=400, epsabs=1e-13, epsrel=1e-11)
        assert kb_transform(nu, S, beta) == pytest.approx(q, rel=1e-9, abs=1e-13)


def _image_error(oracle_mod, table, uv, vis, G, S, O, beta, mutate=None):
    g, sk = oracle_mod.grid(G, S, O, uv, vis[:, None], None, table)
    assert sk == 0
    g = g[0] if mutate is None else mutate(g[0])
    x = np.arange(G) - G // 2
    lidx = np.arange(-G // 4, G // 4)
    E = np.exp(2j * np.pi * np.outer(lidx, x) / G)             # [l, cell]
    img = E @ g @ E.T                                           # [m, l]: rows v<->m, columns u<->l
    c = kb_transform(lidx / G, S, beta)
    corrected = img / np.outer(c, c)
    # direct DFT: sum_n V_n exp(2 pi i (u_n l + v_n m) / G), indexed [m, l]
    direct = (np.exp(2j * np.pi * np.outer(lidx, uv[:, 1]) / G) * vis[None, :]) @ np.exp(2j * np.pi * np.outer(uv[:, 0], lidx) / G)
    return np.max(np.abs(corrected - direct))


def test_imaging_matches_direct_dft(oracle_mod):
    """FFT(grid) divided by the GCF transform equals the direct DFT in the inner half, within the aliasing bound."""
    G, S, O = 64, 7, 8
    beta = 2.34 * S
    table = oracle_mod.kb_table(S, O, beta)
    rng = np.random.default_rng(8)
    n = 6
    lim = (G // 2 - 4) * O
    uv = rng.integers(-lim, lim, size=(n, 2)) / O                   # exact fine positions
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    err = _image_error(oracle_mod, table, uv, vis, G, S, O, beta)
    # Aliasing bound (Poisson summation): per axis eps(nu) = sum_{k != 0} |C(nu+k)| / |C(nu)|,
    # plus the KB value at the support edge (one tap can fall just outside the footprint).
    lidx = np.arange(-G // 4, G // 4) / G
    ks = np.concatenate([np.arange(-60, 0), np.arange(1, 61)])
    c0 = np.abs(kb_transform(lidx, S, beta))
    eps = np.array([np.sum(np.abs(kb_transform(nu + ks, S, beta))) for nu in lidx]) / c0
    eps = eps + 2.0 / special.i0(beta) / c0
    e = eps.max()
    bound = ((1 + e) ** 2 - 1) * np.sum(np.abs(vis))
    assert bound < 0.05 * np.sum(np.abs(vis))
    assert err <= bound, (err, bound)
    # The check has teeth: mirrored table rows (a sign slip in the sub-offset) or transposed
    # coordinates break it by far more than the bound.
    assert _image_error(oracle_mod, table[::-1].copy(), uv, vis, G, S, O, beta) > 3 * bound
    assert _image_error(oracle_mod, table, uv, vis, G, S, O, beta, mutate=lambda g: g.T) > 3 * bound
