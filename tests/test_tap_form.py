"""The tap-product form each kernel uses, against the multiplication counts of Sec. 6.

The paper counts, for a B x B block and P polarizations, B^2 + B^2 P multiplications to form
G_ij V_p as written and B P + B^2 P to form it as G^u_i (G^v_j V_p). The fixture
tests/golden/sec6_multiplications.txt holds those counts worked out by hand. Each built square
kernel must report the smaller count, in the form that gives it (the product form on a tie, where
it needs no extra products to be kept). Rectangular kernels must report the fewest multiplications
over the three forms (product first, then the v and u factorings). Host only: no GPU is touched.
"""
import os

import pytest

from paper_1605_07023_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(1, 1), (2, 1), (1, 2), (2, 2), (4, 1), (1, 4), (4, 2), (2, 4), (3, 3), (4, 4), (8, 1), (1, 8), (8, 2), (2, 8)]


@pytest.fixture(scope="module")
def gb():
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    import paper_1605_07023_gb300 as gb
    return gb


def golden():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "sec6_multiplications.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    return rows


def test_fixture_is_complete():
    keys = {(b, p) for b, p, _, _ in golden()}
    assert keys == {(b, p) for b in (1, 2, 3, 4, 8) for p in (1, 4)} | {(1, 2), (2, 2), (4, 2)}


def test_square_kernels_match_sec6_counts(gb):
    checked = 0
    for B, P, as_written, factored in golden():
        if (B, B) not in SHAPES:
            with pytest.raises(gb.GridderError):
                gb.tap_form(B, B, P)
            continue
        form, mults = gb.tap_form(B, B, P)
        assert mults == min(as_written, factored), (B, P)
        assert (form == "product") == (as_written <= factored), (B, P, form)
        checked += 1
    assert checked == 11


@pytest.mark.parametrize("P", [1, 2, 4])
def test_rectangular_kernels_take_the_fewest_multiplications(gb, P):
    for Bu, Bv in SHAPES:
        form, mults = gb.tap_form(Bu, Bv, P)
        counts = {"product": Bu * Bv, "factor_v": Bv * P, "factor_u": Bu * P}
        assert mults == min(counts.values()) + Bu * Bv * P, (Bu, Bv, P)
        best = [f for f in ("product", "factor_v", "factor_u") if counts[f] == min(counts.values())][0]
        assert form == best, (Bu, Bv, P, form)


def test_invalid_and_unsupported(gb):
    for args in [(0, 2, 1), (2, 0, 1), (2, 2, 3), (2, 2, 0)]:
        with pytest.raises(gb.GridderError):
            gb.tap_form(*args)
    with pytest.raises(gb.GridderError):
        gb.tap_form(8, 8, 4)
