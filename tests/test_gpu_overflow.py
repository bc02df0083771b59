"""Per-edge count overflow: uint32 rows saturate, int64 totals stay exact.

A per-edge count above 2^32 - 1 is written as 2^32 - 1 and raises
TG_ERR_OVERFLOW, while the global totals come from the 64-bit per-edge
values and stay exact (the counts are integers with no upper bound in the
paper's Problem 1; the uint32 row width is the reading of its 4-byte count
storage in the space analysis of Sec. 7).

The graph is a star K_{1,n} with every node of one type (L = 1).  Every
edge (centre, leaf) has |S_centre| = n - 1 and |S_leaf| = 0, so by Lemma 2
its 4-star orbit g5 is C(n - 1, 2), its 3-path slot n - 1 and every other
slot 0; globally there are n edges, C(n, 2) 3-paths and C(n, 3) 4-stars.
With n = 92,700, C(92,699, 2) = 4,296,505,951 > 2^32 - 1 on every edge.
"""
from math import comb

import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_count
from oracle_pins import graph_from_edges

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def star(n_leaves: int):
    return graph_from_edges(n_leaves + 1, [(0, x) for x in range(1, n_leaves + 1)], [0] * (n_leaves + 1), 1)


def star_expected(n_leaves: int):
    """Closed-form rows (int64, not saturated) and totals of a one-type star."""
    lay = tg.tg_layout(1, 4)
    row = np.zeros(lay["per_edge_slots"], dtype=np.int64)
    row[lay["orbit_offset"][1]] = n_leaves - 1                  # 3-path (g1): S_centre
    row[lay["orbit_offset"][5]] = comb(n_leaves - 1, 2)         # 4-star (g5), Lemma 2
    gl = np.zeros(lay["global_slots"], dtype=np.int64)
    off = lay["global_block_offset"]
    gl[off[0]] = n_leaves
    gl[off[1]] = comb(n_leaves, 2)
    gl[off[4]] = comb(n_leaves, 3)
    return np.tile(row, (n_leaves, 1)), gl


def test_star_closed_form_matches_oracle():
    # the closed form used below is the oracle's answer on a smaller star
    g = star(300)
    pe_o, gl_o = oracle.paper(g)
    pe_c, gl_c = star_expected(300)
    np.testing.assert_array_equal(pe_o, pe_c)
    np.testing.assert_array_equal(gl_o, gl_c)
    pe, gl, st = gpu_count(g)
    assert st == 0
    np.testing.assert_array_equal(pe, pe_o)
    np.testing.assert_array_equal(gl, gl_o)


def test_per_edge_overflow_saturates_and_totals_stay_exact():
    n = 92_700
    assert comb(n - 1, 2) > 2**32 - 1
    pe, gl, st = gpu_count(star(n))
    assert tg.STATUS[st] == "TG_ERR_OVERFLOW"
    pe_c, gl_c = star_expected(n)
    g5 = tg.tg_layout(1, 4)["orbit_offset"][5]
    assert (pe[:, g5] == 2**32 - 1).all()                       # every g5 slot saturated
    pe_c[:, g5] = 2**32 - 1
    np.testing.assert_array_equal(pe, pe_c)                     # every other slot exact
    np.testing.assert_array_equal(gl, gl_c)                     # int64 totals from 64-bit values
    assert gl[tg.tg_layout(1, 4)["global_block_offset"][4]] == comb(n, 3)


def test_no_overflow_at_the_limit():
    # the largest star without overflow: C(92,682, 2) = 4,294,930,221 fits
    # in 32 bits (C(92,683, 2) would not): no saturation, status OK
    n = 92_683
    assert comb(n - 1, 2) <= 2**32 - 1
    pe, gl, st = gpu_count(star(n))
    assert st == 0
    pe_c, gl_c = star_expected(n)
    np.testing.assert_array_equal(pe, pe_c)
    np.testing.assert_array_equal(gl, gl_c)
