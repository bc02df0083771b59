"""The oracle's position-aware typed graphlet counts (Sec. 5, Def. 8) pinned
to what the definition and the mathematics fix.

* Class counts: Burnside's lemma over each shape's automorphism group, and
  the figure of Sec. 5 (eight labellings of the 3-path; F3, F4, F5 map to
  one typed graphlet).
* Merging: summing position-aware counts over the positions of each type
  multiset gives the typed counts of Alg. 1-3 + Lemmas (another route), per
  edge and globally; the Property of Sec. 5 (P_H >= T_H).
* Sec. 6 per class: every instance is counted once on each of its |E(H)|
  edges (per-edge slots mapped to classes here, in the test's own code).
* Closed forms of typed paths, stars, cycles, the tailed triangle and the
  chordal cycle; the per-edge route against brute force over all node sets.

Layout (shared by specification with the GPU library): numbered shapes
0 edge 0-1; 1 3-path, 0 the centre; 2 triangle; 3 4-path 0-1-2-3; 4 4-star,
0 the centre; 5 4-cycle 0-1-2-3-0; 6 tailed triangle, 0 the degree-3 node,
1 the tail; 7 chordal cycle, 0-1 the chord; 8 4-clique.  A class is ranked
by its lexicographically smallest labelling.  Per-edge blocks O1..O12 as
documented in oracle.c, sides 0 = lo, 1 = hi (lo < hi, caller ids).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle_pins import (BLOCK_EDGES, automorphisms, burnside, canonical_classes, edge_list, global_slot_pa,
                         graph_from_edges, merge_pa_global, merge_per_edge, multisets, pa_offsets, pa_sizes, pairs,
                         random_graph, read_golden, slot_instance)

# ------------------------------------------------------------------ classes

@pytest.mark.parametrize("L", range(1, 9))
def test_class_counts_follow_burnside(L):
    assert oracle.pa_block_sizes(L) == burnside(L)
    assert oracle.pa_per_edge_slots(L) == sum(pa_sizes(L))


@pytest.mark.parametrize("L", [2, 3])
def test_class_ranks_match_enumeration(L):
    for b in range(9):
        for lab, rank in canonical_classes(L, b).items():
            assert oracle.pa_class(L, b, lab) == rank


def test_figure_of_sec5():
    """Eight labellings (L^K = 2^3) of the 3-path; Def. 8 identifies the two
    that are mirror images (F3 ~ F4, F6 ~ F7), leaving six classes; the
    classes of F3, F4 and F5 all merge into the typed graphlet {1, 1, 2}."""
    rows = read_golden("position_aware_3path_figure.txt")
    assert len(rows) == 2 ** 3
    cls = {}
    for name, top, mid, bot in rows:
        lab = (int(mid) - 1, int(top) - 1, int(bot) - 1)          # numbered: centre first
        cls[name] = oracle.pa_class(2, 1, lab)
    assert len(set(cls.values())) == 6
    assert cls["F3"] == cls["F4"] and cls["F6"] == cls["F7"] and cls["F3"] != cls["F5"]
    ms = {name: tuple(sorted(int(v) for v in row)) for name, *row in rows}
    assert ms["F3"] == ms["F4"] == ms["F5"] == (1, 1, 2)


# ------------------------------------------------------------- merging pins

@pytest.mark.parametrize("seed", range(8))
def test_per_edge_merges_to_typed_counts(seed):
    g = random_graph(10 + seed, 0.45, [1, 2, 3, 4][seed % 4], 6100 + seed)
    pe_pa, gl_pa = oracle.position_aware(g)
    pe, gl = oracle.paper(g)
    np.testing.assert_array_equal(merge_per_edge(g["L"], pe_pa), pe)


@pytest.mark.parametrize("seed", range(8))
def test_global_merges_to_typed_counts_and_brute_force(seed):
    """Per class -> its type multiset gives the typed totals; the per-edge
    route equals brute force over all node sets; P_H >= T_H (Sec. 5)."""
    L = [2, 3, 4, 3][seed % 4]
    g = random_graph(11 + seed, 0.4, L, 6200 + seed)
    _, gl_pa = oracle.position_aware(g)
    np.testing.assert_array_equal(gl_pa, oracle.position_aware_brute(g))
    _, gl = oracle.paper(g)
    merged = merge_pa_global(L, gl_pa)
    sizes = burnside(L)
    typed_sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    s = t = 0
    for b in range(9):
        assert np.count_nonzero(gl_pa[s:s + sizes[b]]) >= np.count_nonzero(gl[t:t + typed_sizes[b]])
        s += sizes[b]
        t += typed_sizes[b]
    np.testing.assert_array_equal(merged, gl)


@pytest.mark.parametrize("seed", range(6))
def test_per_edge_sums_are_edges_times_global(seed):
    """Sec. 6 per position-aware class: mapping every per-edge slot to the
    class of its instance and summing over edges gives |E(H)| x the global
    count (the edge itself for block 0)."""
    L = [2, 3, 3][seed % 3]
    g = random_graph(12 + seed, 0.45, L, 6300 + seed)
    pe_pa, gl_pa = oracle.position_aware(g)
    ty = g["types"]
    sizes = burnside(L)
    off_b = np.concatenate([[0], np.cumsum(sizes)])
    raw = np.zeros_like(gl_pa)
    classes = {}
    for e, (lo, hi) in enumerate(edge_list(g)):
        raw[global_slot_pa(L, 0, (ty[lo], ty[hi]), classes)] += 1
        for slot in np.nonzero(pe_pa[e])[0]:
            b, lab = slot_instance(L, int(slot), int(ty[lo]), int(ty[hi]))
            raw[global_slot_pa(L, b, lab, classes)] += pe_pa[e, slot]
    for b in range(9):
        np.testing.assert_array_equal(raw[off_b[b]:off_b[b + 1]], BLOCK_EDGES[b] * gl_pa[off_b[b]:off_b[b + 1]])


# ------------------------------------------------------------- closed forms

def _row_for(L, entries):
    row = np.zeros(sum(pa_sizes(L)), np.int64)
    off = pa_offsets(L)
    for (o, idx), v in entries.items():
        row[off[o - 1] + idx] += v
    return row


@pytest.mark.parametrize("types,L", [([0, 1, 2, 1, 0, 2, 2], 3), ([1, 0, 0, 1, 1], 2), ([0] * 6, 1)])
def test_typed_path(types, L):
    """Path v0 - v1 - ... : edge (k, k+1) has lo = k.  Its 3-paths are
    centred at lo (third node v_{k-1}) and at hi (v_{k+2}); it ends the
    4-paths v_{k-2}..v_{k+1} (inner lo) and v_k..v_{k+3} (inner hi) and is
    the centre of v_{k-1}..v_{k+2}.  Globally every window of four nodes
    is one 4-path, its class fixed by the window or its reverse."""
    n = len(types)
    g = graph_from_edges(n, [(k, k + 1) for k in range(n - 1)], types, L)
    pe, gl = oracle.position_aware(g)
    LL = L * L
    for k in range(n - 1):
        ent = {}
        t = lambda x: types[x]                                 # noqa: E731
        if k >= 1:
            ent[(1, t(k - 1))] = 1
        if k + 2 < n:
            ent[(1, L + t(k + 2))] = 1
        if k >= 2:
            ent[(3, t(k - 1) * L + t(k - 2))] = 1
        if k + 3 < n:
            ent[(3, LL + t(k + 2) * L + t(k + 3))] = 1
        if k >= 1 and k + 2 < n:
            ent[(4, t(k - 1) * L + t(k + 2))] = 1
        np.testing.assert_array_equal(pe[k], _row_for(L, ent))
    sizes = burnside(L)
    reps = sorted({min(w, w[::-1]) for w in itertools.product(range(L), repeat=4)})
    want = np.zeros(sizes[3], np.int64)
    for k in range(n - 3):
        w = tuple(types[k:k + 4])
        want[reps.index(min(w, w[::-1]))] += 1
    s3 = sum(sizes[:3])
    np.testing.assert_array_equal(gl[s3:s3 + sizes[3]], want)


def test_typed_star():
    """Star with centre 0: every edge has lo = the centre; its 3-paths are
    centred at lo, its 4-stars too; globally (centre type, leaf multiset)."""
    L, leaves = 3, [0, 2, 2, 1, 0]
    types = [1] + leaves
    n = len(types)
    g = graph_from_edges(n, [(0, a) for a in range(1, n)], types, L)
    pe, gl = oracle.position_aware(g)
    pr = pairs(L)
    for e, (c, a) in enumerate(edge_list(g)):
        rest = [x for x in range(1, n) if x != a]
        ent = {}
        for b in rest:
            ent[(1, types[b])] = ent.get((1, types[b]), 0) + 1
        for b, b2 in itertools.combinations(rest, 2):
            key = (5, pr.index(tuple(sorted((types[b], types[b2])))))
            ent[key] = ent.get(key, 0) + 1
        np.testing.assert_array_equal(pe[e], _row_for(L, ent))
    sizes = burnside(L)
    s4 = sum(sizes[:4])
    reps = sorted((c,) + ms for c in range(L) for ms in itertools.combinations_with_replacement(range(L), 3))
    want = np.zeros(sizes[4], np.int64)
    for trio in itertools.combinations(leaves, 3):
        want[reps.index((1,) + tuple(sorted(trio)))] += 1
    np.testing.assert_array_equal(gl[s4:s4 + sizes[4]], want)


@pytest.mark.parametrize("types", [(0, 1, 2, 1), (2, 0, 0, 1), (1, 1, 0, 0)])
def test_typed_four_cycle(types):
    """C4 0-1-2-3-0: edge (lo, hi) is a 4-cycle edge keyed by (type of lo's
    other neighbour, type of hi's); 3-paths centred at each endpoint; one
    4-cycle, its class the smallest rotation or reflection."""
    L = 3
    g = graph_from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 3)], list(types), L)
    pe, gl = oracle.position_aware(g)
    nb = {0: (1, 3), 1: (0, 2), 2: (1, 3), 3: (0, 2)}
    for e, (lo, hi) in enumerate(edge_list(g)):
        x = [v for v in nb[lo] if v != hi][0]
        y = [v for v in nb[hi] if v != lo][0]
        ent = {(6, types[x] * L + types[y]): 1, (1, types[x]): 1, (1, L + types[y]): 1}
        np.testing.assert_array_equal(pe[e], _row_for(L, ent))
    sizes = burnside(L)
    s5 = sum(sizes[:5])
    D4 = [(0, 1, 2, 3), (1, 2, 3, 0), (2, 3, 0, 1), (3, 0, 1, 2), (3, 2, 1, 0), (0, 3, 2, 1), (1, 0, 3, 2),
          (2, 1, 0, 3)]
    reps = sorted({min(tuple(w[p] for p in d) for d in D4) for w in itertools.product(range(L), repeat=4)})
    assert len(reps) == sizes[5]
    want = np.zeros(sizes[5], np.int64)
    want[reps.index(min(tuple(types[p] for p in d) for d in D4))] = 1
    np.testing.assert_array_equal(gl[s5:s5 + sizes[5]], want)


def test_tailed_triangle_and_chordal_cycle_written_out():
    """Tailed triangle: triangle 0-1-2, tail 3 on node 2 (types 0, 1, 2, 1);
    chordal cycle: chord 1-2, nodes 0 and 3 on both (types 2, 0, 1, 0).
    Keys (block, index) of each edge's nonzero slots, worked out by hand."""
    L, LL = 3, 9
    pr = pairs(L)
    g = graph_from_edges(4, [(0, 1), (0, 2), (1, 2), (2, 3)], [0, 1, 2, 1], L)
    pe, _ = oracle.position_aware(g)
    want = {
        (0, 1): {(2, 2): 1, (8, 2 * L + 1): 1},                   # opposite node 2: (its type, tail's type)
        (0, 2): {(2, 1): 1, (1, L + 1): 1, (9, LL + 1 * L + 1): 1},  # degree-3 node is hi; third node 1, tail 3
        (1, 2): {(2, 0): 1, (1, L + 1): 1, (9, LL + 0 * L + 1): 1},  # third node 0, tail 3
        (2, 3): {(1, 0): 1, (1, 1): 1, (7, pr.index((0, 1))): 1},    # tail edge, degree-3 node is lo
    }
    for e, (lo, hi) in enumerate(edge_list(g)):
        np.testing.assert_array_equal(pe[e], _row_for(L, want[(lo, hi)]), err_msg=str((lo, hi)))
    g = graph_from_edges(4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)], [2, 0, 1, 0], L)
    pe, _ = oracle.position_aware(g)
    want = {
        (0, 1): {(2, 1): 1, (1, L + 0): 1, (10, LL + 1 * L + 0): 1},  # degree-3 hi; other degree-3 node 2, node 3
        (0, 2): {(2, 0): 1, (1, L + 0): 1, (10, LL + 0 * L + 0): 1},  # degree-3 hi; node 1, node 3
        (1, 2): {(2, 2): 1, (2, 0): 1, (11, pr.index((0, 2))): 1},    # the chord: nodes 0 and 3
        (1, 3): {(2, 1): 1, (1, 2): 1, (10, 1 * L + 2): 1},           # degree-3 lo; node 2, node 0
        (2, 3): {(2, 0): 1, (1, 2): 1, (10, 0 * L + 2): 1},           # degree-3 lo; node 1, node 0
    }
    for e, (lo, hi) in enumerate(edge_list(g)):
        np.testing.assert_array_equal(pe[e], _row_for(L, want[(lo, hi)]), err_msg=str((lo, hi)))


def test_empty_graph_and_bad_types():
    pe, gl = oracle.position_aware(graph_from_edges(4, [], [0, 1, 0, 1], 2))
    assert pe.shape == (0, oracle.pa_per_edge_slots(2)) and not gl.any()
    with pytest.raises(oracle.OracleError):
        oracle.position_aware(graph_from_edges(2, [(0, 1)], [0, 0], 9))
