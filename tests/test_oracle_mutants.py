"""Planted mistakes in the oracle must fail the pins.

Each mutant is a copy of oracle.c compiled with -DORACLE_MUTANT=k, which
plants one plausible mistake: a dropped term in Lemma 1, a lost tie-break
in Alg. 2, j left inside S_i, transposed operands in Lemma 3, a wrong branch
in Alg. 3, an unsorted type multiset, a missing 1/2 in Lemma 2, a lost
exclusion of i and j in Alg. 2; in the weighted graph of Alg. 5, tailed
triangles booked as 4-cycles and D missing one endpoint of each edge; in
the position-aware counts of Sec. 5, the two sides of a 4-cycle key swapped
and the degree-3 side of a tailed triangle swapped; in the directed counts
of Sec. 4.8, the signs of S_j flipped and the edge's own orientation
dropped from the class key; in the edge-typed counts, a 3-path of S_j keyed
by the edge's own type and a triangle keyed without j's edge.  The pin battery here (closed forms,
layout enumeration, the brute-force and networkx-free subset count) must
reject every one of them, on the CPU.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle_pins import (BLOCK_EDGES, burnside, directed_pins, edge_typed_pins, expected_clique,
                         expected_complete_bipartite, expected_cycle, expected_star, global_slot_pa, graph_from_edges,
                         multisets, random_graph, slot_instance)

MUTANTS = {
    1: "Lemma 1 without the 4-cycle term",
    2: "Alg. 2 tailed-triangle tie-break dropped",
    3: "S_i keeps node j",
    4: "Lemma 3 with t and t' swapped",
    5: "Alg. 3 chordal-cycle edges booked as tailed-triangle centre",
    6: "type multiset not sorted before ranking",
    7: "Lemma 2 without the 1/2",
    8: "Alg. 2 scans i and j as neighbours of w_k",
    9: "Alg. 5 weights book a tailed triangle as a 4-cycle",
    10: "Alg. 5 degree adds each edge's weight to one endpoint only",
    11: "Sec. 5 4-cycle key (lo's neighbour, hi's neighbour) transposed",
    12: "Sec. 5 tailed-triangle edge at the degree-3 node booked on the other side",
    13: "Sec. 4.8 S_j counted with the opposite arc direction",
    14: "Sec. 4.8 class key without the edge's own orientation",
    15: "edge-typed 3-path of S_j keyed by the edge's own type",
    16: "edge-typed triangle keyed without j's edge to the third node",
}


def _battery(lib) -> list:
    """Names of the pins that fail for this oracle build."""
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except oracle.OracleError:
            failed.append(name + " (error)")

    for L in (3, 4):
        for K in (2, 3, 4):
            def ranks(L=L, K=K):
                return all(oracle.multiset_rank(L, ms[::-1], lib) == k for k, ms in enumerate(multisets(L, K)))
            check(f"rank L={L} K={K}", ranks)

    cases = []
    t = np.array([0, 0, 1, 2, 1, 0, 2])
    e, pe, gl = expected_clique(t, 3)
    cases.append(("clique", graph_from_edges(7, e, t, 3), pe, gl))
    ty, e, pe, gl = expected_star(1, [0, 1, 2, 0, 2, 2], 3)
    cases.append(("star", graph_from_edges(len(ty), e, ty, 3), pe, gl))
    ty, e, pe, gl = expected_complete_bipartite(3, 4)
    cases.append(("K34", graph_from_edges(7, e, ty, 2), pe, gl))
    t = [1, 0, 2, 3, 0, 1, 3, 2, 2]
    e, pe, gl = expected_cycle(t, 4)
    cases.append(("cycle", graph_from_edges(9, e, t, 4), pe, gl))
    for name, g, pe, gl in cases:
        def cf(g=g, pe=pe, gl=gl):
            a, b = oracle.paper(g, lib=lib)
            return np.array_equal(a, pe) and np.array_equal(b, gl)
        check("closed form " + name, cf)

    for seed in range(10):
        g = random_graph(7 + seed % 5, 0.55, [2, 3, 4][seed % 3], 70 + seed)

        def vs_brute(g=g):
            a, b = oracle.paper(g, lib=lib)
            c, d = oracle.brute(g, lib=lib)
            return np.array_equal(a, c) and np.array_equal(b, d)
        check(f"brute seed={seed}", vs_brute)

    # weighted graph of Alg. 5: column sums are |E(H)| x global counts, D
    # sums W over each node's edges
    edges_of = np.repeat([1, 2, 3, 3, 3, 4, 4, 5, 6], [6, 10, 10, 15, 15, 15, 15, 15, 15])
    for seed in range(3):
        g = random_graph(10 + seed, 0.5, 3, 90 + seed)

        def w_sums(g=g):
            w, d = oracle.weights(g, lib=lib)
            _, gl = oracle.paper(g, lib=lib)
            want_d = np.zeros_like(d)
            src, dst = oracle.edges(g, lib=lib)
            np.add.at(want_d, src, w)
            np.add.at(want_d, dst, w)
            return np.array_equal(w.sum(0), edges_of * gl) and np.array_equal(d, want_d)
        check(f"weights seed={seed}", w_sums)

    # position-aware counts of Sec. 5: mapping every per-edge slot to the
    # class of its instance and summing gives |E(H)| x the global counts
    for seed in range(3):
        g = random_graph(11 + seed, 0.5, 3, 95 + seed)

        def pa_sums(g=g):
            pe, gl = oracle.position_aware(g, lib=lib)
            src, dst = oracle.edges(g, lib=lib)
            ty, L = g["types"], g["L"]
            raw = np.zeros_like(gl)
            classes = {}
            for e in range(len(src)):
                raw[global_slot_pa(L, 0, (ty[src[e]], ty[dst[e]]), classes)] += 1
                for slot in np.nonzero(pe[e])[0]:
                    b, lab = slot_instance(L, int(slot), int(ty[src[e]]), int(ty[dst[e]]))
                    raw[global_slot_pa(L, b, lab, classes)] += pe[e, slot]
            off = np.concatenate([[0], np.cumsum(burnside(L))])
            return all(np.array_equal(raw[off[b]:off[b + 1]], BLOCK_EDGES[b] * gl[off[b]:off[b + 1]])
                       for b in range(9))
        check(f"position-aware seed={seed}", pa_sums)
    failed += directed_pins(lib)
    failed += edge_typed_pins(lib)
    return failed


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def _compile(k, out_dir):
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    out = os.path.join(out_dir, f"liboracle_m{k}.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", f"-DORACLE_MUTANT={k}",
                           "-o", out, src])
    return oracle.open_library(out)


def test_unmutated_build_passes_battery(mutant_dir):
    lib = _compile(0, str(mutant_dir))
    assert _battery(lib) == []


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_planted_mistake_is_caught(k, mutant_dir):
    lib = _compile(k, str(mutant_dir))
    failed = _battery(lib)
    assert failed, f"mutant {k} ({MUTANTS[k]}) passed every pin"
