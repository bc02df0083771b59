"""The edge-typed 3-node oracle (Def. 1's edge types xi; Defs. 4-5: a
typed graphlet's class is its shape with the multisets of its node types and
of its edge types), pinned on the CPU against what the definitions fix:

* brute force over every 3-node subset of small random graphs;
* the edge types summed out give the typed (node types only) 3-node rows
  and totals of the independent Alg. 1 route (oracle.paper, k = 3);
* a permutation of the edge types permutes the slots accordingly;
* closed forms: a triangle with three distinct edge types, and a star whose
  leaves' edges carry two types (C(4,2), 4·3 and C(3,2) 3-paths by pair);
* inputs whose two entries of an edge disagree on its type, or whose types
  are out of range, are rejected.
"""
import numpy as np
import pytest

import oracle
from oracle_pins import edge_typed_pins, edge_types_for, graph_from_edges, multisets, random_graph


def test_pins():
    assert edge_typed_pins() == []


@pytest.mark.parametrize("L,X", [(1, 1), (2, 3), (5, 4), (8, 8)])
def test_layout_sizes(L, X):
    assert oracle.edge_typed_per_edge_slots(L, X) == L * X + L * X * (X + 1) // 2
    assert oracle.edge_typed_global_slots(L, X) == (len(multisets(L, 2)) * X + len(multisets(L, 3)) * len(multisets(X, 2))
                                                    + len(multisets(L, 3)) * len(multisets(X, 3)))


def test_one_edge_type_is_the_typed_count():
    g = random_graph(12, 0.45, 3, 31)
    xi = np.zeros(len(g["col"]), dtype=np.uint8)
    pe, gl = oracle.edge_typed3(g, xi, 1)
    pt, gt = oracle.paper(g, k=3)
    assert np.array_equal(pe, pt) and np.array_equal(gl, gt)


def test_disagreeing_entries_are_rejected():
    g = graph_from_edges(3, [(0, 1), (1, 2)], [0, 0, 0], 1)
    xi = edge_types_for(g, 2, 5)
    rp, col = g["row_ptr"], g["col"]
    k = int(rp[0])                                      # the entry of edge {0, 1} in row 0
    xi[k] = 1 - xi[k]
    with pytest.raises(oracle.OracleError):
        oracle.edge_typed3(g, xi, 2)


def test_out_of_range_types_are_rejected():
    g = graph_from_edges(3, [(0, 1), (1, 2)], [0, 0, 0], 1)
    xi = np.full(len(g["col"]), 2, dtype=np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.edge_typed3(g, xi, 2)


def test_seeded_edge_types_are_symmetric_and_reproducible():
    # the bench's input generator: one type per edge on both of its entries,
    # the same for the same seed, spread over [0, X)
    import graphgen
    g = graphgen.chung_lu(3000, 20000, 2.1, 600.0, 3, 17)
    xi = graphgen.edge_types(g, 4, 99)
    assert np.array_equal(xi, graphgen.edge_types(g, 4, 99))
    assert not np.array_equal(xi, graphgen.edge_types(g, 4, 98))
    pe, gl = oracle.edge_typed3(g, xi, 4, per_edge=False)        # rejects unequal entries
    counts = np.bincount(xi, minlength=4)
    assert counts.min() > 0.2 * len(xi) and xi.max() < 4
