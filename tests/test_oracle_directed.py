"""The directed typed 3-node oracle (Sec. 4.8), pinned on the CPU.

Pins: the number of classes equals Burnside's count for every L = 1..8;
Alg. 1 with direction-split sets equals brute force over all 3-subsets;
summing over the directions gives the undirected typed counts of the
undirected oracle (per edge and global); reversing every arc maps out- to
in-neighbours and every class to its reversed class; closed forms for a
transitive tournament, directed stars, and the Kendall-Babington Smith
count of cyclic triangles in a tournament.  Invalid oriented graphs
(reciprocal pairs, repeated arcs, self-loops) are rejected.
"""
import numpy as np
import pytest

import oracle
from oracle_pins import directed_burnside, directed_pins, oriented_graph, random_oriented


def test_directed_pins():
    assert directed_pins() == []


@pytest.mark.parametrize("L", range(1, 9))
def test_class_count_is_burnside(L):
    assert oracle.directed_classes(L) == directed_burnside(L)
    assert oracle.directed_global_slots(L) == L * L + directed_burnside(L)


def test_classes_of_one_type():
    # out-star, in-star, chain, transitive and cyclic triangle: five classes,
    # each configuration of a class gets the same rank
    z = [0, 0, 0]
    ranks = {
        "out-star": [oracle.directed_class(1, z, a) for a in ([1, 1, 0], [2, 0, 1], [0, 2, 2])],
        "in-star": [oracle.directed_class(1, z, a) for a in ([2, 2, 0], [1, 0, 2], [0, 1, 1])],
        "chain": [oracle.directed_class(1, z, a) for a in ([1, 0, 1], [2, 1, 0], [0, 2, 1])],
        "transitive": [oracle.directed_class(1, z, a) for a in ([1, 1, 1], [2, 2, 2], [1, 2, 2])],
        "cyclic": [oracle.directed_class(1, z, a) for a in ([1, 2, 1], [2, 1, 2])],
    }
    reps = {k: set(v) for k, v in ranks.items()}
    assert all(len(v) == 1 for v in reps.values())
    assert sorted(r for v in reps.values() for r in v) == list(range(5))
    assert oracle.directed_class(1, z, [1, 0, 0]) == -1        # one arc: not connected


def test_invalid_oriented_graphs_are_rejected():
    t = [0, 0, 0]
    for arcs in ([(0, 1), (1, 0)],            # reciprocal pair
                 [(0, 1), (0, 1)],            # repeated arc
                 [(0, 0)]):                   # self-loop
        with pytest.raises(oracle.OracleError):
            oracle.directed3(oriented_graph(3, arcs, t, 1))


def test_brute_force_larger_types():
    for seed in range(3):
        g = random_oriented(10, 0.6, 5, 900 + seed)
        pe, gl = oracle.directed3(g)
        pb, gb = oracle.directed3_brute(g)
        np.testing.assert_array_equal(pe, pb)
        np.testing.assert_array_equal(gl, gb)
