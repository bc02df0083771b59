"""The oracle's typed-graphlet weighted graph (Alg. 5, first two steps) pinned
to closed forms, to the global counts of Sec. 4.4 / Sec. 6 and the per-edge
orbit counts of Alg. 1-3 (a different route through the oracle), and to a
networkx classification of every node set containing an edge.

W[e][s] is the number of instances of typed graphlet s (global slot) that
contain both endpoints of edge e; D[v][s] is the sum of W over the edges at v.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import oracle
from oracle_pins import (GRAPHLET_EDGES, edge_list, global_size, global_slot, graph_from_edges, per_edge_slot,
                         random_graph)

BLOCK_EDGES = {0: 1, **GRAPHLET_EDGES}          # |E(H)| per global block
ORBITS_OF = {3: (3, 4), 4: (5,), 5: (6,), 6: (7, 8, 9), 7: (10, 11), 8: (12,)}


def _blocks(L):
    sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    return np.concatenate([[0], np.cumsum(sizes)])


def _untyped_rows(g):
    """W of an L = 1 graph as [m, 9]: one slot per block."""
    w, _ = oracle.weights(dict(g, L=1, types=np.zeros_like(g["types"])))
    return w


# ----------------------------------------------------------- closed forms

@pytest.mark.parametrize("types,L", [([0] * 6, 1), ([0, 0, 1, 2, 1, 0, 2], 3), ([3, 1, 1, 0, 2, 3, 3, 1], 4)])
def test_typed_clique(types, L):
    """K_n: the other n-2 nodes each close a triangle with the edge and every
    pair of them a 4-clique; nothing else is induced."""
    n = len(types)
    g = graph_from_edges(n, [(a, b) for a in range(n) for b in range(a + 1, n)], types, L)
    w, d = oracle.weights(g)
    for e, (i, j) in enumerate(edge_list(g)):
        want = np.zeros(global_size(L), np.int64)
        want[global_slot(L, 0, [types[i], types[j]])] = 1
        others = [x for x in range(n) if x not in (i, j)]
        for t, c in Counter(types[x] for x in others).items():
            want[global_slot(L, 2, [types[i], types[j], t])] += c
        for x, y in itertools.combinations(others, 2):
            want[global_slot(L, 8, [types[i], types[j], types[x], types[y]])] += 1
        np.testing.assert_array_equal(w[e], want)


def test_typed_star():
    """Star: a leaf edge lies on a 3-path with every other leaf and on a
    4-star with every pair of other leaves."""
    leaves = [0, 1, 2, 0, 2, 2]
    L, n = 3, 7
    types = [1] + leaves
    g = graph_from_edges(n, [(0, a) for a in range(1, n)], types, L)
    w, _ = oracle.weights(g)
    for e, (c, a) in enumerate(edge_list(g)):
        want = np.zeros(global_size(L), np.int64)
        want[global_slot(L, 0, [1, types[a]])] = 1
        rest = [x for x in range(1, n) if x != a]
        for b in rest:
            want[global_slot(L, 1, [1, types[a], types[b]])] += 1
        for b, b2 in itertools.combinations(rest, 2):
            want[global_slot(L, 4, [1, types[a], types[b], types[b2]])] += 1
        np.testing.assert_array_equal(w[e], want)


@pytest.mark.parametrize("types,L", [([0, 1, 2, 0, 1], 3), ([1, 0, 2, 3, 0, 1, 3, 2, 2], 4), ([0] * 7, 1)])
def test_typed_cycle(types, L):
    """Cycle C_n, n >= 5: the edge (v_k, v_k+1) is on the 3-paths through
    v_k-1 and v_k+2 and on the three 4-paths that extend it by two nodes."""
    n = len(types)
    g = graph_from_edges(n, [(a, (a + 1) % n) for a in range(n)], types, L)
    w, _ = oracle.weights(g)
    for e, (i, j) in enumerate(edge_list(g)):
        k = i if (i + 1) % n == j else j                 # the edge is (v_k, v_k+1)
        v = lambda r: types[(k + r) % n]                  # noqa: E731
        want = np.zeros(global_size(L), np.int64)
        want[global_slot(L, 0, [v(0), v(1)])] = 1
        for x in (-1, 2):
            want[global_slot(L, 1, [v(0), v(1), v(x)])] += 1
        for x, y in ((-2, -1), (-1, 2), (2, 3)):
            want[global_slot(L, 3, [v(0), v(1), v(x), v(y)])] += 1
        np.testing.assert_array_equal(w[e], want)


def test_four_cycle():
    g = graph_from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 3)], [0] * 4, 1)
    np.testing.assert_array_equal(oracle.weights(g)[0], [[1, 2, 0, 0, 0, 1, 0, 0, 0]] * 4)


@pytest.mark.parametrize("a,b", [(2, 3), (3, 4), (4, 4), (1, 5)])
def test_complete_bipartite(a, b):
    """K_{a,b}: the edge (x, y) is on a+b-2 3-paths, on C(b-1,2) + C(a-1,2)
    4-stars (two more nodes on one side) and (a-1)(b-1) 4-cycles."""
    g = graph_from_edges(a + b, [(x, a + y) for x in range(a) for y in range(b)], [0] * (a + b), 1)
    want = [1, a + b - 2, 0, 0, math.comb(a - 1, 2) + math.comb(b - 1, 2), (a - 1) * (b - 1), 0, 0, 0]
    np.testing.assert_array_equal(oracle.weights(g)[0], [want] * (a * b))


def test_tailed_triangle_and_diamond():
    """A tailed triangle (triangle 0-1-2, tail 2-3) and a diamond (K4 less
    the edge 0-3), written out edge by edge; slots are blocks for L = 1."""
    tt = graph_from_edges(4, [(0, 1), (0, 2), (1, 2), (2, 3)], [0] * 4, 1)
    #               edge   2-node 3-path tri 4-path star cycle tailed chordal clique
    np.testing.assert_array_equal(oracle.weights(tt)[0], [
        [1, 0, 1, 0, 0, 0, 1, 0, 0],      # 0-1: third node 2 closes the triangle
        [1, 1, 1, 0, 0, 0, 1, 0, 0],      # 0-2: 3 hangs off 2
        [1, 1, 1, 0, 0, 0, 1, 0, 0],      # 1-2
        [1, 2, 0, 0, 0, 0, 1, 0, 0]])     # 2-3: paths 3-2-0 and 3-2-1
    di = graph_from_edges(4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)], [0] * 4, 1)
    np.testing.assert_array_equal(oracle.weights(di)[0], [
        [1, 1, 1, 0, 0, 0, 0, 1, 0],      # 0-1: 0-1-2 triangle, 0-1-3 path
        [1, 1, 1, 0, 0, 0, 0, 1, 0],      # 0-2
        [1, 0, 2, 0, 0, 0, 0, 1, 0],      # 1-2: the chord, in both triangles
        [1, 1, 1, 0, 0, 0, 0, 1, 0],      # 1-3
        [1, 1, 1, 0, 0, 0, 0, 1, 0]])     # 2-3


def test_empty_and_edgeless():
    w, d = oracle.weights(graph_from_edges(5, [], [0, 1, 0, 1, 1], 2))
    assert w.shape == (0, global_size(2)) and not d.any()


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("seed", range(6))
def test_sums_equal_edges_times_global_count(seed):
    """Sec. 4.4 / Sec. 6: every instance of H is counted once on each of its
    |E(H)| edges, so the column sums of W are |E(H)| times the global counts
    (here from Alg. 1-3 + Lemmas, another route); D sums W over each node's
    edges."""
    g = random_graph(12 + seed, 0.4, [2, 3, 4][seed % 3], 5100 + seed)
    L = g["L"]
    w, d = oracle.weights(g)
    _, gl = oracle.paper(g)
    off = _blocks(L)
    for b in range(9):
        np.testing.assert_array_equal(w[:, off[b]:off[b + 1]].sum(0), BLOCK_EDGES[b] * gl[off[b]:off[b + 1]])
    want_d = np.zeros_like(d)
    for e, (i, j) in enumerate(edge_list(g)):
        want_d[i] += w[e]
        want_d[j] += w[e]
    np.testing.assert_array_equal(d, want_d)


@pytest.mark.parametrize("seed", range(6))
def test_matches_per_edge_orbits(seed):
    """With the edge's types (p, q) fixed, the instances of a typed graphlet
    containing the edge are its orbit counts whose other nodes complete the
    type multiset: the orbit slots of Alg. 1-3 + Lemmas, summed over the
    graphlet's orbits."""
    g = random_graph(11 + seed, 0.45, [2, 3][seed % 2], 5200 + seed)
    L, ty = g["L"], g["types"]
    w, _ = oracle.weights(g)
    pe, _ = oracle.paper(g)
    for e, (i, j) in enumerate(edge_list(g)):
        p, q = int(ty[i]), int(ty[j])
        want = np.zeros(global_size(L), np.int64)
        want[global_slot(L, 0, [p, q])] = 1
        for t in range(L):
            want[global_slot(L, 1, [p, q, t])] += pe[e, per_edge_slot(L, 1, t)]
            want[global_slot(L, 2, [p, q, t])] += pe[e, per_edge_slot(L, 2, t)]
        for h, orbits in ORBITS_OF.items():
            for t, u in itertools.combinations_with_replacement(range(L), 2):
                want[global_slot(L, h, [p, q, t, u])] += sum(pe[e, per_edge_slot(L, o, t, u)] for o in orbits)
        np.testing.assert_array_equal(w[e], want)


def test_untyped_is_sum_over_types():
    """Prop. 1 for W: summing a block over all type multisets gives the
    untyped weight."""
    g = random_graph(13, 0.4, 3, 5300)
    w, _ = oracle.weights(g)
    w1 = _untyped_rows(g)
    off = _blocks(3)
    for b in range(9):
        np.testing.assert_array_equal(w[:, off[b]:off[b + 1]].sum(1), w1[:, b])


@pytest.mark.parametrize("seed", range(3))
def test_networkx_classification(seed):
    """Every connected node set containing the edge, classified by networkx
    isomorphism against the eight graphlets."""
    nx = pytest.importorskip("networkx")
    shapes = [nx.path_graph(2), nx.path_graph(3), nx.complete_graph(3), nx.path_graph(4), nx.star_graph(3),
              nx.cycle_graph(4), nx.Graph([(0, 1), (0, 2), (1, 2), (2, 3)]),
              nx.Graph([(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)]), nx.complete_graph(4)]
    g = random_graph(9 + seed, 0.5, 2, 5400 + seed)
    n, L, ty = g["n"], g["L"], g["types"]
    G = nx.Graph(edge_list(g))
    G.add_nodes_from(range(n))
    want = np.zeros((len(edge_list(g)), global_size(L)), np.int64)
    for e, (i, j) in enumerate(edge_list(g)):
        others = [x for x in range(n) if x not in (i, j)]
        for extra in range(3):
            for rest in itertools.combinations(others, extra):
                nodes = (i, j) + rest
                sub = G.subgraph(nodes)
                if not nx.is_connected(sub):
                    continue
                b = next(k for k, s in enumerate(shapes) if len(s) == len(nodes) and nx.is_isomorphic(sub, s))
                want[e, global_slot(L, b, [ty[x] for x in nodes])] += 1
    np.testing.assert_array_equal(oracle.weights(g)[0], want)
