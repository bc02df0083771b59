"""The CPU oracle pinned to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), closed forms of graph families, invariants the
paper states (Prop. 1, Sec. 4.4, Sec. 6), standard untyped identities,
subgraph isomorphism by networkx, and library enumeration order for the
layout.  The three oracle routes (Alg. 1-3 + Lemmas, Table 3 definitions,
brute force) must also agree with each other.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen
import oracle
from oracle_pins import (GRAPHLET_EDGES, edge_list, expected_clique, expected_complete_bipartite,
                         expected_cycle, expected_path, expected_star, global_size, global_slot,
                         graph_from_edges, multisets, pairs, per_edge_slot, random_graph, read_golden,
                         untyped_identities)


# ------------------------------------------------------------------ layout

def test_table2_typed_graphlet_counts():
    """Table 2: ((L multichoose K)) for K = 2..4, L = 1..9 equals the
    oracle's global block sizes."""
    for row in read_golden("table2_typed_graphlet_counts.txt"):
        K = int(row[0])
        for L, val in enumerate(map(int, row[1:]), start=1):
            assert math.comb(L + K - 1, K) == val
            sizes2 = oracle.global_slots(L, 3) - 2 * math.comb(L + 2, 3)   # block 0 alone
            if K == 2:
                assert sizes2 == val
            if K == 3:
                assert (oracle.global_slots(L, 3) - sizes2) == 2 * val
            if K == 4:
                assert (oracle.global_slots(L, 4) - oracle.global_slots(L, 3)) == 6 * val


def test_layout_figures_printed_in_paper():
    fig = {r[0]: int(r[1]) for r in read_golden("layout_figures.txt")}
    L = 7
    n2 = math.comb(L + 1, 2)
    assert oracle.global_slots(L, 4) - n2 == fig["possible_3_4_node_typed_graphlets_L7"]
    assert oracle.global_slots(L, 3) - n2 == fig["possible_3_node_typed_graphlets_L7"]
    assert 10 * math.comb(L + 3, 4) == fig["typed_4_node_orbits_L7"]
    orbit_slots = 2 * math.comb(L + 2, 3) + 10 * math.comb(L + 3, 4)
    assert 10_000_000 * 4 * orbit_slots == fig["dense_orbit_bytes_M1e7_L7"]


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8])
def test_ranks_follow_lexicographic_enumeration(L):
    for k, (t, tp) in enumerate(pairs(L)):
        assert oracle.pair_index(L, t, tp) == k
        assert oracle.pair_index(L, tp, t) == k
    for K in (2, 3, 4):
        for k, ms in enumerate(multisets(L, K)):
            for perm in set(itertools.permutations(ms)):
                assert oracle.multiset_rank(L, perm) == k
    assert oracle.per_edge_slots(L, 4) == 2 * L + 10 * L * (L + 1) // 2
    assert oracle.per_edge_slots(L, 3) == 2 * L
    assert oracle.global_slots(L, 4) == global_size(L)


# ------------------------------------------------------------ closed forms

def _check(g, edges, pe_exp, gl_exp):
    pe, gl = oracle.paper(g)
    assert edge_list(g) == [tuple(e) for e in edges]
    np.testing.assert_array_equal(pe, pe_exp)
    np.testing.assert_array_equal(gl, gl_exp)
    pe3, gl3 = oracle.table3(g)
    np.testing.assert_array_equal(pe3, pe_exp)
    np.testing.assert_array_equal(gl3, gl_exp)


@pytest.mark.parametrize("types,L", [([0] * 6, 1), ([0, 0, 1, 2, 1, 0, 2], 3), ([3, 1, 1, 0, 2, 3, 3, 1], 4)])
def test_typed_clique(types, L):
    edges, pe, gl = expected_clique(np.array(types), L)
    g = graph_from_edges(len(types), edges, types, L)
    _check(g, edges, pe, gl)


@pytest.mark.parametrize("center,leaves,L", [(0, [0, 0, 0, 0], 1), (1, [0, 1, 2, 0, 2, 2], 3), (2, [0, 1, 2, 3, 0, 1, 1], 4)])
def test_typed_star(center, leaves, L):
    types, edges, pe, gl = expected_star(center, leaves, L)
    g = graph_from_edges(len(types), edges, types, L)
    _check(g, edges, pe, gl)


@pytest.mark.parametrize("types,L", [([0, 1, 2, 0, 1], 3), ([0, 0, 1, 1, 0, 2], 3), ([1, 0, 2, 3, 0, 1, 3, 2, 2], 4), ([0] * 7, 1)])
def test_typed_cycle(types, L):
    edges, pe, gl = expected_cycle(types, L)
    g = graph_from_edges(len(types), edges, types, L)
    _check(g, edges, pe, gl)


def test_four_cycle():
    types, L = [0, 1, 1, 2], 3
    edges = [(0, 1), (1, 2), (2, 3), (0, 3)]
    g = graph_from_edges(4, edges, types, L)
    pe, gl = oracle.paper(g)
    for e, (a, b) in enumerate(edge_list(g)):
        others = [x for x in range(4) if x not in (a, b)]
        row = np.zeros(pe.shape[1], dtype=np.int64)
        for x in others:
            row[per_edge_slot(L, 1, types[x])] += 1
        row[per_edge_slot(L, 6, types[others[0]], types[others[1]])] = 1
        np.testing.assert_array_equal(pe[e], row)
    assert gl[global_slot(L, 5, types)] == 1
    assert gl.sum() == 4 + 4 + 1


@pytest.mark.parametrize("a,b", [(2, 3), (3, 4), (4, 4), (1, 5)])
def test_complete_bipartite(a, b):
    types, edges, pe, gl = expected_complete_bipartite(a, b)
    g = graph_from_edges(a + b, edges, types, 2)
    _check(g, edges, pe, gl)


@pytest.mark.parametrize("types,L", [([0, 1, 0, 2, 1, 1, 0], 3), ([0, 0], 1), ([1, 0, 1], 2)])
def test_typed_path(types, L):
    edges, pe, gl = expected_path(types, L)
    g = graph_from_edges(len(types), edges, types, L)
    _check(g, edges, pe, gl)


def test_empty_and_isolated():
    g = graph_from_edges(5, [], [0, 1, 2, 0, 1], 3)
    pe, gl = oracle.paper(g)
    assert pe.shape == (0, oracle.per_edge_slots(3, 4))
    assert not gl.any()
    g = graph_from_edges(6, [(1, 4)], [0, 1, 2, 0, 1, 2], 3)
    pe, gl = oracle.paper(g)
    assert not pe.any()
    assert gl[global_slot(3, 0, (1, 1))] == 1 and gl.sum() == 1


# ------------------------------------------------ three routes agree

@pytest.mark.parametrize("seed", range(40))
def test_paper_table3_brute_agree(seed):
    n = 5 + seed % 9
    p = [0.25, 0.45, 0.65, 0.9][seed % 4]
    L = [1, 2, 3, 5, 8][seed % 5]
    g = random_graph(n, p, L, 1000 + seed)
    a = oracle.paper(g)
    b = oracle.table3(g)
    c = oracle.brute(g)
    for x, y in ((a, c), (b, c)):
        np.testing.assert_array_equal(x[0], y[0])
        np.testing.assert_array_equal(x[1], y[1])


def test_k3_is_prefix_of_k4():
    g = random_graph(12, 0.4, 3, 7)
    pe4, gl4 = oracle.paper(g, k=4)
    pe3, gl3 = oracle.paper(g, k=3)
    np.testing.assert_array_equal(pe3, pe4[:, :6])
    np.testing.assert_array_equal(gl3, gl4[:len(gl3)])


def test_sampled_edges_match_full_run():
    g = graphgen.erdos_renyi(300, 2000, 4, 99)
    pe, _ = oracle.paper(g)
    ids = np.array([0, 5, 17, 1999, 1000, 5], dtype=np.int64)
    rows, sums = oracle.paper_edges(g, ids)
    np.testing.assert_array_equal(rows, pe[ids])
    _, gl = oracle.paper(g)


# ---------------------------------------------------- networkx isomorphism

def test_networkx_isomorphism_classification():
    """Each connected induced 3-/4-node subgraph classified by isomorphism
    to the named graphlets, each edge's orbit read from a fixed drawing of
    the graphlet (Table 3's orbit pictures)."""
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.isomorphism import GraphMatcher

    def G(edges):
        h = nx.Graph()
        h.add_edges_from(edges)
        return h

    # (graphlet index in the global vector, graph, {edge: orbit})
    canon4 = [
        (3, G([(0, 1), (1, 2), (2, 3)]), {(0, 1): 3, (2, 3): 3, (1, 2): 4}),
        (4, G([(0, 1), (0, 2), (0, 3)]), {(0, 1): 5, (0, 2): 5, (0, 3): 5}),
        (5, G([(0, 1), (1, 2), (2, 3), (0, 3)]), {e: 6 for e in [(0, 1), (1, 2), (2, 3), (0, 3)]}),
        (6, G([(0, 1), (1, 2), (0, 2), (2, 3)]), {(2, 3): 7, (0, 1): 8, (0, 2): 9, (1, 2): 9}),
        (7, G([(0, 1), (1, 2), (2, 3), (0, 3), (0, 2)]), {(0, 2): 11, (0, 1): 10, (1, 2): 10, (2, 3): 10, (0, 3): 10}),
        (8, nx.complete_graph(4), {e: 12 for e in itertools.combinations(range(4), 2)}),
    ]
    for seed in range(12):
        n, L = 8 + seed % 3, [2, 3, 4][seed % 3]
        g = random_graph(n, 0.5, L, 500 + seed)
        ty = g["types"]
        H = nx.Graph()
        H.add_nodes_from(range(n))
        H.add_edges_from(edge_list(g))
        eid = {e: k for k, e in enumerate(edge_list(g))}
        S = oracle.per_edge_slots(L, 4)
        pe = np.zeros((len(eid), S), dtype=np.int64)
        gl = np.zeros(global_size(L), dtype=np.int64)
        for e in eid:
            gl[global_slot(L, 0, (ty[e[0]], ty[e[1]]))] += 1
        for sub in itertools.combinations(range(n), 3):
            h = H.subgraph(sub)
            if h.number_of_edges() < 2:
                continue
            gid = 1 if h.number_of_edges() == 2 else 2
            gl[global_slot(L, gid, [ty[x] for x in sub])] += 1
            for a, b in h.edges():
                (z,) = [x for x in sub if x not in (a, b)]
                pe[eid[(min(a, b), max(a, b))], per_edge_slot(L, gid, ty[z])] += 1
        for sub in itertools.combinations(range(n), 4):
            h = H.subgraph(sub)
            if not nx.is_connected(h):
                continue
            for gid, c, orb in canon4:
                gm = GraphMatcher(h, c)
                if gm.is_isomorphic():
                    mapping = next(gm.isomorphisms_iter())
                    gl[global_slot(L, gid, [ty[x] for x in sub])] += 1
                    for a, b in h.edges():
                        ca, cb = mapping[a], mapping[b]
                        o = orb[(min(ca, cb), max(ca, cb))]
                        z = [x for x in sub if x not in (a, b)]
                        pe[eid[(min(a, b), max(a, b))], per_edge_slot(L, o, ty[z[0]], ty[z[1]])] += 1
                    break
        pe_o, gl_o = oracle.paper(g)
        np.testing.assert_array_equal(pe_o, pe)
        np.testing.assert_array_equal(gl_o, gl)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(6))
def test_sum_over_types_is_untyped(seed):
    """Prop. 1: summing typed counts over all type combinations gives the
    untyped counts (per edge and global)."""
    g = random_graph(14, 0.35, 4, 2000 + seed)
    L = g["L"]
    pe, gl = oracle.paper(g)
    g1 = dict(g, L=1, types=np.zeros_like(g["types"]))
    pe1, gl1 = oracle.paper(g1)
    P = L * (L + 1) // 2
    np.testing.assert_array_equal(pe[:, :L].sum(1), pe1[:, 0])
    np.testing.assert_array_equal(pe[:, L:2 * L].sum(1), pe1[:, 1])
    for o in range(10):
        np.testing.assert_array_equal(pe[:, 2 * L + o * P:2 * L + (o + 1) * P].sum(1), pe1[:, 2 + o])
    sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(9):
        assert gl[off[b]:off[b + 1]].sum() == gl1[b]


@pytest.mark.parametrize("seed", range(4))
def test_type_permutation_equivariance(seed):
    rng = np.random.default_rng(seed)
    g = random_graph(13, 0.4, 4, 3000 + seed)
    L = g["L"]
    pi = rng.permutation(L)
    gp = dict(g, types=pi[g["types"]].astype(np.uint8))
    pe, gl = oracle.paper(g)
    pep, glp = oracle.paper(gp)
    for o in (1, 2):
        for t in range(L):
            np.testing.assert_array_equal(pep[:, per_edge_slot(L, o, pi[t])], pe[:, per_edge_slot(L, o, t)])
    for o in range(3, 13):
        for t, tp in pairs(L):
            np.testing.assert_array_equal(pep[:, per_edge_slot(L, o, pi[t], pi[tp])],
                                          pe[:, per_edge_slot(L, o, t, tp)])
    for gid, K in [(0, 2), (1, 3), (2, 3)] + [(h, 4) for h in range(3, 9)]:
        for ms in multisets(L, K):
            assert glp[global_slot(L, gid, [pi[x] for x in ms])] == gl[global_slot(L, gid, ms)]


@pytest.mark.parametrize("seed", range(4))
def test_untyped_identities_and_property1(seed):
    g = graphgen.erdos_renyi(60, 400 + 100 * seed, 3, 4000 + seed)
    g1 = dict(g, L=1, types=np.zeros_like(g["types"]))
    pe1, gl1 = oracle.paper(g1)
    for lhs, rhs in untyped_identities(g, gl1):
        assert lhs == rhs
    # the degree identity of Sec. 7.1 with S_i excluding j (and S_j excluding i):
    # d_i + d_j = 2|T_ij| + |S_i| + |S_j| + 2
    deg = np.diff(g["row_ptr"])
    for e, (a, b) in enumerate(edge_list(g)):
        assert deg[a] + deg[b] == 2 * pe1[e, 1] + pe1[e, 0] + 2
    # Sec. 6: per-edge sums are exact multiples of |E(H)|
    s = pe1[:, 2:].sum(0)
    per_graphlet = [s[0] + s[1], s[2], s[3], s[4] + s[5] + s[6], s[7] + s[8], s[9]]
    for h, tot in zip(range(3, 9), per_graphlet):
        assert tot == GRAPHLET_EDGES[h] * gl1[h]


def test_er_distinct_typed_graphlets_statistical():
    """Sanity only (another random graph than the paper's): ER(10K, 0.001),
    L = 5 uniform types shows nearly every 3-path and 4-path/4-star type
    multiset and few distinct typed 4-cliques (Table 6, synthetic rows)."""
    ref = [int(x) for x in read_golden("er_distinct_typed_graphlets.txt")[0]]
    g = graphgen.erdos_renyi(10_000, 49_995, 5, 77)
    _, gl = oracle.paper(g, per_edge=False)
    L = 5
    sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    off = np.concatenate([[0], np.cumsum(sizes)])
    distinct = [int((gl[off[b]:off[b + 1]] > 0).sum()) for b in range(1, 9)]
    assert distinct[0] == ref[0]                      # 3-path: all 35
    assert abs(distinct[1] - ref[1]) <= 8             # triangles: ~30
    assert distinct[2] == ref[2] and distinct[3] == ref[3]   # 4-path, 4-star: all 70
    assert distinct[6] <= 6 and distinct[7] <= 2      # chordal-cycle, 4-clique: rare


# ------------------------------------------------------------- validation

def test_invalid_graphs_rejected():
    L = 2
    ok = graph_from_edges(3, [(0, 1), (1, 2)], [0, 1, 0], L)
    assert oracle.validate(ok) == 0
    bad_type = dict(ok, types=np.array([0, 2, 0], dtype=np.uint8))
    assert oracle.validate(bad_type) == 2
    self_loop = dict(ok, row_ptr=np.array([0, 2, 3, 4]), col=np.array([0, 1, 0, 1], dtype=np.int32))
    assert oracle.validate(self_loop) == 2
    asym = dict(ok, row_ptr=np.array([0, 1, 2, 2]), col=np.array([1, 2], dtype=np.int32))
    assert oracle.validate(asym) == 2
    dup = dict(ok, row_ptr=np.array([0, 2, 4, 4]), col=np.array([1, 1, 0, 0], dtype=np.int32))
    assert oracle.validate(dup) == 2
