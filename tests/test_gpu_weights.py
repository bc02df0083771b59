"""Typed-graphlet weighted graph (Alg. 5): W_ij, the number of instances of
a typed graphlet H containing both endpoints of edge (i, j), counted here by
brute force over all 2-, 3- and 4-node sets of small graphs, for every
typed graphlet; and D = row sums of W."""
import itertools

import numpy as np
import pytest

from oracle_pins import random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def shape_block(nodes, adj):
    """Global block of the induced subgraph's shape, or None if disconnected."""
    nodes = list(nodes)
    deg = sorted(sum(1 for y in nodes if y != x and y in adj[x]) for x in nodes)
    ne = sum(deg) // 2
    seen, stack = {nodes[0]}, [nodes[0]]
    while stack:
        x = stack.pop()
        for y in nodes:
            if y in adj[x] and y not in seen:
                seen.add(y)
                stack.append(y)
    if len(seen) < len(nodes):
        return None
    if len(nodes) == 2:
        return 0
    if len(nodes) == 3:
        return 1 if ne == 2 else 2
    if ne == 3:
        return 3 if deg == [1, 1, 2, 2] else 4
    if ne == 4:
        return 5 if deg == [2, 2, 2, 2] else 6
    return 7 if ne == 5 else 8


def brute_weights(g):
    """{(block, rank): int64 [m]} over every typed graphlet, edges in id order."""
    n, L, rp, col, ty = g["n"], g["L"], g["row_ptr"], g["col"], g["types"]
    adj = [set(col[rp[x]:rp[x + 1]].tolist()) for x in range(n)]
    edges = sorted((x, y) for x in range(n) for y in adj[x] if x < y)
    ranks = {K: {ms: r for r, ms in enumerate(itertools.combinations_with_replacement(range(L), K))} for K in (2, 3, 4)}
    W = {}
    for e, (i, j) in enumerate(edges):
        others = [x for x in range(n) if x not in (i, j)]
        for extra in range(3):
            for rest in itertools.combinations(others, extra):
                nodes = (i, j) + rest
                b = shape_block(nodes, adj)
                if b is None:
                    continue
                r = ranks[len(nodes)][tuple(sorted(int(ty[x]) for x in nodes))]
                W.setdefault((b, r), np.zeros(len(edges), np.int64))[e] += 1
    return W, edges


@pytest.mark.parametrize("seed", range(4))
def test_weights_equal_brute_force(seed):
    L = [2, 3, 2, 3][seed]
    g = random_graph(11, [0.4, 0.55, 0.7, 0.5][seed], L, 700 + seed)
    W, edges = brute_weights(g)
    lay = tg.tg_layout(L, 4)
    h = tg.tg_build(*tg.to_device(g), L)
    rows = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    tg.tg_count(h, 4, rows, None)
    w = torch.zeros(h.m, dtype=torch.int64, device="cuda")
    d = torch.zeros(g["n"], dtype=torch.int64, device="cuda")
    for b in range(9):
        for r in range(lay["global_block_size"][b]):
            tg.tg_graphlet_weights(h, 4, rows, b, r, w, d)
            want = W.get((b, r), np.zeros(len(edges), np.int64))
            np.testing.assert_array_equal(w.cpu().numpy(), want, err_msg=f"block {b} rank {r}")
            deg = np.zeros(g["n"], np.int64)
            for e, (i, j) in enumerate(edges):
                deg[i] += want[e]
                deg[j] += want[e]
            np.testing.assert_array_equal(d.cpu().numpy(), deg)
    with pytest.raises(tg.TGError):
        tg.tg_graphlet_weights(h, 4, rows, 9, 0, w)
    with pytest.raises(tg.TGError):
        tg.tg_graphlet_weights(h, 4, rows, 3, lay["global_block_size"][3], w)
    h.free()


def test_weights_k3_one_type_and_empty():
    from oracle_pins import graph_from_edges
    # L = 1: the triangle weight of every edge of K4 is 2, the 3-path weight 0
    g = graph_from_edges(4, [(a, b) for a in range(4) for b in range(a + 1, 4)], [0, 0, 0, 0], 1)
    h = tg.tg_build(*tg.to_device(g), 1)
    rows = torch.zeros((h.m, tg.tg_layout(1, 3)["per_edge_slots"]), dtype=torch.int32, device="cuda")
    tg.tg_count(h, 3, rows, None)
    w = torch.zeros(h.m, dtype=torch.int64, device="cuda")
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    tg.tg_graphlet_weights(h, 3, rows, 2, 0, w, d)
    assert w.tolist() == [2] * 6 and d.tolist() == [6] * 4
    tg.tg_graphlet_weights(h, 3, rows, 1, 0, w)
    assert w.tolist() == [0] * 6
    with pytest.raises(tg.TGError):
        tg.tg_graphlet_weights(h, 3, rows, 3, 0, w)                  # 4-node block with k = 3 rows
    h.free()
    e = graph_from_edges(3, [], [0, 0, 0], 1)
    h = tg.tg_build(*tg.to_device(e), 1)
    d3 = torch.full((3,), 7, dtype=torch.int64, device="cuda")
    tg.tg_graphlet_weights(h, 3, torch.zeros(1, dtype=torch.int32, device="cuda"), 0, 0,
                           torch.zeros(1, dtype=torch.int64, device="cuda"), d3)
    assert d3.tolist() == [0, 0, 0]
    h.free()
