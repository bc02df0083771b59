"""Typed-graphlet weighted graph (Alg. 5): W_ij, the number of instances of
a typed graphlet H containing both endpoints of edge (i, j), and D = the row
sums of W, for every typed graphlet, equal to the oracle's direct
enumeration: small graphs, and graphs whose edges span several 256-edge
tiles with a ragged tail, one with a hub adjacent to every node."""
import numpy as np
import pytest

import oracle
from oracle_pins import graph_from_edges, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def with_hub(g):
    """g plus edges from node 0 to every other node."""
    rp, col = g["row_ptr"], g["col"]
    e = {(u, int(v)) for u in range(g["n"]) for v in col[rp[u]:rp[u + 1]] if u < v}
    e |= {(0, v) for v in range(1, g["n"])}
    return graph_from_edges(g["n"], sorted(e), g["types"], g["L"])


CASES = [(11, 0.4, 2, 700), (11, 0.55, 3, 701), (11, 0.7, 2, 702), (11, 0.5, 3, 703),
         (150, 0.15, 3, 704), (120, 0.1, 2, "hub")]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_weights_equal_oracle(case):
    n, p, L, seed = CASES[case]
    g = with_hub(random_graph(n, p, L, 705)) if seed == "hub" else random_graph(n, p, L, seed)
    W, D = oracle.weights(g)
    lay = tg.tg_layout(L, 4)
    h = tg.tg_build(*tg.to_device(g), L)
    rows = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    tg.tg_count(h, 4, rows, None)
    w = torch.zeros(h.m, dtype=torch.int64, device="cuda")
    d = torch.zeros(g["n"], dtype=torch.int64, device="cuda")
    s = 0
    for b in range(9):
        for r in range(lay["global_block_size"][b]):
            tg.tg_graphlet_weights(h, 4, rows, b, r, w, d)
            np.testing.assert_array_equal(w.cpu().numpy(), W[:, s], err_msg=f"block {b} rank {r}")
            np.testing.assert_array_equal(d.cpu().numpy(), D[:, s], err_msg=f"block {b} rank {r}")
            s += 1
    assert s == W.shape[1]
    with pytest.raises(tg.TGError):
        tg.tg_graphlet_weights(h, 4, rows, 9, 0, w)
    with pytest.raises(tg.TGError):
        tg.tg_graphlet_weights(h, 4, rows, 3, lay["global_block_size"][3], w)
    h.free()


def test_weights_k3_one_type_and_empty():
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
