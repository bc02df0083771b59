"""Directed typed 3-node graphlets (Sec. 4.8) on the GPU vs the CPU oracle:
per-edge rows and global totals bit-exact on tiny oriented graphs (against
brute force), tournaments, oriented Chung-Lu and Erdos-Renyi graphs that
span many warps and several CTAs with a ragged tail, every L from 1 to 8,
host buffers, an empty graph, and rejection of reciprocal pairs, repeated
arcs and self-loops."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle_pins import oriented_graph, random_oriented

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def gpu_directed(g, host=False, options=None):
    L = g["L"]
    lay = tg.tg_directed_layout(L)
    if host:
        h = tg.tg_build_directed(np.ascontiguousarray(g["out_row_ptr"], dtype=np.int64),
                                 np.ascontiguousarray(g["out_col"], dtype=np.int32),
                                 np.ascontiguousarray(g["types"], dtype=np.uint8), L)
        pe = np.zeros((h.m, lay["per_edge_slots"]), dtype=np.uint32)
        gl = np.zeros(lay["global_slots"], dtype=np.int64)
        tg.tg_count_directed3(h, pe, gl)
        st = tg.tg_query_status(h)
        h.free()
        return pe.astype(np.int64), gl, st
    rp = torch.as_tensor(np.ascontiguousarray(g["out_row_ptr"], dtype=np.int64), device="cuda")
    col = torch.as_tensor(np.ascontiguousarray(g["out_col"], dtype=np.int32), device="cuda")
    ty = torch.as_tensor(np.ascontiguousarray(g["types"], dtype=np.uint8), device="cuda")
    h = tg.tg_build_directed(rp, col, ty, L, options=options)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count_directed3(h, pe, gl)
    st = tg.tg_query_status(h)
    h.free()
    return pe.cpu().numpy().view(np.uint32).astype(np.int64), gl.cpu().numpy(), st


def assert_directed_parity(g, reference="paper", host=False, options=None):
    pe, gl, st = gpu_directed(g, host=host, options=options)
    assert st == 0, tg.STATUS[st]
    pe_o, gl_o = (oracle.directed3_brute if reference == "brute" else oracle.directed3)(g)
    np.testing.assert_array_equal(pe, pe_o)
    np.testing.assert_array_equal(gl, gl_o)


def oriented_from_undirected(u, seed):
    """Every edge of an undirected graph oriented by a seeded coin."""
    rng = np.random.default_rng(seed)
    rp, col = u["row_ptr"], u["col"]
    arcs = []
    for x in range(u["n"]):
        for y in col[rp[x]:rp[x + 1]]:
            if x < y:
                arcs.append((x, int(y)) if rng.random() < 0.5 else (int(y), x))
    return oriented_graph(u["n"], arcs, u["types"], u["L"])


@pytest.mark.parametrize("seed", range(12))
def test_tiny_oriented_graphs_vs_brute_force(seed):
    L = [1, 2, 3, 5, 8][seed % 5]
    assert_directed_parity(random_oriented(6 + seed, 0.6, L, 1200 + seed), reference="brute")


@pytest.mark.parametrize("L", range(1, 9))
def test_tournaments(L):
    assert_directed_parity(random_oriented(40, 1.0, L, 1300 + L, tournament=True))


@pytest.mark.parametrize("L", [1, 3, 5, 8])
def test_oriented_er_many_ctas_and_ragged_tail(L):
    # 9,123 edges over warps of 8 per CTA: many CTAs, a ragged last one
    assert_directed_parity(oriented_from_undirected(graphgen.erdos_renyi(1500, 9123, L, 51 + L), 61 + L))


def test_oriented_chung_lu_with_hubs():
    u = graphgen.chung_lu(6000, 60000, 2.1, 1500.0, 4, 71, type_zipf=1.2)
    assert_directed_parity(oriented_from_undirected(u, 72))


def test_host_buffers_and_empty_graph():
    assert_directed_parity(random_oriented(30, 0.3, 3, 1400), host=True)
    assert_directed_parity(oriented_graph(5, [], [0, 1, 2, 0, 1], 3))
    assert_directed_parity(oriented_graph(2, [(1, 0)], [0, 1], 2))


def test_direction_sums_equal_undirected_counts():
    g = oriented_from_undirected(graphgen.chung_lu(2000, 12000, 2.2, 400.0, 3, 81), 82)
    pe, _, st = gpu_directed(g)
    assert st == 0
    L = g["L"]
    rp = torch.as_tensor(np.ascontiguousarray(g["out_row_ptr"], dtype=np.int64), device="cuda")
    col = torch.as_tensor(np.ascontiguousarray(g["out_col"], dtype=np.int32), device="cuda")
    ty = torch.as_tensor(np.ascontiguousarray(g["types"], dtype=np.uint8), device="cuda")
    h = tg.tg_build_directed(rp, col, ty, L)        # the same handle counts the underlying undirected graph
    und = torch.zeros((h.m, 2 * L), dtype=torch.int32, device="cuda")
    tg.tg_count(h, 3, und, None)
    h.free()
    und = und.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(pe[:, :4 * L].reshape(-1, 4, L).sum(1), und[:, :L])
    np.testing.assert_array_equal(pe[:, 4 * L:].reshape(-1, 4, L).sum(1), und[:, L:])


@pytest.mark.parametrize("arcs", [[(0, 1), (1, 0)], [(0, 1), (0, 1)], [(2, 2)], [(0, 5)]])
def test_invalid_oriented_graphs_are_rejected(arcs):
    g = oriented_graph(3, [a for a in arcs if a[1] < 3], [0, 0, 0], 1)
    if any(a[1] >= 3 for a in arcs):                      # an arc head out of range
        g["out_col"] = np.array([5], dtype=np.int32)
        g["out_row_ptr"] = np.array([0, 1, 1, 1], dtype=np.int64)
    with pytest.raises(tg.TGError) as e:
        gpu_directed(g, host=True)
    assert e.value.name == "TG_ERR_INVALID_GRAPH"


@pytest.mark.parametrize("modes", [0b01010101, 0b10101010])
def test_intersection_methods(modes):
    # every typed intersection by binary search, then by merge
    u = graphgen.chung_lu(5000, 50000, 2.1, 1500.0, 3, 91, type_zipf=1.2)
    assert_directed_parity(oriented_from_undirected(u, 92), options={"isect_modes": modes})
