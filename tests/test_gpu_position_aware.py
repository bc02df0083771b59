"""Position-aware typed graphlets (Sec. 5, Def. 8) on the GPU, through the C
ABI, bit-exact against the oracle: per-edge rows (uint32) and per-class
totals (int64) on tiny graphs, graphs spanning many epilogue tiles with
a ragged tail (L = 2, 5, 8), a skewed Chung-Lu graph with every wedge anchor
routed through each kernel variant, a batch handle, host buffers; and, on a
larger graph, the position-aware rows and totals merge into the typed ones of
tg_count on the same handle."""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import concat_graphs
from oracle_pins import graph_from_edges, merge_pa_global, merge_per_edge, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402

ALL_HEAVY = {"light_edge_max_degree": 1, "light_anchor_max_wedges": 1}
ALL_HUB = {"light_edge_max_degree": 1, "light_anchor_max_wedges": 1, "hub_min_wedges": 1}


def pa_gpu(g, options=None, host_buffers=False):
    L = g["L"]
    lay = tg.tg_pa_layout(L)
    h = tg.tg_build(*tg.to_device(g), L, options=options)
    if host_buffers:
        pe = np.zeros((h.m, lay["per_edge_slots"]), dtype=np.uint32)
        gl = np.zeros(lay["global_slots"], dtype=np.int64)
        tg.tg_count_position_aware(h, pe, gl)
        pe_np, gl_np = pe.astype(np.int64), gl
    else:
        pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
        gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
        tg.tg_count_position_aware(h, pe, gl)
        pe_np, gl_np = pe.cpu().numpy().view(np.uint32).astype(np.int64), gl.cpu().numpy()
    st = tg.tg_query_status(h)
    h.free()
    return pe_np, gl_np, st


def assert_pa(g, options=None, host_buffers=False):
    pe, gl, st = pa_gpu(g, options, host_buffers)
    assert st == 0, tg.STATUS[st]
    pe_o, gl_o = oracle.position_aware(g)
    np.testing.assert_array_equal(pe, pe_o)
    np.testing.assert_array_equal(gl, gl_o)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_graphs(seed):
    g = random_graph(5 + seed % 11, [0.3, 0.5, 0.7, 0.95][seed % 4], [1, 2, 3, 4, 5, 8][seed % 6], 9500 + seed)
    assert_pa(g, options=[None, ALL_HEAVY, ALL_HUB][seed % 3])


def test_degenerate_graphs():
    assert_pa(graph_from_edges(4, [], [0, 1, 2, 0], 3))
    assert_pa(graph_from_edges(6, [(2, 5)], [0, 1, 2, 0, 1, 2], 3))
    assert_pa(graph_from_edges(7, [(0, x) for x in range(1, 7)], [1, 0, 1, 2, 0, 2, 2], 3))
    assert_pa(graph_from_edges(8, [(a, b) for a in range(8) for b in range(a + 1, 8)], [0, 1, 2, 3, 0, 1, 2, 3], 4))
    assert_pa(graph_from_edges(7, [(a, b) for a in range(3) for b in range(3, 7)], [0, 0, 0, 1, 1, 1, 1], 2))


@pytest.mark.parametrize("L", [2, 5, 8])
def test_er_several_tiles_and_ragged_tail(L):
    # 9,123 edges: 142 full epilogue tiles plus a ragged one (64-edge tiles at this size on 152 SMs)
    assert_pa(graphgen.erdos_renyi(1500, 9123, L, 31 + L))


@pytest.mark.parametrize("options", [None, ALL_HEAVY, ALL_HUB, {"hub_min_wedges": 300}])
def test_chung_lu_every_kernel_variant(options):
    assert_pa(graphgen.chung_lu(2000, 10000, 2.1, 300.0, 5, 77, type_zipf=1.2), options=options)


def test_host_buffers():
    assert_pa(graphgen.erdos_renyi(800, 5000, 4, 3), host_buffers=True)


def test_batch_handle_per_graph():
    graphs = [graphgen.erdos_renyi(60 + 40 * x, 300 + 200 * x, 3, 700 + x) for x in range(4)]
    graphs.insert(2, graph_from_edges(5, [], [0, 1, 2, 0, 1], 3))      # an empty graph inside the batch
    node_off, rp, col, ty = concat_graphs(graphs)
    L = 3
    lay = tg.tg_pa_layout(L)
    h = tg.tg_build_batch(node_off, torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                          torch.as_tensor(ty, device="cuda"), L)
    eoff = tg.tg_edge_offsets(h)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros((len(graphs), lay["global_slots"]), dtype=torch.int64, device="cuda")
    tg.tg_count_position_aware(h, pe, gl)
    assert tg.tg_query_status(h) == 0
    pe_np = pe.cpu().numpy().view(np.uint32).astype(np.int64)
    for x, g in enumerate(graphs):
        pe_o, gl_o = oracle.position_aware(g)
        np.testing.assert_array_equal(gl.cpu().numpy()[x], gl_o)
        np.testing.assert_array_equal(pe_np[eoff[x]:eoff[x + 1]], pe_o)
    h.free()


def test_merges_into_typed_counts_on_the_same_handle():
    """Summing sides and orderings of the position-aware rows gives the rows
    of tg_count (k = 4), and the classes merged by type multiset give its
    totals; tg_count after tg_count_position_aware is unaffected."""
    g = graphgen.chung_lu(30000, 200000, 2.1, 3000.0, 5, 5, type_zipf=1.2)
    L = 5
    lay_pa, lay = tg.tg_pa_layout(L), tg.tg_layout(L, 4)
    h = tg.tg_build(*tg.to_device(g), L)
    pe_pa = torch.zeros((h.m, lay_pa["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl_pa = torch.zeros(lay_pa["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count_position_aware(h, pe_pa, gl_pa)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, pe, gl)
    assert tg.tg_query_status(h) == 0
    h.free()
    pe_pa_np = pe_pa.cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(merge_per_edge(L, pe_pa_np), pe.cpu().numpy().view(np.uint32).astype(np.int64))
    np.testing.assert_array_equal(merge_pa_global(L, gl_pa.cpu().numpy()), gl.cpu().numpy())
