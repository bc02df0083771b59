"""Edge-typed 3-node graphlets on the GPU (tg_build_edge_typed,
tg_count_edge_typed3), bit-exact against the CPU oracle's Alg. 1 route
split by edge type (oracle.edge_typed3, pinned in test_oracle_edge_typed.py):
per-edge rows and global totals on small and mid-size graphs, every
intersection method, host buffers; with one edge type the rows are the typed
3-node rows of tg_count; invalid edge types are rejected.
"""
import numpy as np
import pytest

import graphgen
import oracle
from oracle_pins import edge_types_for, graph_from_edges, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def gpu_edge_typed(g, xi, X, options=None, host=False):
    L = g["L"]
    lay = tg.tg_edge_typed_layout(L, X)
    if host:
        h = tg.tg_build_edge_typed(np.ascontiguousarray(g["row_ptr"], dtype=np.int64),
                                   np.ascontiguousarray(g["col"], dtype=np.int32),
                                   np.ascontiguousarray(g["types"], dtype=np.uint8), np.ascontiguousarray(xi), L, X,
                                   options=options)
        pe = np.zeros((h.m, lay["per_edge_slots"]), dtype=np.uint32)
        gl = np.zeros(lay["global_slots"], dtype=np.int64)
        tg.tg_count_edge_typed3(h, pe, gl)
        st = tg.tg_query_status(h)
        h.free()
        return pe.astype(np.int64), gl, st
    rp, col, ty = tg.to_device(g)
    h = tg.tg_build_edge_typed(rp, col, ty, torch.as_tensor(xi, device="cuda"), L, X, options=options)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count_edge_typed3(h, pe, gl)
    st = tg.tg_query_status(h)
    h.free()
    return pe.cpu().numpy().view(np.uint32).astype(np.int64), gl.cpu().numpy(), st


def assert_parity(g, X, seed, options=None, host=False):
    xi = edge_types_for(g, X, seed)
    pe, gl, st = gpu_edge_typed(g, xi, X, options, host)
    assert st == 0, tg.STATUS[st]
    pe_o, gl_o = oracle.edge_typed3(g, xi, X)
    np.testing.assert_array_equal(pe, pe_o)
    np.testing.assert_array_equal(gl, gl_o)


@pytest.mark.parametrize("seed", range(8))
def test_small_random_graphs(seed):
    L, X = [1, 2, 3, 5][seed % 4], [1, 2, 3, 4][(seed // 2) % 4]
    assert_parity(random_graph(14 + seed, 0.4, L, 300 + seed), X, 400 + seed)


@pytest.mark.parametrize("X", [2, 4])
def test_chung_lu(X):
    assert_parity(graphgen.chung_lu(3000, 20000, 2.1, 600.0, 4, 23), X, 50 + X)


def test_erdos_renyi_several_tiles():
    assert_parity(graphgen.erdos_renyi(2000, 12000, 3, 7), 3, 61)


@pytest.mark.parametrize("options", [{"isect_modes": 0b01010101}, {"isect_modes": 0b10101010}])
def test_intersection_methods(options):
    assert_parity(graphgen.chung_lu(2000, 15000, 2.1, 700.0, 5, 9), 3, 71, options=options)


def test_host_buffers():
    assert_parity(graphgen.chung_lu(1500, 8000, 2.1, 300.0, 3, 11), 2, 81, host=True)


def test_one_edge_type_is_the_typed_count():
    g = graphgen.chung_lu(2500, 15000, 2.1, 500.0, 5, 13)
    xi = np.zeros(len(g["col"]), dtype=np.uint8)
    pe, gl, st = gpu_edge_typed(g, xi, 1)
    assert st == 0
    h = tg.tg_build(*tg.to_device(g), g["L"])
    lay = tg.tg_layout(g["L"], 3)
    pt = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gt = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 3, pt, gt)
    h.free()
    np.testing.assert_array_equal(pe, pt.cpu().numpy().view(np.uint32).astype(np.int64))
    np.testing.assert_array_equal(gl, gt.cpu().numpy())


def test_invalid_edge_types_are_rejected():
    g = graph_from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 2)], [0, 1, 0, 1], 2)
    xi = edge_types_for(g, 2, 5)
    bad = xi.copy()
    bad[int(g["row_ptr"][1])] ^= 1                      # one entry of an edge of row 1 disagrees
    for types, X in ((bad, 2), (np.full_like(xi, 3), 3 - 1)):
        with pytest.raises(tg.TGError) as e:
            tg.tg_build_edge_typed(*tg.to_device(g), torch.as_tensor(types, device="cuda"), g["L"], X)
        assert e.value.name == "TG_ERR_INVALID_GRAPH"
    with pytest.raises(tg.TGError) as e:
        tg.tg_build_edge_typed(*tg.to_device(g), torch.as_tensor(xi, device="cuda"), g["L"], 5)
    assert e.value.name == "TG_ERR_TOO_MANY_TYPES"
    h = tg.tg_build(*tg.to_device(g), g["L"])
    with pytest.raises(tg.TGError) as e:
        tg.tg_count_edge_typed3(h, None, None)
    assert e.value.name == "TG_ERR_INVALID_ARG"
    h.free()
