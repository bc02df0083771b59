"""GPU path (through the C ABI) vs the CPU oracle: bit-exact counts.

Per-edge rows (uint32) and global totals (int64) must equal the oracle's
exactly on every graph: tiny graphs against brute force, seeded ER /
Chung-Lu / SBM graphs that span many tiles and a ragged last tile, graphs
that force every kernel variant (warp and CTA per edge, shared-memory and
global T lists, warp and CTA wedge anchors), the 3-node mode, edge ranges,
batches, host buffers, and the error paths.
"""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import concat_graphs, gpu_count
from oracle_pins import graph_from_edges, random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402

# options that route every edge and every anchor through the CTA variants
ALL_HEAVY = {"light_edge_max_degree": 1, "light_anchor_max_wedges": 1}
# ... and every anchor with more than one wedge through the whole-GPU hub pass
ALL_HUB = {"light_edge_max_degree": 1, "light_anchor_max_wedges": 1, "hub_min_wedges": 1}


def assert_parity(g, k=4, options=None, reference="paper"):
    pe, gl, st = gpu_count(g, k=k, options=options)
    assert st == 0, tg.STATUS[st]
    if reference == "brute":
        pe_o, gl_o = oracle.brute(g)
        if k == 3:
            L = g["L"]
            pe_o = pe_o[:, :2 * L]
            gl_o = gl_o[:oracle.global_slots(L, 3)]
    else:
        pe_o, gl_o = oracle.paper(g, k=k)
    np.testing.assert_array_equal(pe, pe_o)
    np.testing.assert_array_equal(gl, gl_o)


@pytest.mark.parametrize("seed", range(24))
def test_tiny_graphs_vs_brute_force(seed):
    n = 5 + seed % 11
    p = [0.3, 0.5, 0.7, 0.95][seed % 4]
    L = [1, 2, 3, 4, 5, 8][seed % 6]
    assert_parity(random_graph(n, p, L, 9000 + seed), reference="brute")


@pytest.mark.parametrize("options", [ALL_HEAVY, ALL_HUB])
@pytest.mark.parametrize("seed", range(6))
def test_tiny_graphs_all_cta_variants(seed, options):
    g = random_graph(9 + seed, 0.6, [2, 3, 8][seed % 3], 9100 + seed)
    assert_parity(g, options=options, reference="brute")


def test_degenerate_graphs():
    # no edges, isolated nodes, one edge, a path, a star, a clique, K_{3,4}
    assert_parity(graph_from_edges(4, [], [0, 1, 2, 0], 3))
    assert_parity(graph_from_edges(1, [], [0], 1))
    assert_parity(graph_from_edges(6, [(2, 5)], [0, 1, 2, 0, 1, 2], 3))
    assert_parity(graph_from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4)], [0, 1, 0, 1, 0], 2))
    assert_parity(graph_from_edges(7, [(0, x) for x in range(1, 7)], [1, 0, 1, 2, 0, 2, 2], 3))
    assert_parity(graph_from_edges(8, [(a, b) for a in range(8) for b in range(a + 1, 8)], [0, 1, 2, 3, 0, 1, 2, 3], 4))
    assert_parity(graph_from_edges(7, [(a, b) for a in range(3) for b in range(3, 7)], [0, 0, 0, 1, 1, 1, 1], 2))
    for opt in (ALL_HEAVY, ALL_HUB):
        assert_parity(graph_from_edges(8, [(a, b) for a in range(8) for b in range(a + 1, 8)], [0, 1, 2, 3, 0, 1, 2, 3], 4),
                      options=opt)
        assert_parity(graph_from_edges(7, [(a, b) for a in range(3) for b in range(3, 7)], [0, 0, 0, 1, 1, 1, 1], 2),
                      options=opt)


def test_large_tiles_and_ragged_tail():
    # 60,001 edges: 2,048-edge epilogue tiles at this size (29 full, one ragged)
    assert_parity(graphgen.erdos_renyi(4000, 60001, 3, 93), k=3)
    assert_parity(graphgen.erdos_renyi(4000, 60001, 3, 93))


@pytest.mark.parametrize("L", [1, 2, 5, 8])
def test_er_several_tiles_and_ragged_tail(L):
    # 9,123 edges: 142 full epilogue tiles plus a ragged one (64-edge tiles at this size on 152 SMs)
    g = graphgen.erdos_renyi(1500, 9123, L, 31 + L)
    assert_parity(g)


def test_er_small_workload():
    assert_parity(graphgen.workload("er_small"))


def test_er_small_workload_k3():
    assert_parity(graphgen.workload("er_small"), k=3)


@pytest.mark.parametrize("options", [None, ALL_HEAVY, ALL_HUB, {"light_edge_max_degree": 16, "light_anchor_max_wedges": 8},
                                     {"hub_min_wedges": 300}, {"hub_min_wedges": 2000, "hub_l2_mb": 1}])
def test_chung_lu_with_hubs(options):
    # hubs route edges and anchors through both variants
    g = graphgen.chung_lu(4000, 30000, 2.1, 1200.0, 5, 77, type_zipf=1.2)
    assert_parity(g, options=options)


@pytest.mark.parametrize("budget_mb", [1, 12288])
def test_heavy_anchors_with_few_dense_tables(budget_mb):
    # 506 heavy anchors and no hubs; 64 of them have more wedges than the
    # shared-memory hash holds and go to dense node tables.  A 1 MB table
    # budget gives 10 tables (100 KB each), so 10 CTAs take those 64 and the
    # rest of the grid (two CTAs per SM) only hash anchors; 12 GB gives every
    # CTA a table.
    g = graphgen.chung_lu(5000, 40000, 2.1, 900.0, 5, 19)
    assert_parity(g, options={"hub_min_wedges": 1 << 30, "anchor_table_budget_mb": budget_mb})


# typed set intersection forced to one method in every length bucket
ALL_BINARY = {"isect_modes": 0b01010101}
ALL_MERGE = {"isect_modes": 0b10101010}


@pytest.mark.parametrize("options", [ALL_BINARY, ALL_MERGE])
def test_intersection_methods(options):
    # hubs give long typed segments on both sides (merge windows advance on
    # either side, equal last entries, ragged windows), leaves short ones
    assert_parity(graphgen.chung_lu(4000, 30000, 2.1, 1200.0, 5, 77, type_zipf=1.2), options=options)
    assert_parity(graphgen.erdos_renyi(300, 20000, 2, 78), options=options)            # dense: |A| ~ |B|
    for seed in range(4):
        assert_parity(random_graph(12 + seed, 0.7, 2, 9300 + seed), options=options, reference="brute")


def test_global_t_list_path():
    # edge (0,1) has |T| = 9000 > the shared-memory T list of a CTA
    a = 9000
    edges = [(0, 1)] + [(0, 2 + x) for x in range(a)] + [(1, 2 + x) for x in range(a)]
    edges += [(2 + x, 2 + x + 1) for x in range(0, 200, 2)]
    rng = np.random.default_rng(5)
    types = rng.integers(0, 3, a + 2)
    assert_parity(graph_from_edges(a + 2, edges, types, 3))


def test_sbm_small():
    aff = np.full((4, 4), 1.0)
    np.fill_diagonal(aff, 0.05)
    g = graphgen.sbm([500, 300, 150, 50], aff, 20000, 12)
    assert_parity(g)


def test_host_buffers_match_device_buffers():
    g = graphgen.erdos_renyi(800, 5000, 4, 3)
    pe_d, gl_d, st_d = gpu_count(g)
    pe_h, gl_h, st_h = gpu_count(g, host_buffers=True)
    assert st_d == 0 and st_h == 0
    np.testing.assert_array_equal(pe_d, pe_h)
    np.testing.assert_array_equal(gl_d, gl_h)


def test_edge_endpoints_and_ranges():
    g = graphgen.chung_lu(3000, 20000, 2.2, 800.0, 3, 8)
    src, dst = oracle.edges(g)
    h = tg.tg_build(*tg.to_device(g), g["L"])
    s = torch.zeros(h.m, dtype=torch.int32, device="cuda")
    d = torch.zeros(h.m, dtype=torch.int32, device="cuda")
    tg.tg_edge_endpoints(h, s, d)
    np.testing.assert_array_equal(s.cpu().numpy(), src)
    np.testing.assert_array_equal(d.cpu().numpy(), dst)
    lay = tg.tg_layout(g["L"], 4)
    full = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    glob = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, full, glob)
    raw = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    cuts = [0, 1, 777, 5000, 5001, 19999, h.m]
    for a, b in zip(cuts[:-1], cuts[1:]):
        part = torch.zeros((b - a, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
        tg.tg_count_range(h, 4, a, b, part, raw)
        assert torch.equal(part, full[a:b])
    assert tg.tg_query_status(h) == 0
    np.testing.assert_array_equal(tg.tg_finalize_global(g["L"], 4, 1, raw.cpu().numpy()), glob.cpu().numpy())
    h.free()


@pytest.mark.parametrize("options", [None, {"cycle_budget_mb": 1}, {"cycle_budget_mb": 1, "hub_min_wedges": 257}])
def test_batch_equals_separate_graphs(options):
    # cycle_budget_mb = 1 splits the batch into many chunks of whole graphs
    graphs = [graphgen.erdos_renyi(50 + 30 * x, 200 + 150 * x, 3, 400 + x) for x in range(7)]
    graphs.append(graphgen.chung_lu(2000, 9000, 2.1, 500.0, 3, 9))
    graphs.insert(3, graph_from_edges(5, [], [0, 1, 2, 0, 1], 3))      # an empty graph inside the batch
    graphs += [graphgen.erdos_renyi(300, 1500, 3, 600 + x) for x in range(12)]
    node_off, rp, col, ty = concat_graphs(graphs)
    L = 3
    lay = tg.tg_layout(L, 4)
    h = tg.tg_build_batch(node_off, torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                          torch.as_tensor(ty, device="cuda"), L, options=options)
    assert h.ngraphs == len(graphs)
    eoff = tg.tg_edge_offsets(h)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros((len(graphs), lay["global_slots"]), dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        tg.tg_count_batch(h, 4, pe, gl, stream=stream)
        first = gl.clone()
        pe.zero_()
        gl.zero_()
        tg.tg_count_batch(h, 4, pe, gl, stream=stream)        # CUDA-graph replay
    stream.synchronize()
    assert tg.tg_query_status(h) == 0
    assert torch.equal(first, gl)
    pe_np = pe.cpu().numpy().view(np.uint32).astype(np.int64)
    for x, g in enumerate(graphs):
        pe_o, gl_o = oracle.paper(g)
        np.testing.assert_array_equal(gl.cpu().numpy()[x], gl_o)
        np.testing.assert_array_equal(pe_np[eoff[x]:eoff[x + 1]], pe_o)
    # plain count of the same batch handle gives the same numbers
    gl2 = torch.zeros_like(gl)
    tg.tg_count(h, 4, None, gl2)
    assert torch.equal(gl2, gl)
    # ranges that cut across graphs (and chunks) give the same rows and sums
    raw = torch.zeros_like(gl)
    cuts = [0, 7, int(eoff[4]) + 3, int(eoff[9]) - 1, int(eoff[15]), h.m]
    for a, b in zip(cuts[:-1], cuts[1:]):
        part = torch.zeros((b - a, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
        tg.tg_count_range(h, 4, a, b, part, raw)
        assert torch.equal(part, pe[a:b])
    np.testing.assert_array_equal(tg.tg_finalize_global(L, 4, len(graphs), raw.cpu().numpy().ravel()),
                                  gl.cpu().numpy().ravel())
    assert tg.tg_query_status(h) == 0
    h.free()


def test_invalid_graphs_are_rejected():
    ok = graph_from_edges(3, [(0, 1), (1, 2)], [0, 1, 0], 2)
    cases = [
        dict(ok, types=np.array([0, 2, 0], dtype=np.uint8)),                                     # type >= L
        dict(ok, row_ptr=np.array([0, 2, 3, 4]), col=np.array([0, 1, 0, 1], dtype=np.int32)),    # self-loop
        dict(ok, row_ptr=np.array([0, 1, 2, 2]), col=np.array([1, 2], dtype=np.int32)),          # one-sided
        dict(ok, row_ptr=np.array([0, 2, 4, 4]), col=np.array([1, 1, 0, 0], dtype=np.int32)),    # repeated
        dict(ok, col=np.array([1, 0, 5, 1], dtype=np.int32)),                                    # id out of range
    ]
    for bad in cases:
        with pytest.raises(tg.TGError) as e:
            tg.tg_build(*tg.to_device(bad), bad["L"])
        assert e.value.name == "TG_ERR_INVALID_GRAPH"
    with pytest.raises(tg.TGError) as e:
        tg.tg_build(*tg.to_device(ok), 9)
    assert e.value.name == "TG_ERR_TOO_MANY_TYPES"
    # a cross-graph edge in a batch
    g2 = graph_from_edges(4, [(0, 1), (1, 3), (2, 3)], [0, 1, 0, 1], 2)
    with pytest.raises(tg.TGError) as e:
        tg.tg_build_batch(np.array([0, 2, 4]), *tg.to_device(g2), 2)
    assert e.value.name == "TG_ERR_INVALID_GRAPH"


def test_repeated_counts_are_identical():
    g = graphgen.chung_lu(3000, 15000, 2.1, 600.0, 4, 21)
    h = tg.tg_build(*tg.to_device(g), g["L"])
    lay = tg.tg_layout(g["L"], 4)
    outs = []
    for _ in range(3):
        pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
        gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
        tg.tg_count(h, 4, pe, gl)
        outs.append((pe, gl))
    assert tg.tg_query_status(h) == 0
    for pe, gl in outs[1:]:
        assert torch.equal(pe, outs[0][0]) and torch.equal(gl, outs[0][1])
    h.free()


def test_big_t_with_long_neighbour_lists():
    # edge (0, 1) has |T| = 360 (one CTA) and every triangle node has ~1,100
    # neighbours of higher priority (hubs padded with private leaves), all
    # scanned warp-wide
    nt, nh, leaves = 360, 1100, 760
    T = np.arange(2, 2 + nt)
    H = np.arange(2 + nt, 2 + nt + nh)
    first_leaf = 2 + nt + nh
    n = first_leaf + nh * leaves
    eu = [np.array([0]), np.zeros(nt, np.int64), np.ones(nt, np.int64), T[:-1], np.repeat(T, nh),
          np.repeat(H, leaves)]
    ev = [np.array([1]), T, T, T[1:], np.tile(H, nt), first_leaf + np.arange(nh * leaves)]
    eu, ev = np.concatenate(eu).astype(np.int32), np.concatenate(ev).astype(np.int32)
    order = np.lexsort((ev, eu))
    types = np.random.default_rng(8).integers(0, 3, n).astype(np.uint8)
    g = graphgen.csr_from_edges(n, eu[order], ev[order], types, 3, "long N+ lists")
    pe, gl, st = gpu_count(g)
    assert st == 0, tg.STATUS[st]
    ids = np.array([0, 1, 2, 3, 400, 700, 721, 722, 1000, 5000])   # (0,1), (0,t), (1,t), (t,t+1), (t,h)
    rows_o, _ = oracle.paper_edges(g, ids)
    np.testing.assert_array_equal(pe[ids], rows_o)
    assert pe[0, 3:6].sum() == nt                           # the triangle slots of edge (0, 1)


def test_degree_above_65535_uses_wide_sums():
    # a hub of degree 70,060 (70,000 leaves and a 60-node random cluster that
    # is also joined to it): the per-edge sums take the 64-bit path
    leaves, nc = 70_000, 60
    hub, c0 = 0, 1
    l0 = c0 + nc
    rng = np.random.default_rng(61)
    cl = [(c0 + a, c0 + b) for a in range(nc) for b in range(a + 1, nc) if rng.random() < 0.3]
    eu = np.concatenate([np.zeros(nc + leaves, np.int64), np.array([a for a, _ in cl])])
    ev = np.concatenate([np.arange(c0, c0 + nc), np.arange(l0, l0 + leaves), np.array([b for _, b in cl])])
    order = np.lexsort((ev, eu))
    n = l0 + leaves
    g = graphgen.csr_from_edges(n, eu[order].astype(np.int32), ev[order].astype(np.int32),
                                rng.integers(0, 3, n).astype(np.uint8), 3, "hub of degree 70,060")
    assert np.diff(g["row_ptr"]).max() >= 1 << 16
    pe, gl, st = gpu_count(g)
    assert st == 0, tg.STATUS[st]
    ids = np.array([0, 5, 59, 60, 61, 5000, 70_059, nc + leaves, nc + leaves + 7, g["m"] - 1])
    rows_o, _ = oracle.paper_edges(g, ids)
    np.testing.assert_array_equal(pe[ids], rows_o)


def test_count_handles_list_form():
    # several handles the caller holds (single graphs of different L and a
    # batch), counted on one stream into one concatenated totals array
    singles = [graphgen.erdos_renyi(300, 1500, 3, 501), graphgen.chung_lu(2000, 9000, 2.1, 400.0, 5, 502)]
    parts = [graphgen.erdos_renyi(80 + 20 * x, 300 + 100 * x, 2, 510 + x) for x in range(3)]
    node_off, rp, col, ty = concat_graphs(parts)
    handles = [tg.tg_build(*tg.to_device(g), g["L"]) for g in singles]
    handles.append(tg.tg_build_batch(node_off, torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                                     torch.as_tensor(ty, device="cuda"), 2))
    want = [oracle.paper(g)[1] for g in singles] + [oracle.paper(g)[1] for g in parts]
    total = sum(len(w) for w in want)
    for host in (False, True):
        out = np.zeros(total, dtype=np.int64) if host else torch.zeros(total, dtype=torch.int64, device="cuda")
        tg.tg_count_handles(handles, 4, out)
        got = out if host else out.cpu().numpy()
        np.testing.assert_array_equal(got, np.concatenate(want))
    assert all(tg.tg_query_status(h) == 0 for h in handles)
    for h in handles:
        h.free()
