"""Full-size workloads on the GPU: sampled per-edge parity with the oracle
and exact global invariants.

At 20-30 M edges the oracle cannot count every edge, so:
* per-edge rows of a seeded sample -- the heaviest edges by d_i + d_j plus a
  uniform sample -- must equal the oracle's rows exactly;
* the global totals must satisfy, exactly, three untyped degree identities
  (Sigma C(d,2) = 3-paths + 3 triangles; Sigma C(d,3) = stars + paws +
  2 diamonds + 4 cliques; Sigma_E (d_u-1)(d_v-1) - 3 triangles = 4-paths +
  4 C4 + 2 paws + 6 diamonds + 12 cliques), every per-edge orbit sum must be
  |E(H)| times the matching global total (Sec. 6), and the degree identity of
  Sec. 7.1 with S_i excluding j must hold on every edge.
The run is the same launch configuration bench.py times (tg_build +
tg_count, k = 4, device buffers).
"""
import math

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402

GRAPHLET_EDGES = [1, 2, 3, 3, 3, 4, 4, 5, 6]


def multisets(L, K):
    import itertools
    return list(itertools.combinations_with_replacement(range(L), K))


@pytest.fixture(scope="module", params=["cl_large", "sbm_typed"])
def counted(request):
    g = graphgen.workload(request.param)
    L, m = g["L"], g["m"]
    lay = tg.tg_layout(L, 4)
    h = tg.tg_build(*tg.to_device(g), L)
    pe = torch.empty((m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.empty(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, pe, gl)
    st = tg.tg_query_status(h)
    src = torch.empty(m, dtype=torch.int32, device="cuda")
    dst = torch.empty(m, dtype=torch.int32, device="cuda")
    tg.tg_edge_endpoints(h, src, dst)
    h.free()
    yield g, lay, pe, gl.cpu().numpy(), st, src, dst
    del pe


def test_status_clean(counted):
    assert counted[4] == 0, tg.STATUS[counted[4]]


def test_sampled_edges_match_oracle(counted):
    g, lay, pe, _, _, src, dst = counted
    m = g["m"]
    deg = torch.as_tensor(np.diff(g["row_ptr"]), device="cuda")
    cost = deg[src.long()] + deg[dst.long()]
    heavy = torch.topk(cost, 24).indices.cpu().numpy()
    rng = np.random.default_rng(20201029)
    uniform = rng.choice(m, size=300, replace=False)
    ids = np.unique(np.concatenate([heavy, uniform, [0, m - 1]])).astype(np.int64)
    rows_o, _ = oracle.paper_edges(g, ids)
    rows_g = pe[torch.as_tensor(ids, device="cuda")].cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(rows_g, rows_o)


def test_untyped_identities(counted):
    g, lay, _, gl, _, src, dst = counted
    L = g["L"]
    off, size = lay["global_block_offset"], lay["global_block_size"]
    N = [int(gl[off[b]:off[b] + size[b]].sum()) for b in range(9)]
    _, n3p, ntri, np4, nstar, nc4, npaw, ndia, nk4 = N
    d = np.diff(g["row_ptr"]).astype(np.int64)
    assert N[0] == g["m"]
    assert int((d * (d - 1) // 2).sum()) == n3p + 3 * ntri
    assert sum(int(x) for x in (d * (d - 1) * (d - 2) // 6)) == nstar + npaw + 2 * ndia + 4 * nk4
    dd = torch.as_tensor(d, device="cuda")
    s = int(((dd[src.long()] - 1) * (dd[dst.long()] - 1)).sum().item())
    assert s - 3 * ntri == np4 + 4 * nc4 + 2 * npaw + 6 * ndia + 12 * nk4


def test_per_edge_sums_equal_global_totals(counted):
    g, lay, pe, gl, _, src, dst = counted
    L = g["L"]
    P = L * (L + 1) // 2
    ty = torch.as_tensor(g["types"], device="cuda").long()
    key = ty[src.long()] * L + ty[dst.long()]              # ordered endpoint types (p, q)
    sums = torch.zeros((L * L, lay["per_edge_slots"]), dtype=torch.int64, device="cuda")
    chunk = 1 << 22
    for a in range(0, g["m"], chunk):
        rows = pe[a:a + chunk].long() & 0xFFFFFFFF
        sums.index_add_(0, key[a:a + chunk], rows)
    sums = sums.cpu().numpy()
    off = lay["global_block_offset"]
    raw = np.zeros(lay["global_slots"], dtype=np.int64)
    m3, m4 = multisets(L, 3), multisets(L, 4)
    pairs = multisets(L, 2)
    orbit_block = {3: 3, 4: 3, 5: 4, 6: 5, 7: 6, 8: 6, 9: 6, 10: 7, 11: 7, 12: 8}
    for p in range(L):
        for q in range(L):
            row = sums[p * L + q]
            for t in range(L):
                r = m3.index(tuple(sorted((p, q, t))))
                raw[off[1] + r] += row[t]
                raw[off[2] + r] += row[L + t]
            for o in range(3, 13):
                for pi, (t, u) in enumerate(pairs):
                    raw[off[orbit_block[o]] + m4.index(tuple(sorted((p, q, t, u))))] += row[2 * L + (o - 3) * P + pi]
    for b in range(1, 9):
        sl = slice(off[b], off[b] + lay["global_block_size"][b])
        np.testing.assert_array_equal(raw[sl], GRAPHLET_EDGES[b] * gl[sl])


def test_property1_every_edge(counted):
    g, lay, pe, _, _, src, dst = counted
    L = g["L"]
    d = torch.as_tensor(np.diff(g["row_ptr"]), device="cuda")
    chunk = 1 << 22
    for a in range(0, g["m"], chunk):
        rows = pe[a:a + chunk].long()
        lhs = rows[:, :L].sum(1) + 2 * rows[:, L:2 * L].sum(1) + 2
        rhs = d[src[a:a + chunk].long()] + d[dst[a:a + chunk].long()]
        assert torch.equal(lhs, rhs)
