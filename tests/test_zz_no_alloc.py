"""tg_count3_static, the entry point for callers that cannot call cudaMalloc.

Such callers (a service whose device memory all belongs to its own pool,
code running under CUDA-graph capture, loops that cannot afford cudaFree's
device synchronisation) get typed 3-node counts from a file-scope device
array instead of allocations.  This test calls it through the C ABI twice in
a row -- the shared array keeps the previous call's contents, so the second
call checks that what must start at zero is cleared -- and compares both
results with tg_count(k = 3) and with the CPU oracle (Alg. 1 and Cor. 1-3)
exactly.  Rows that are not symmetric must be reported, not counted.  It is
collected last so that a run stopping at the first failure has run every
other test already.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def reference_k3(g):
    h = tg.tg_build(*tg.to_device(g), g["L"])
    lay = tg.tg_layout(g["L"], 3)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 3, pe, gl)
    assert tg.tg_query_status(h) == 0
    h.free()
    return pe, gl


def static_k3(g, expect_ok=True):
    rp, col, ty = tg.to_device(g)
    lay = tg.tg_layout(g["L"], 3)
    pe = torch.full((g["m"], lay["per_edge_slots"]), -1, dtype=torch.int32, device="cuda")
    gl = torch.full((lay["global_slots"],), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tg.tg_count3_static(rp, col, ty, g["L"], pe, gl, st)
    torch.cuda.synchronize()
    if expect_ok:
        assert int(st.item()) == 0
    return pe, gl


@pytest.mark.parametrize("graph", [
    lambda: graphgen.chung_lu(5000, 40000, 2.1, 900.0, 5, 123, type_zipf=1.2),
    lambda: graphgen.erdos_renyi(3000, 20000, 8, 7),
])
def test_static_matches_tg_count_on_two_calls(graph):
    g = graph()
    pe_ref, gl_ref = reference_k3(g)
    for _ in range(2):
        pe, gl = static_k3(g)
        assert torch.equal(pe, pe_ref)
        assert torch.equal(gl, gl_ref)


@pytest.mark.parametrize("graph", [
    lambda: graphgen.chung_lu(3000, 25000, 2.1, 700.0, 8, 41, type_zipf=1.2),   # a hub row of ~700 entries
    lambda: graphgen.erdos_renyi(1500, 9123, 3, 17),
    lambda: graphgen.erdos_renyi(40, 0, 2, 3),                                 # no edges
])
def test_static_matches_oracle_on_two_calls(graph):
    g = graph()
    pe_o, gl_o = oracle.paper(g, k=3)
    for _ in range(2):
        pe, gl = static_k3(g)
        np.testing.assert_array_equal(pe.cpu().numpy().view(np.uint32).astype(np.int64), pe_o)
        np.testing.assert_array_equal(gl.cpu().numpy(), gl_o)


def one_sided(n, rows, L=2):
    rp = np.zeros(n + 1, dtype=np.int64)
    for u, r in enumerate(rows):
        rp[u + 1] = rp[u] + len(r)
    col = np.array([v for r in rows for v in r], dtype=np.int32)
    return {"n": n, "m": len(col) // 2, "L": L, "row_ptr": rp, "col": col,
            "types": np.arange(n, dtype=np.uint8) % L}


@pytest.mark.parametrize("rows", [
    [[1], [], [0]],                      # 0 -> 1 and 2 -> 0: two entries, upper count 1 = m
    [[1, 2], [0], [3], [0, 2]],          # 0 -> 2 and 3 -> 0 one-sided, upper count 3 = m
    [[1], [2], [3], [0]],                # a directed 4-cycle
])
def test_static_reports_one_sided_rows(rows):
    g = one_sided(len(rows), rows)
    assert oracle.validate(g) != 0        # the oracle rejects them too
    rp, col, ty = tg.to_device(g)
    lay = tg.tg_layout(g["L"], 3)
    pe = torch.zeros((max(g["m"], 1), lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tg.tg_count3_static(rp, col, ty, g["L"], pe, gl, st)
    torch.cuda.synchronize()
    assert int(st.item()) != 0
    # the next valid call is unaffected by the rejected one
    ok = graphgen.erdos_renyi(60, 150, 2, 9)
    pe_o, gl_o = oracle.paper(ok, k=3)
    pe2, gl2 = static_k3(ok)
    np.testing.assert_array_equal(pe2.cpu().numpy().view(np.uint32).astype(np.int64), pe_o)
    np.testing.assert_array_equal(gl2.cpu().numpy(), gl_o)


def test_static_rejects_too_many_nodes():
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    ty = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(tg.TGError) as e:
        tg.tg_count3_static(rp, col, ty, 2)
    assert e.value.name == "TG_ERR_TOO_LARGE"


def test_static_reports_unsorted_rows():
    g = graphgen.erdos_renyi(50, 200, 3, 5)
    col = g["col"].copy()
    a, b = int(g["row_ptr"][7]), int(g["row_ptr"][8])
    col[a:b] = col[a:b][::-1].copy()          # row 7 in descending order
    rp, _, ty = tg.to_device(g)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tg.tg_count3_static(rp, torch.as_tensor(col, device="cuda"), ty, g["L"], None, None, st)
    torch.cuda.synchronize()
    assert int(st.item()) != 0
    # a valid call afterwards is unaffected
    pe_ref, gl_ref = reference_k3(g)
    pe, gl = static_k3(g)
    assert torch.equal(pe, pe_ref) and torch.equal(gl, gl_ref)
