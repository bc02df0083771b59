"""tg_count3_static, the entry point for callers that cannot call cudaMalloc.

Such callers (a service whose device memory all belongs to its own pool,
code running under CUDA-graph capture, loops that cannot afford cudaFree's
device synchronisation) get typed 3-node counts from a file-scope device
array instead of allocations.  This test calls it through the C ABI twice in
a row -- the shared array keeps the previous call's contents, so the second
call checks that what must start at zero is cleared -- and compares both
results with tg_count(k = 3) exactly.  It is collected last so that a run
stopping at the first failure has run every other test already.
"""
import numpy as np
import pytest

import graphgen

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


def static_k3(g):
    rp, col, ty = tg.to_device(g)
    lay = tg.tg_layout(g["L"], 3)
    pe = torch.full((g["m"], lay["per_edge_slots"]), -1, dtype=torch.int32, device="cuda")
    gl = torch.full((lay["global_slots"],), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tg.tg_count3_static(rp, col, ty, g["L"], pe, gl, st)
    torch.cuda.synchronize()
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
