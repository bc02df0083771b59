"""Sparse per-edge output (Sec. 4.6's X_ij): the pairs are exactly the
nonzero entries of the dense rows, edge by edge in slot order."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def sparse(h, k, m):
    row_off = torch.zeros(m + 1, dtype=torch.int64, device="cuda")
    nnz = tg.tg_count_sparse(h, k, row_off)                        # sizing only
    slot = torch.zeros(max(nnz, 1), dtype=torch.int16, device="cuda")
    value = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    gl = torch.zeros(tg.tg_layout(h.L, k)["global_slots"], dtype=torch.int64, device="cuda")
    assert tg.tg_count_sparse(h, k, row_off, slot, value, gl) == nnz
    assert tg.tg_query_status(h) == 0
    return (row_off.cpu().numpy(), slot[:nnz].cpu().numpy().view(np.uint16).astype(np.int64),
            value[:nnz].cpu().numpy().view(np.uint32).astype(np.int64), gl.cpu().numpy())


def expected(dense):
    mask = dense != 0
    row_off = np.concatenate([[0], np.cumsum(mask.sum(1))])
    return row_off, np.nonzero(mask)[1], dense[mask]


@pytest.mark.parametrize("k", [3, 4])
def test_sparse_equals_oracle_nonzeros(k):
    g = graphgen.chung_lu(3000, 20000, 2.1, 900.0, 5, 31, type_zipf=1.2)
    h = tg.tg_build(*tg.to_device(g), g["L"])
    ro, sl, va, gl = sparse(h, k, g["m"])
    pe_o, gl_o = oracle.paper(g, k=k)
    ro_e, sl_e, va_e = expected(pe_o)
    np.testing.assert_array_equal(ro, ro_e)
    np.testing.assert_array_equal(sl, sl_e)
    np.testing.assert_array_equal(va, va_e)
    np.testing.assert_array_equal(gl, gl_o)
    # too small: TG_ERR_TOO_LARGE with the size needed
    small = torch.zeros(max(len(va_e) // 3, 1), dtype=torch.int16, device="cuda")
    smallv = torch.zeros_like(small, dtype=torch.int32)
    with pytest.raises(tg.TGError) as e:
        tg.tg_count_sparse(h, k, None, small, smallv)
    assert e.value.name == "TG_ERR_TOO_LARGE" and e.value.nnz == len(va_e)
    h.free()


def test_sparse_many_windows_equals_dense():
    # cl_mid's dense rows span two windows of the library's 1 GB scratch
    g = graphgen.workload("cl_mid")
    h = tg.tg_build(*tg.to_device(g), g["L"])
    ro, sl, va, gl = sparse(h, 4, g["m"])
    S = tg.tg_layout(g["L"], 4)["per_edge_slots"]
    dense = torch.zeros((g["m"], S), dtype=torch.int32, device="cuda")
    gd = torch.zeros_like(torch.as_tensor(gl), device="cuda")
    tg.tg_count(h, 4, dense, gd)
    h.free()
    d = dense.cpu().numpy().view(np.uint32).astype(np.int64)
    ro_e, sl_e, va_e = expected(d)
    np.testing.assert_array_equal(ro, ro_e)
    np.testing.assert_array_equal(sl, sl_e)
    np.testing.assert_array_equal(va, va_e)
    np.testing.assert_array_equal(gl, gd.cpu().numpy())
    assert 0 < ro[-1] <= g["m"] * S, (ro[-1], g["m"] * S)


def test_sparse_empty_and_errors():
    from oracle_pins import graph_from_edges
    g = graph_from_edges(5, [], [0, 1, 2, 0, 1], 3)                  # nodes, no edges
    h = tg.tg_build(*tg.to_device(g), 3)
    row_off = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert tg.tg_count_sparse(h, 4, row_off) == 0 and int(row_off[0]) == 0
    with pytest.raises(tg.TGError) as e:                             # host arrays are refused
        tg.tg_count_sparse(h, 4, np.zeros(1, np.int64))
    assert e.value.name == "TG_ERR_INVALID_ARG"
    h.free()


def test_sparse_on_a_chunked_batch():
    graphs = [graphgen.erdos_renyi(60 + 20 * x, 300 + 90 * x, 3, 50 + x) for x in range(9)]
    graphs.append(graphgen.chung_lu(1500, 7000, 2.1, 400.0, 3, 77))
    u = graphgen.concat(graphs)
    rp, col, ty = (torch.as_tensor(u[k], device="cuda") for k in ("row_ptr", "col", "types"))
    h = tg.tg_build_batch(u["node_off"], rp, col, ty, 3, options={"cycle_budget_mb": 1})
    ro, sl, va, _ = sparse_batch(h, 4)
    dense = torch.zeros((h.m, tg.tg_layout(3, 4)["per_edge_slots"]), dtype=torch.int32, device="cuda")
    tg.tg_count(h, 4, dense, None)
    ro_e, sl_e, va_e = expected(dense.cpu().numpy().view(np.uint32).astype(np.int64))
    np.testing.assert_array_equal(ro, ro_e)
    np.testing.assert_array_equal(sl, sl_e)
    np.testing.assert_array_equal(va, va_e)
    h.free()


def sparse_batch(h, k):
    row_off = torch.zeros(h.m + 1, dtype=torch.int64, device="cuda")
    nnz = tg.tg_count_sparse(h, k, row_off)
    slot = torch.zeros(max(nnz, 1), dtype=torch.int16, device="cuda")
    value = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
    gl = torch.zeros((h.ngraphs, tg.tg_layout(h.L, k)["global_slots"]), dtype=torch.int64, device="cuda")
    assert tg.tg_count_sparse(h, k, row_off, slot, value, gl) == nnz
    assert tg.tg_query_status(h) == 0
    return (row_off.cpu().numpy(), slot[:nnz].cpu().numpy().view(np.uint16).astype(np.int64),
            value[:nnz].cpu().numpy().view(np.uint32).astype(np.int64), gl.cpu().numpy())
