"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
bring results back as int64 numpy arrays."""
from __future__ import annotations

import numpy as np


def gpu_count(graph: dict, k: int = 4, options=None, per_edge: bool = True, host_buffers: bool = False):
    """(per_edge int64 [m,S] or None, global int64 [G], status code)."""
    import torch

    import paper_2010_14058_gb300 as tg
    L = graph["L"]
    lay = tg.tg_layout(L, k)
    if host_buffers:
        g = tg.tg_build(np.ascontiguousarray(graph["row_ptr"], dtype=np.int64),
                        np.ascontiguousarray(graph["col"], dtype=np.int32),
                        np.ascontiguousarray(graph["types"], dtype=np.uint8), L, options=options)
        pe = np.zeros((g.m, lay["per_edge_slots"]), dtype=np.uint32) if per_edge else None
        gl = np.zeros(lay["global_slots"], dtype=np.int64)
        tg.tg_count(g, k, pe, gl)
        st = tg.tg_query_status(g)
        g.free()
        return (pe.astype(np.int64) if pe is not None else None), gl, st
    rp, col, ty = tg.to_device(graph)
    g = tg.tg_build(rp, col, ty, L, options=options)
    pe = torch.zeros((g.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda") if per_edge else None
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(g, k, pe, gl)
    st = tg.tg_query_status(g)
    g.free()
    pe_np = pe.cpu().numpy().view(np.uint32).astype(np.int64) if pe is not None else None
    return pe_np, gl.cpu().numpy(), st


def concat_graphs(graphs):
    """Block-diagonal union: (node_off, row_ptr, col, types)."""
    node_off = [0]
    rps, cols, tys = [], [], []
    base_n, base_nnz = 0, 0
    for g in graphs:
        rps.append(g["row_ptr"][:-1] + base_nnz)
        cols.append(g["col"].astype(np.int64) + base_n)
        tys.append(g["types"])
        base_n += g["n"]
        base_nnz += int(g["row_ptr"][-1])
        node_off.append(base_n)
    rp = np.concatenate(rps + [np.array([base_nnz])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    ty = np.concatenate(tys).astype(np.uint8)
    return np.array(node_off, dtype=np.int64), rp, col, ty
