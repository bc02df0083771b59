"""Exact typed-graphlet counting on one GB300 (sm_103a).

The computation lives in libtg.so (CUDA, C ABI in include/tg.h); this
package is its Python binding plus device-memory plumbing through PyTorch.

    import paper_2010_14058_gb300 as tg
    g = tg.tg_build(row_ptr, col, types, L)          # tensors or arrays
    tg.tg_count(g, 4, per_edge_out, global_out)      # uint32 [m,S], int64 [G]

``count`` below does the same for a graph given as host arrays.
"""
from __future__ import annotations

from .tg import (Graph, LibraryMissing, STATUS, STATUS_CODE, TGError, TG_MAX_TYPES, load, tg_abi_version,
                 tg_build, tg_build_batch, tg_count, tg_count3_static, tg_count_batch, tg_count_position_aware,
                 tg_count_range, tg_count_sparse, tg_edge_endpoints, tg_edge_offsets, tg_finalize_global, tg_free,
                 tg_get_timing, tg_graphlet_weights, tg_last_error, tg_layout, tg_pa_labelling, tg_pa_layout,
                 tg_pa_slot_class, tg_query_status, tg_set_timing, tg_status_string,
                 tg_set_work_counting, tg_get_work, tg_build_directed, tg_count_directed3, tg_directed_layout,
                 tg_directed_class_code, tg_count_handles, tg_build_edge_typed, tg_edge_typed_layout,
                 tg_count_edge_typed3)

__all__ = ["Graph", "LibraryMissing", "STATUS", "STATUS_CODE", "TGError", "TG_MAX_TYPES", "load", "tg_abi_version",
           "tg_build", "tg_build_batch", "tg_count", "tg_count3_static", "tg_count_batch", "tg_count_position_aware",
           "tg_count_range", "tg_count_sparse", "tg_edge_endpoints", "tg_edge_offsets", "tg_finalize_global",
           "tg_free", "tg_get_timing", "tg_graphlet_weights", "tg_last_error", "tg_layout", "tg_pa_labelling",
           "tg_pa_layout", "tg_pa_slot_class", "tg_query_status", "tg_set_timing", "tg_status_string",
           "tg_set_work_counting", "tg_get_work", "tg_build_directed", "tg_count_directed3", "tg_directed_layout",
           "tg_directed_class_code", "tg_count_handles", "tg_build_edge_typed", "tg_edge_typed_layout",
           "tg_count_edge_typed3",
           "to_device", "count"]


def to_device(graph: dict, device="cuda"):
    """(row_ptr int64, col int32, types uint8) as device tensors."""
    import torch
    rp = torch.as_tensor(graph["row_ptr"], dtype=torch.int64).to(device)
    col = torch.as_tensor(graph["col"], dtype=torch.int32).to(device)
    ty = torch.as_tensor(graph["types"], dtype=torch.uint8).to(device)
    return rp, col, ty


def count(graph: dict, k: int = 4, per_edge: bool = True, device="cuda", options=None, check=True):
    """Builds and counts one graph on the GPU.

    Returns (per_edge uint32 tensor [m, S] or None, global int64 tensor [G]),
    both on `device`.  Raises TGError if the device status word reports an
    error (check=True).
    """
    import torch
    rp, col, ty = to_device(graph, device)
    g = tg_build(rp, col, ty, graph["L"], options=options)
    lay = tg_layout(graph["L"], k)
    pe = torch.empty((g.m, lay["per_edge_slots"]), dtype=torch.int32, device=device) if per_edge else None
    gl = torch.empty(lay["global_slots"], dtype=torch.int64, device=device)
    tg_count(g, k, pe, gl)
    if check:
        st = tg_query_status(g)
        if st != 0:
            raise TGError(st, "device status")
    g.free()
    return pe, gl
