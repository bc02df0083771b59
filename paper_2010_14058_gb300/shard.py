"""One graph's edges counted by several ranks (one GPU per rank).

Edges are independent once the graph is fixed (the per-edge counts of
Problem 1 read the graph only), so rank r counts the contiguous edge-id
range edge_ranges(m, world, weights)[r] with tg_count_range into a raw
per-graphlet accumulator (sums over edges of the per-edge orbit values,
Sec. 6).  The one exchange is a sum of that accumulator -- G(L) int64
values -- over the ranks; tg_finalize_global then divides each block by the
number of edges of its graphlet.  Per-edge rows stay on the rank that
counted them.

count_sharded takes the range counter as a parameter: by default the GPU
path (tg_count_range on a handle built on this rank's device); any other
counter with the same contract may be passed in.
"""
from __future__ import annotations

import numpy as np

from . import tg


def edge_weights(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Work estimate d_u + d_v of every edge, in edge-id order (edges (u, v),
    u < v, in lexicographic order)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(deg.size, dtype=np.int64), deg)
    up = col > rows
    u, v = rows[up], col[up]
    order = np.lexsort((v, u))
    return (deg[u] + deg[v])[order]


def edge_ranges(m: int, world: int, weights: np.ndarray | None = None) -> list:
    """Contiguous [begin, end) edge ranges, one per rank, with about equal
    total weight (equal edge counts without weights)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if weights is None:
        cuts = [m * r // world for r in range(world + 1)]
    else:
        w = np.asarray(weights, dtype=np.float64)
        if w.shape != (m,):
            raise ValueError("weights must have one entry per edge")
        c = np.concatenate([[0.0], np.cumsum(w)])
        cuts = [int(np.searchsorted(c, c[-1] * r / world, side="left")) for r in range(world)] + [m]
        cuts[0] = 0
        for r in range(1, world + 1):
            cuts[r] = max(cuts[r], cuts[r - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gpu_range_counter(handle: tg.Graph, k: int = 4, per_edge_out=None, stream=None):
    """Range counter on this rank's GPU: raw per-graphlet sums of [b, e) as
    int64 numpy (per-edge rows into per_edge_out[b:e] when given)."""
    import torch

    def count(b: int, e: int) -> np.ndarray:
        G = tg.tg_layout(handle.L, k)["global_slots"]
        raw = torch.zeros(G, dtype=torch.int64, device="cuda")
        rows = None if per_edge_out is None else per_edge_out[b:e]
        tg.tg_count_range(handle, k, b, e, rows, raw, stream=stream)
        st = tg.tg_query_status(handle)
        if st != 0:
            raise tg.TGError(st, "tg_count_range")
        return raw.cpu().numpy()
    return count


def count_sharded(count_range, L: int, m: int, rank: int, world: int, k: int = 4, weights=None,
                  group=None) -> np.ndarray:
    """Global typed totals of one graph whose edges are split over `world`
    ranks: this rank counts its range, the raw sums are added over the
    process group, and every rank returns the finalised totals."""
    import torch
    import torch.distributed as dist
    b, e = edge_ranges(m, world, weights)[rank]
    raw = np.ascontiguousarray(count_range(b, e), dtype=np.int64)
    if world > 1:
        t = torch.from_numpy(raw.copy())
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        raw = t.cpu().numpy()
    return tg.tg_finalize_global(L, k, 1, raw)
