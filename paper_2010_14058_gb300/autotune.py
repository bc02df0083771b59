"""Autotuner for the launch knobs of libtg.

The knobs never change a count (tg_options: "results never depend on
them"); they pick which kernel variant takes which part of the work:

  light_edge_max_degree    heavy-edge threshold of the 4-clique pass: edges
                           whose triangle set T is larger go to one CTA per
                           edge instead of one warp per edge
  light_anchor_max_wedges  wedge anchors with at most this many wedges are
                           one warp each (shared-memory hash per warp)
  hub_min_wedges           anchors with more wedges are counted by the whole
                           GPU against an L2-resident node table (the others
                           by one CTA each with a shared-memory hash) -- the
                           table-versus-hash choice per degree bucket
  ctas_per_sm              resident CTAs per SM of the orbit epilogue
  hub_l2_mb                hub node tables counted together (more hubs per
                           group against L2 pressure)
  isect_bucket_0 .. 3      typed set intersection per bucket of the shorter
                           segment's length ([1,32) [32,128) [128,512)
                           [512,inf)): 1 binary search, 2 warp-wide merge,
                           3 a dependent-load count picks per pair; packed
                           into tg_options.isect_modes

tune() measures tg_count (CUDA events on the given stream) for one graph or
batch handle per candidate, by coordinate descent from the defaults, and
checks that every candidate produces the same global totals.  Results are
cached in a JSON file keyed by a coarse signature of the workload (L and
power-of-two buckets of nodes, edges, maximum degree and graph count), so
workloads of the same class reuse the choice.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import tg

SPACE = {
    "light_edge_max_degree": [32, 64, 128, 256],
    "light_anchor_max_wedges": [64, 256, 1024, 2048],
    "hub_min_wedges": [1 << 14, 1 << 16, 1 << 18, 1 << 20],
    "ctas_per_sm": [2, 3, 4],
    "hub_l2_mb": [96, 192, 256],
    "isect_bucket_0": [1, 2, 3],
    "isect_bucket_1": [1, 2, 3],
    "isect_bucket_2": [1, 2, 3],
    "isect_bucket_3": [1, 2, 3],
}
DEFAULTS = {"light_edge_max_degree": 256, "light_anchor_max_wedges": 64, "hub_min_wedges": 1 << 14, "ctas_per_sm": 3,
            "hub_l2_mb": 192, "isect_bucket_0": 1, "isect_bucket_1": 1, "isect_bucket_2": 1, "isect_bucket_3": 1}


def library_options(options: dict) -> dict:
    """tg_options fields of a knob setting: the per-bucket intersection modes
    packed into isect_modes (two bits per bucket)."""
    out = {k: v for k, v in options.items() if not k.startswith("isect_bucket_")}
    if len(out) < len(options):
        modes = 0
        for b in range(4):
            modes |= (int(options.get(f"isect_bucket_{b}", 1)) & 3) << (2 * b)
        out["isect_modes"] = modes
    return out

CACHE_PATH = os.environ.get("TG_AUTOTUNE_CACHE", os.path.join(os.path.dirname(__file__), ".autotune.json"))
_lock = threading.Lock()


def _bucket(x: int) -> int:
    return int(math.log2(max(int(x), 1)))


def signature(n: int, m: int, max_degree: int, L: int, ngraphs: int = 1) -> str:
    """Coarse class of a workload: L and log2 buckets of its sizes."""
    return f"L{L}-n{_bucket(n)}-m{_bucket(m)}-d{_bucket(max_degree)}-g{_bucket(ngraphs)}"


def load_cache(path: str = CACHE_PATH) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def cached(sig: str, path: str = CACHE_PATH) -> dict | None:
    """Tuned options of a workload class, or None."""
    return load_cache(path).get(sig, {}).get("options")


def _store(sig: str, entry: dict, path: str) -> None:
    with _lock:
        c = load_cache(path)
        c[sig] = entry
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time_count(build, options: dict, L: int, G: int, ngraphs: int, stream, reps: int):
    """Median tg_count time (ms) of a handle built with `options`, and its totals."""
    import torch
    h = build(options)
    gl = torch.zeros((ngraphs, G), dtype=torch.int64, device="cuda")
    times = []
    with torch.cuda.stream(stream):
        tg.tg_count(h, 4, None, gl, stream=stream)                # warm-up (first count prepares)
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tg.tg_count(h, 4, None, gl, stream=stream)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
    st = tg.tg_query_status(h)
    h.free()
    if st != 0:
        raise tg.TGError(st, "autotune count")
    return float(np.median(times)), gl.cpu().numpy()


def tune(row_ptr, col, types, L: int, node_off=None, space: dict | None = None, reps: int = 2,
         rounds: int = 1, path: str = CACHE_PATH, stream=None, store: bool = True) -> dict:
    """Tunes the knobs for one workload (device tensors of a CSR, or a
    block-diagonal batch when node_off is given) and caches the result.
    Returns {"options", "ms", "default_ms", "signature", "trials"}."""
    import torch
    space = space or SPACE
    stream = stream or torch.cuda.current_stream()
    n = int(row_ptr.shape[0]) - 1
    m = int(col.shape[0]) // 2
    deg = row_ptr[1:] - row_ptr[:-1]
    dmax = int(deg.max().item()) if n > 0 else 0
    ngraphs = 1 if node_off is None else len(node_off) - 1
    sig = signature(n, m, dmax, L, ngraphs)
    G = tg.tg_layout(L, 4)["global_slots"]

    def build(options):
        opts = library_options(options)
        if node_off is None:
            return tg.tg_build(row_ptr, col, types, L, options=opts, stream=stream)
        return tg.tg_build_batch(node_off, row_ptr, col, types, L, options=opts, stream=stream)

    best = {k: DEFAULTS[k] for k in space}
    best_ms, ref = _time_count(build, best, L, G, ngraphs, stream, reps)
    default_ms = best_ms
    trials = [{"options": dict(best), "ms": round(best_ms, 3)}]
    for _ in range(rounds):
        for knob, values in space.items():
            start = best[knob]                       # measured already (as part of `best`)
            for v in values:
                if v == start:
                    continue
                cand = dict(best)
                cand[knob] = v
                ms, tot = _time_count(build, cand, L, G, ngraphs, stream, reps)
                if not np.array_equal(tot, ref):
                    raise RuntimeError(f"autotune: options {cand} changed the counts")
                trials.append({"options": dict(cand), "ms": round(ms, 3)})
                if ms < best_ms:
                    best, best_ms = cand, ms
    entry = {"options": library_options(best), "knobs": best, "ms": round(best_ms, 3), "default_ms": round(default_ms, 3), "signature": sig,
             "n": n, "m": m, "max_degree": dmax, "ngraphs": ngraphs, "trials": trials}
    if store:
        _store(sig, entry, path)
    return entry
