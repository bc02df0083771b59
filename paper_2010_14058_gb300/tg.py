"""Thin Python binding of libtg (include/tg.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
counting itself: arrays are passed as raw pointers (torch tensors on the GPU
or the CPU, or numpy arrays), streams as ``cudaStream_t`` handles.  If
libtg.so is missing or cannot be loaded, every call raises
:class:`LibraryMissing`; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtg.so")

TG_MAX_TYPES = 8
STATUS = {
    0: "TG_OK", 1: "TG_ERR_INVALID_ARG", 2: "TG_ERR_INVALID_GRAPH", 3: "TG_ERR_TOO_MANY_TYPES",
    4: "TG_ERR_OOM", 5: "TG_ERR_OVERFLOW", 6: "TG_ERR_TIMEOUT", 7: "TG_ERR_CUDA", 8: "TG_ERR_INTERNAL",
    9: "TG_ERR_TOO_LARGE",
}
STATUS_CODE = {v: k for k, v in STATUS.items()}

# every symbol include/tg.h declares: name -> (argtypes, restype)
_i32, _i64, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p


class tg_layout_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("k", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("per_edge_slots", ctypes.c_int64), ("global_slots", ctypes.c_int64),
                ("orbit_offset", ctypes.c_int64 * 13), ("global_block_offset", ctypes.c_int64 * 9),
                ("global_block_size", ctypes.c_int64 * 9), ("graphlet_edges", ctypes.c_int32 * 9)]


class tg_pa_layout_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("per_edge_slots", ctypes.c_int64), ("global_slots", ctypes.c_int64),
                ("block_offset", ctypes.c_int64 * 13), ("global_block_offset", ctypes.c_int64 * 9),
                ("global_block_size", ctypes.c_int64 * 9), ("graphlet_edges", ctypes.c_int32 * 9)]


class tg_edge_typed_layout_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("X", ctypes.c_int32), ("per_edge_slots", ctypes.c_int64),
                ("triangle_offset", ctypes.c_int64), ("global_slots", ctypes.c_int64),
                ("global_block_offset", ctypes.c_int64 * 3), ("global_block_size", ctypes.c_int64 * 3)]


class tg_directed_layout_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("per_edge_slots", ctypes.c_int64), ("global_slots", ctypes.c_int64),
                ("classes", ctypes.c_int64)]


class tg_options(ctypes.Structure):
    _fields_ = [("light_edge_max_degree", ctypes.c_int32), ("light_anchor_max_wedges", ctypes.c_int32),
                ("anchor_table_budget_mb", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("cycle_budget_mb", ctypes.c_int32), ("hub_min_wedges", ctypes.c_int32),
                ("hub_l2_mb", ctypes.c_int32), ("isect_modes", ctypes.c_int32)]


SIGNATURES = {
    "tg_layout": ([_i32, _i32, ctypes.POINTER(tg_layout_t)], _i32),
    "tg_default_options": ([ctypes.POINTER(tg_options)], None),
    "tg_build": ([_i64, _i64, _vp, _vp, _vp, _i32, ctypes.POINTER(tg_options), _vp, ctypes.POINTER(_vp)], _i32),
    "tg_build_batch": ([_i32, _vp, _i64, _i64, _vp, _vp, _vp, _i32, ctypes.POINTER(tg_options), _vp,
                        ctypes.POINTER(_vp)], _i32),
    "tg_free": ([_vp], None),
    "tg_num_nodes": ([_vp], _i64),
    "tg_num_edges": ([_vp], _i64),
    "tg_num_graphs": ([_vp], _i32),
    "tg_num_types": ([_vp], _i32),
    "tg_device_bytes": ([_vp], _i64),
    "tg_edge_endpoints": ([_vp, _vp, _vp], _i32),
    "tg_edge_offsets": ([_vp, _vp], _i32),
    "tg_count": ([_vp, _i32, _vp, _vp, _vp], _i32),
    "tg_count_range": ([_vp, _i32, _i64, _i64, _vp, _vp, _vp], _i32),
    "tg_finalize_global": ([_i32, _i32, _i32, _vp, _vp], _i32),
    "tg_count_batch": ([_vp, _i32, _vp, _vp, _vp], _i32),
    "tg_pa_layout": ([_i32, ctypes.POINTER(tg_pa_layout_t)], _i32),
    "tg_directed_layout": ([_i32, ctypes.POINTER(tg_directed_layout_t)], _i32),
    "tg_directed_class_code": ([_i32, _i64, _vp, _vp], _i32),
    "tg_build_directed": ([_i64, _i64, _vp, _vp, _vp, _i32, ctypes.POINTER(tg_options), _vp, ctypes.POINTER(_vp)],
                          _i32),
    "tg_count_directed3": ([_vp, _vp, _vp, _vp], _i32),
    "tg_edge_typed_layout": ([_i32, _i32, ctypes.POINTER(tg_edge_typed_layout_t)], _i32),
    "tg_build_edge_typed": ([_i64, _i64, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.POINTER(tg_options), _vp,
                             ctypes.POINTER(_vp)], _i32),
    "tg_count_edge_typed3": ([_vp, _vp, _vp, _vp], _i32),
    "tg_count_handles": ([_vp, _i32, _i32, _vp, _vp], _i32),
    "tg_pa_labelling": ([_i32, _i32, _i64, _vp], _i32),
    "tg_pa_slot_class": ([_i32, _i32, _i32, _i64, ctypes.POINTER(_i64)], _i32),
    "tg_count_position_aware": ([_vp, _vp, _vp, _vp], _i32),
    "tg_query_status": ([_vp], _i32),
    "tg_count_sparse": ([_vp, _i32, _vp, _vp, _vp, _i64, ctypes.POINTER(_i64), _vp, _vp], _i32),
    "tg_graphlet_weights": ([_vp, _i32, _vp, _i32, _i64, _vp, _vp, _vp], _i32),
    "tg_status_string": ([_i32], ctypes.c_char_p),
    "tg_last_error": ([], ctypes.c_char_p),
    "tg_last_launch_count": ([_vp], _i64),
    "tg_abi_version": ([], _i32),
    "tg_count3_static": ([_i64, _i64, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "tg_set_timing": ([_vp, _i32], _i32),
    "tg_set_work_counting": ([_vp, _i32], _i32),
    "tg_get_work": ([_vp, _vp, _i32], _i32),
    "tg_get_timing": ([_vp, _i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], _i32),
}


class LibraryMissing(RuntimeError):
    """libtg.so is not built or cannot be loaded (no CPU fallback exists)."""


class TGError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        self.name = STATUS.get(code, f"status {code}")
        self.detail = detail
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Loads libtg.so and declares every entry point; raises LibraryMissing."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise LibraryMissing(f"{path} not found; build it with `python -m paper_2010_14058_gb300.build`")
    try:
        lib = ctypes.CDLL(path)
    except OSError as exc:
        raise LibraryMissing(f"cannot load {path}: {exc}") from exc
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(code: int, where: str) -> None:
    if code != 0:
        raise TGError(code, where, tg_last_error())


def _ptr(a) -> int | None:
    """Raw address of a torch tensor or numpy array (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _options(opts: dict | None):
    if opts is None:
        return None
    o = tg_options()
    load().tg_default_options(ctypes.byref(o))
    for k, v in opts.items():
        setattr(o, k, int(v))
    return ctypes.byref(o)


# ------------------------------------------------------------------ calls

def tg_abi_version() -> int:
    return int(load().tg_abi_version())


def tg_status_string(code: int) -> str:
    return load().tg_status_string(code).decode()


def tg_last_error() -> str:
    """The calling thread's most recent failure text ("" if none)."""
    return load().tg_last_error().decode(errors="replace")


def tg_layout(L: int, k: int = 4) -> dict:
    lay = tg_layout_t()
    _check(load().tg_layout(L, k, ctypes.byref(lay)), "tg_layout")
    return {"L": lay.L, "k": lay.k, "pairs": lay.pairs, "per_edge_slots": lay.per_edge_slots,
            "global_slots": lay.global_slots, "orbit_offset": list(lay.orbit_offset),
            "global_block_offset": list(lay.global_block_offset),
            "global_block_size": list(lay.global_block_size), "graphlet_edges": list(lay.graphlet_edges)}


class Graph:
    """Owner of a tg_graph* handle (freed with tg_free)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None):
            try:
                load().tg_free(self.handle)
            except LibraryMissing:
                pass
            self.handle = None

    @property
    def n(self) -> int:
        return int(load().tg_num_nodes(self.handle))

    @property
    def m(self) -> int:
        return int(load().tg_num_edges(self.handle))

    @property
    def ngraphs(self) -> int:
        return int(load().tg_num_graphs(self.handle))

    @property
    def L(self) -> int:
        return int(load().tg_num_types(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(load().tg_device_bytes(self.handle))

    @property
    def last_launch_count(self) -> int:
        return int(load().tg_last_launch_count(self.handle))


def tg_build(row_ptr, col, node_types, L: int, options: dict | None = None, stream=None) -> Graph:
    n = int(row_ptr.shape[0]) - 1
    nnz = int(col.shape[0])
    h = _vp()
    _check(load().tg_build(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(node_types), L, _options(options),
                           _stream(stream), ctypes.byref(h)), "tg_build")
    return Graph(h.value)


def tg_build_batch(node_off, row_ptr, col, node_types, L: int, options: dict | None = None, stream=None) -> Graph:
    node_off = np.ascontiguousarray(node_off, dtype=np.int64)
    n = int(row_ptr.shape[0]) - 1
    nnz = int(col.shape[0])
    h = _vp()
    _check(load().tg_build_batch(len(node_off) - 1, node_off.ctypes.data, n, nnz, _ptr(row_ptr), _ptr(col),
                                 _ptr(node_types), L, _options(options), _stream(stream), ctypes.byref(h)),
           "tg_build_batch")
    return Graph(h.value)


def tg_build_directed(out_row_ptr, out_col, node_types, L: int, options: dict | None = None, stream=None) -> Graph:
    """Handle of an oriented graph given by its out-neighbour CSR (Sec. 4.8)."""
    n = int(out_row_ptr.shape[0]) - 1
    na = int(out_col.shape[0])
    h = _vp()
    _check(load().tg_build_directed(n, na, _ptr(out_row_ptr), _ptr(out_col), _ptr(node_types), L, _options(options),
                                    _stream(stream), ctypes.byref(h)), "tg_build_directed")
    return Graph(h.value)


def tg_directed_layout(L: int) -> dict:
    lay = tg_directed_layout_t()
    _check(load().tg_directed_layout(L, ctypes.byref(lay)), "tg_directed_layout")
    return {"L": lay.L, "per_edge_slots": lay.per_edge_slots, "global_slots": lay.global_slots,
            "classes": lay.classes}


def tg_directed_class_code(L: int, rank: int) -> tuple:
    """(types of nodes 0,1,2; arc states of pairs (0,1), (0,2), (1,2)) of class `rank`."""
    t = np.zeros(3, dtype=np.int32)
    a = np.zeros(3, dtype=np.int32)
    _check(load().tg_directed_class_code(L, rank, t.ctypes.data, a.ctypes.data), "tg_directed_class_code")
    return tuple(int(x) for x in t), tuple(int(x) for x in a)


def tg_count_directed3(g: Graph, per_edge_out=None, global_out=None, stream=None) -> None:
    _check(load().tg_count_directed3(g.handle, _ptr(per_edge_out), _ptr(global_out), _stream(stream)),
           "tg_count_directed3")


def tg_build_edge_typed(row_ptr, col, node_types, edge_types, L: int, X: int, options: dict | None = None,
                        stream=None) -> Graph:
    """Handle of a graph whose edges carry types too (one per entry of col, the
    same on both entries of an edge; Def. 1's xi)."""
    n = int(row_ptr.shape[0]) - 1
    nnz = int(col.shape[0])
    h = _vp()
    _check(load().tg_build_edge_typed(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(node_types), _ptr(edge_types), L, X,
                                      _options(options), _stream(stream), ctypes.byref(h)), "tg_build_edge_typed")
    return Graph(h.value)


def tg_edge_typed_layout(L: int, X: int) -> dict:
    lay = tg_edge_typed_layout_t()
    _check(load().tg_edge_typed_layout(L, X, ctypes.byref(lay)), "tg_edge_typed_layout")
    return {"L": lay.L, "X": lay.X, "per_edge_slots": lay.per_edge_slots, "triangle_offset": lay.triangle_offset,
            "global_slots": lay.global_slots, "global_block_offset": list(lay.global_block_offset),
            "global_block_size": list(lay.global_block_size)}


def tg_count_edge_typed3(g: Graph, per_edge_out=None, global_out=None, stream=None) -> None:
    _check(load().tg_count_edge_typed3(g.handle, _ptr(per_edge_out), _ptr(global_out), _stream(stream)),
           "tg_count_edge_typed3")


def tg_count_handles(graphs: list, k: int, global_out, stream=None) -> None:
    """Global totals of several handles on one stream, concatenated in order
    (handle h: ngraphs_h x global_slots(L_h, k) values)."""
    arr = (_vp * max(len(graphs), 1))(*[g.handle for g in graphs])
    _check(load().tg_count_handles(arr, len(graphs), k, _ptr(global_out), _stream(stream)), "tg_count_handles")


def tg_free(g: Graph) -> None:
    g.free()


def tg_edge_endpoints(g: Graph, src, dst) -> None:
    _check(load().tg_edge_endpoints(g.handle, _ptr(src), _ptr(dst)), "tg_edge_endpoints")


def tg_edge_offsets(g: Graph) -> np.ndarray:
    out = np.zeros(g.ngraphs + 1, dtype=np.int64)
    _check(load().tg_edge_offsets(g.handle, out.ctypes.data), "tg_edge_offsets")
    return out


def tg_count(g: Graph, k: int, per_edge_out=None, global_out=None, stream=None) -> None:
    _check(load().tg_count(g.handle, k, _ptr(per_edge_out), _ptr(global_out), _stream(stream)), "tg_count")


def tg_count_range(g: Graph, k: int, e_begin: int, e_end: int, per_edge_out=None, global_accum=None,
                   stream=None) -> None:
    _check(load().tg_count_range(g.handle, k, e_begin, e_end, _ptr(per_edge_out), _ptr(global_accum),
                                 _stream(stream)), "tg_count_range")


def tg_finalize_global(L: int, k: int, ngraphs: int, raw: np.ndarray) -> np.ndarray:
    raw = np.ascontiguousarray(raw, dtype=np.int64)
    out = np.zeros_like(raw)
    _check(load().tg_finalize_global(L, k, ngraphs, raw.ctypes.data, out.ctypes.data), "tg_finalize_global")
    return out


def tg_count_sparse(g: Graph, k: int, row_off=None, slot=None, value=None, global_out=None, stream=None) -> int:
    """Sparse per-edge counts (device tensors: row_off int64 [m+1], slot
    int16/uint16, value int32/uint32); returns the number of pairs.  With
    slot = value = None only sizes.  Raises TGError(TG_ERR_TOO_LARGE) when
    the pairs exceed the arrays (the needed size is in .nnz)."""
    cap = 0 if slot is None else int(slot.shape[0])
    if value is not None and int(value.shape[0]) < cap:
        cap = int(value.shape[0])
    nnz = _i64(0)
    code = load().tg_count_sparse(g.handle, k, _ptr(row_off), _ptr(slot), _ptr(value), cap, ctypes.byref(nnz),
                                  _ptr(global_out), _stream(stream))
    if code != 0:
        err = TGError(code, "tg_count_sparse", tg_last_error())
        err.nnz = int(nnz.value)
        raise err
    return int(nnz.value)


def tg_graphlet_weights(g: Graph, k: int, per_edge_rows, block: int, rank: int, weights, degree=None,
                        stream=None) -> None:
    """W (int64 [m]) and, optionally, D (int64 [n]) of the typed graphlet
    (block, rank), from this handle's per-edge rows (device tensors)."""
    _check(load().tg_graphlet_weights(g.handle, k, _ptr(per_edge_rows), block, rank, _ptr(weights), _ptr(degree),
                                      _stream(stream)), "tg_graphlet_weights")


def tg_pa_layout(L: int) -> dict:
    """Position-aware layout (Sec. 5): per-edge blocks O1..O12 and global class blocks."""
    lay = tg_pa_layout_t()
    _check(load().tg_pa_layout(L, ctypes.byref(lay)), "tg_pa_layout")
    return {"L": lay.L, "per_edge_slots": lay.per_edge_slots, "global_slots": lay.global_slots,
            "block_offset": list(lay.block_offset), "global_block_offset": list(lay.global_block_offset),
            "global_block_size": list(lay.global_block_size), "graphlet_edges": list(lay.graphlet_edges)}


def tg_pa_labelling(L: int, block: int, rank: int) -> list:
    """Smallest labelling (types of the numbered shape's nodes) of a position-aware class."""
    out = np.zeros(4, dtype=np.int32)
    _check(load().tg_pa_labelling(L, block, rank, out.ctypes.data), "tg_pa_labelling")
    return out[:2 if block == 0 else (3 if block <= 2 else 4)].tolist()


def tg_pa_slot_class(L: int, phi_lo: int, phi_hi: int, slot: int) -> int:
    """Global slot of the position-aware class that per-edge slot `slot` counts."""
    out = ctypes.c_int64(0)
    _check(load().tg_pa_slot_class(L, phi_lo, phi_hi, slot, ctypes.byref(out)), "tg_pa_slot_class")
    return int(out.value)


def tg_count_position_aware(g: Graph, per_edge_out=None, global_out=None, stream=None) -> None:
    _check(load().tg_count_position_aware(g.handle, _ptr(per_edge_out), _ptr(global_out), _stream(stream)),
           "tg_count_position_aware")


def tg_count_batch(g: Graph, k: int, per_edge_out=None, global_out=None, stream=None) -> None:
    _check(load().tg_count_batch(g.handle, k, _ptr(per_edge_out), _ptr(global_out), _stream(stream)),
           "tg_count_batch")


def tg_query_status(g: Graph) -> int:
    return int(load().tg_query_status(g.handle))


def tg_set_timing(g: Graph, on: bool = True) -> None:
    _check(load().tg_set_timing(g.handle, 1 if on else 0), "tg_set_timing")


def tg_get_timing(g: Graph, max_entries: int = 32) -> dict:
    """{kernel name: (total ms, launches)} accumulated since the last call."""
    names = (ctypes.c_char_p * max_entries)()
    ms = (ctypes.c_double * max_entries)()
    launches = (ctypes.c_int64 * max_entries)()
    n = ctypes.c_int32(0)
    _check(load().tg_get_timing(g.handle, max_entries, names, ms, launches, ctypes.byref(n)), "tg_get_timing")
    return {names[i].decode(): (ms[i], int(launches[i])) for i in range(n.value)}


WORK_SLOTS = {"clique_probes": 0, "clique_searches": 1, "clique_big_probes": 2, "hub_wait_cycles": 3,
              "hub_fill_cycles": 4, "hub_read_cycles": 5, "hub_walk_clear_cycles": 6, "hub_zero_clear_cycles": 7,
              "hub_wedges": 8, "hub_slot_updates": 9}


def tg_set_work_counting(g: "Graph", on: bool = True) -> None:
    """Enables the diagnostic work counters of the counting kernels."""
    _check(load().tg_set_work_counting(g.handle, 1 if on else 0), "tg_set_work_counting")


def tg_get_work(g: "Graph") -> dict:
    """Work counters accumulated since the last call (then cleared)."""
    import numpy as np
    out = np.zeros(16, dtype=np.int64)
    _check(load().tg_get_work(g.handle, out.ctypes.data, 16), "tg_get_work")
    return {name: int(out[k]) for name, k in WORK_SLOTS.items()}


def tg_count3_static(row_ptr, col, node_types, L: int, per_edge_out=None, global_out=None, device_status=None,
                     stream=None) -> None:
    """Allocation-free typed 3-node counts for callers that cannot call
    cudaMalloc (see include/tg.h); device tensors only, rows sorted by id."""
    n = int(row_ptr.shape[0]) - 1
    nnz = int(col.shape[0])
    _check(load().tg_count3_static(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(node_types), L, _ptr(per_edge_out),
                                   _ptr(global_out), _ptr(device_status), _stream(stream)), "tg_count3_static")
