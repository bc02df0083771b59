"""CPU oracle for typed-graphlet counting -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The GPU library neither imports
nor links it, and no product code path may fall back to it.

Three independent routes over the same output layout (see oracle.c):

* :func:`paper`  -- Alg. 1-3 and Lemmas 1-4 of the paper, per edge.
* :func:`table3` -- each orbit from its Table 3 set-builder definition.
* :func:`brute`  -- all 3- and 4-node subsets, classified by induced degrees.

:func:`weights` gives the typed-graphlet weighted graph W and degree D of
Alg. 5 by direct enumeration; :func:`position_aware` the position-aware
typed counts of Sec. 5 (Def. 8), per edge and global; :func:`directed3`
and :func:`directed3_brute` the directed typed 3-node graphlets of Sec. 4.8
(oriented graphs given by their out-neighbour CSR); :func:`edge_typed3`
and :func:`edge_typed3_brute` the typed 3-node graphlets of a graph whose
edges also carry types (Def. 1's xi, classes by Defs. 4-5).

All counts are exact int64.  Parity with these is the acceptance bar for
the GPU path (bit-exact).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "invalid graph", 3: "out of memory",
          4: "inconsistent counts (a global sum not divisible by |E(H)|, a negative count or a rank out of range)"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP when available) into liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base[:4] + ["-fopenmp"] + base[4:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_SIGS = {
    "oracle_per_edge_slots": ("i32 i32", "i64"),
    "oracle_global_slots": ("i32 i32", "i64"),
    "oracle_pair_index": ("i32 i32 i32", "i64"),
    "oracle_multiset_rank": ("i32 i32 vp", "i64"),
    "oracle_paper": ("i64 vp vp vp i32 i32 vp vp i32", "i32"),
    "oracle_paper_edges": ("i64 vp vp vp i32 i32 vp i64 vp vp i32", "i32"),
    "oracle_table3": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_brute": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_edges": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_validate": ("i64 vp vp vp i32", "i32"),
    "oracle_weights": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_pa_per_edge_slots": ("i32", "i64"),
    "oracle_pa_block_size": ("i32 i32", "i64"),
    "oracle_pa_global_slots": ("i32", "i64"),
    "oracle_pa_class": ("i32 i32 vp", "i64"),
    "oracle_position_aware": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_position_aware_brute": ("i64 vp vp vp i32 vp", "i32"),
    "oracle_max_threads": ("", "i32"),
    "oracle_directed_classes": ("i32", "i64"),
    "oracle_directed_global_slots": ("i32", "i64"),
    "oracle_directed_class": ("i32 vp vp", "i64"),
    "oracle_directed3": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_directed3_brute": ("i64 vp vp vp i32 vp vp", "i32"),
    "oracle_directed_edges": ("i64 vp vp vp i32 vp vp vp", "i32"),
    "oracle_et_per_edge_slots": ("i32 i32", "i64"),
    "oracle_et_global_slots": ("i32 i32", "i64"),
    "oracle_edge_typed3": ("i64 vp vp vp vp i32 i32 vp vp", "i32"),
    "oracle_edge_typed3_brute": ("i64 vp vp vp vp i32 i32 vp vp", "i32"),
    "oracle_graph_open": ("i64 vp vp vp i32 vp", "vp"),
    "oracle_graph_close": ("vp", "i32"),
    "oracle_graph_paper_edges": ("vp i32 vp i64 vp vp vp i32", "i32"),
}
_CT = {"i64": ctypes.c_int64, "i32": ctypes.c_int32, "vp": ctypes.c_void_p}


def open_library(path: str):
    """Load an oracle build (the default one, or a variant a test compiled)."""
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = [_CT[a] for a in args.split()]
        f.restype = None if name == "oracle_graph_close" else _CT[res]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = open_library(_LIB_PATH)
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _args(g):
    rp = np.ascontiguousarray(g["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(g["col"], dtype=np.int32)
    ty = np.ascontiguousarray(g["types"], dtype=np.uint8)
    return rp, col, ty


def _check(rc):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, f"error {rc}"))


def per_edge_slots(L: int, k: int = 4, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_per_edge_slots(L, k))


def global_slots(L: int, k: int = 4, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_global_slots(L, k))


def pair_index(L: int, t: int, tp: int, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_pair_index(L, t, tp))


def multiset_rank(L: int, types, lib=None) -> int:
    lib = lib or _load()
    a = np.ascontiguousarray(types, dtype=np.int32)
    return int(lib.oracle_multiset_rank(L, len(a), _p(a)))


def max_threads(lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_max_threads())


def validate(g, lib=None) -> int:
    lib = lib or _load()
    rp, col, ty = _args(g)
    return int(lib.oracle_validate(g["n"], _p(rp), _p(col), _p(ty), g["L"]))


def edges(g, lib=None):
    """(src, dst) int64 arrays in edge-id order, src < dst."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    m = int(rp[-1]) // 2
    s = np.empty(m, dtype=np.int64)
    d = np.empty(m, dtype=np.int64)
    _check(lib.oracle_edges(g["n"], _p(rp), _p(col), _p(ty), g["L"], _p(s), _p(d)))
    return s, d


def paper(g, k: int = 4, per_edge: bool = True, nthreads: int = 0, lib=None):
    """Alg. 1-3 + Lemmas 1-4 on every edge -> (per_edge int64 [m,S] or None, global int64 [G])."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    m = int(rp[-1]) // 2
    pe = np.zeros((m, per_edge_slots(L, k, lib)), dtype=np.int64) if per_edge else None
    gl = np.zeros(global_slots(L, k, lib), dtype=np.int64)
    _check(lib.oracle_paper(g["n"], _p(rp), _p(col), _p(ty), L, k, _p(pe), _p(gl), nthreads))
    return pe, gl


def paper_edges(g, edge_ids, k: int = 4, nthreads: int = 0, lib=None):
    """Alg. 1-3 + Lemmas on selected edges -> (rows int64 [len,S], raw per-graphlet sums int64 [G])."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
    pe = np.zeros((len(ids), per_edge_slots(L, k, lib)), dtype=np.int64)
    sums = np.zeros(global_slots(L, k, lib), dtype=np.int64)
    _check(lib.oracle_paper_edges(g["n"], _p(rp), _p(col), _p(ty), L, k, _p(ids), len(ids),
                                      _p(pe), _p(sums), nthreads))
    return pe, sums


def table3(g, lib=None):
    """Every orbit from Table 3's definitions -> (per_edge int64 [m,S], global int64 [G])."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    m = int(rp[-1]) // 2
    pe = np.zeros((m, per_edge_slots(L, 4, lib)), dtype=np.int64)
    gl = np.zeros(global_slots(L, 4, lib), dtype=np.int64)
    _check(lib.oracle_table3(g["n"], _p(rp), _p(col), _p(ty), L, _p(pe), _p(gl)))
    return pe, gl


def brute(g, lib=None):
    """All 3- and 4-subsets -> (per_edge int64 [m,S], global int64 [G]).  Small n only."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    m = int(rp[-1]) // 2
    pe = np.zeros((m, per_edge_slots(L, 4, lib)), dtype=np.int64)
    gl = np.zeros(global_slots(L, 4, lib), dtype=np.int64)
    _check(lib.oracle_brute(g["n"], _p(rp), _p(col), _p(ty), L, _p(pe), _p(gl)))
    return pe, gl


def weights(g, lib=None):
    """Alg. 5's W and D for every typed graphlet -> (W int64 [m,G], D int64 [n,G]).

    Column s is global slot s (block offset + type-multiset rank).  Small n only."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    m = int(rp[-1]) // 2
    w = np.zeros((m, global_slots(L, 4, lib)), dtype=np.int64)
    d = np.zeros((g["n"], global_slots(L, 4, lib)), dtype=np.int64)
    _check(lib.oracle_weights(g["n"], _p(rp), _p(col), _p(ty), L, _p(w), _p(d)))
    return w, d


def pa_per_edge_slots(L: int, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_pa_per_edge_slots(L))


def pa_block_sizes(L: int, lib=None) -> list:
    """Number of position-aware typed graphlets of each global block (Def. 8)."""
    lib = lib or _load()
    return [int(lib.oracle_pa_block_size(L, b)) for b in range(9)]


def pa_class(L: int, block: int, labelling, lib=None) -> int:
    """Rank, within its block, of the class of a labelling of the numbered shape."""
    lib = lib or _load()
    a = np.ascontiguousarray(labelling, dtype=np.int32)
    return int(lib.oracle_pa_class(L, block, _p(a)))


def position_aware(g, per_edge: bool = True, lib=None):
    """Sec. 5 per edge and global -> (per_edge int64 [m,S_pa] or None, global int64 [G_pa])."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    L = g["L"]
    m = int(rp[-1]) // 2
    if not 1 <= L <= 8:
        raise OracleError(ERRORS[1])
    pe = np.zeros((m, pa_per_edge_slots(L, lib)), dtype=np.int64) if per_edge else None
    gl = np.zeros(int(lib.oracle_pa_global_slots(L)), dtype=np.int64)
    _check(lib.oracle_position_aware(g["n"], _p(rp), _p(col), _p(ty), L, _p(pe), _p(gl)))
    return pe, gl


def position_aware_brute(g, lib=None):
    """Position-aware global counts from every node set of the graph.  Small n only."""
    lib = lib or _load()
    rp, col, ty = _args(g)
    if not 1 <= g["L"] <= 8:
        raise OracleError(ERRORS[1])
    gl = np.zeros(int(lib.oracle_pa_global_slots(g["L"])), dtype=np.int64)
    _check(lib.oracle_position_aware_brute(g["n"], _p(rp), _p(col), _p(ty), g["L"], _p(gl)))
    return gl


# ---------------------------------------------------- directed (Sec. 4.8)

def _dargs(g):
    rp = np.ascontiguousarray(g["out_row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(g["out_col"], dtype=np.int32)
    ty = np.ascontiguousarray(g["types"], dtype=np.uint8)
    return rp, col, ty


def directed_classes(L: int, lib=None) -> int:
    """Number of connected directed typed 3-node graphlets (isomorphism classes)."""
    lib = lib or _load()
    return int(lib.oracle_directed_classes(L))


def directed_global_slots(L: int, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_directed_global_slots(L))


def directed_class(L: int, types, arcs, lib=None) -> int:
    """Class rank of the configuration (types of nodes 0,1,2; arc states of
    pairs (0,1), (0,2), (1,2): 0 none, 1 lower -> higher, 2 higher -> lower),
    -1 when it is not connected."""
    lib = lib or _load()
    t = np.ascontiguousarray(types, dtype=np.int32)
    a = np.ascontiguousarray(arcs, dtype=np.int32)
    return int(lib.oracle_directed_class(L, _p(t), _p(a)))


def directed_edges(g, lib=None):
    """(src, dst, orientation) of the underlying undirected edges in edge-id
    order (src < dst); orientation 0: src -> dst, 1: dst -> src."""
    lib = lib or _load()
    rp, col, ty = _dargs(g)
    m = int(rp[-1])
    s = np.empty(m, dtype=np.int64)
    d = np.empty(m, dtype=np.int64)
    o = np.empty(m, dtype=np.int8)
    _check(lib.oracle_directed_edges(g["n"], _p(rp), _p(col), _p(ty), g["L"], _p(s), _p(d), _p(o)))
    return s, d, o


def _directed(fn, g, per_edge, lib):
    rp, col, ty = _dargs(g)
    L = g["L"]
    m = int(rp[-1])
    pe = np.zeros((m, 8 * L), dtype=np.int64) if per_edge else None
    gl = np.zeros(directed_global_slots(L, lib), dtype=np.int64)
    _check(fn(g["n"], _p(rp), _p(col), _p(ty), L, _p(pe), _p(gl)))
    return pe, gl


def directed3(g, per_edge: bool = True, lib=None):
    """Alg. 1 with the typed sets split by direction (Sec. 4.8) ->
    (per_edge int64 [m, 8L] or None, global int64 [L^2 + classes])."""
    lib = lib or _load()
    return _directed(lib.oracle_directed3, g, per_edge, lib)


def directed3_brute(g, per_edge: bool = True, lib=None):
    """Every 3-node subset of a small oriented graph -> same layout as directed3."""
    lib = lib or _load()
    return _directed(lib.oracle_directed3_brute, g, per_edge, lib)


# ------------------------------------------- edge types (Def. 1, Defs. 4-5)

def edge_typed_per_edge_slots(L: int, X: int, lib=None) -> int:
    """L X path slots, then L X(X+1)/2 triangle slots."""
    lib = lib or _load()
    return int(lib.oracle_et_per_edge_slots(L, X))


def edge_typed_global_slots(L: int, X: int, lib=None) -> int:
    lib = lib or _load()
    return int(lib.oracle_et_global_slots(L, X))


def _edge_typed(fn, g, edge_types, X, per_edge, lib):
    rp, col, ty = _args(g)
    xi = np.ascontiguousarray(edge_types, dtype=np.uint8)
    L = g["L"]
    pe = np.zeros((g["m"], edge_typed_per_edge_slots(L, X, lib)), dtype=np.int64) if per_edge else None
    gl = np.zeros(edge_typed_global_slots(L, X, lib), dtype=np.int64)
    _check(fn(g["n"], _p(rp), _p(col), _p(ty), _p(xi), L, X, _p(pe), _p(gl)))
    return pe, gl


def edge_typed3(g, edge_types, X: int, per_edge: bool = True, lib=None):
    """Alg. 1 with the typed sets split by edge type -> (per_edge int64
    [m, L X + L X(X+1)/2] or None, global int64 [edges, 3-paths, triangles
    by node-type and edge-type multisets]); edge_types: one per entry of col."""
    lib = lib or _load()
    return _edge_typed(lib.oracle_edge_typed3, g, edge_types, X, per_edge, lib)


def edge_typed3_brute(g, edge_types, X: int, per_edge: bool = True, lib=None):
    """Every 3-node subset of a small graph -> same layout as edge_typed3."""
    lib = lib or _load()
    return _edge_typed(lib.oracle_edge_typed3_brute, g, edge_types, X, per_edge, lib)


class OpenGraph:
    """A graph opened once (validated, rows sorted) for several
    :meth:`paper_edges` calls -- the per-edge work of Alg. 1-3 + Lemmas on
    edge samples without re-opening the graph each time.  Used to time the
    oracle; the counts are those of :func:`paper_edges`."""

    def __init__(self, g, lib=None):
        self.lib = lib or _load()
        self.rp, self.col, self.ty = _args(g)            # kept alive: the handle points into them
        self.L = g["L"]
        self.m = int(self.rp[-1]) // 2
        st = ctypes.c_int32(0)
        self.h = self.lib.oracle_graph_open(g["n"], _p(self.rp), _p(self.col), _p(self.ty), self.L,
                                            ctypes.addressof(st))
        if not self.h:
            raise OracleError(ERRORS.get(st.value, f"error {st.value}"))

    def paper_edges(self, edge_ids, k: int = 4, nthreads: int = 0, per_edge: bool = False, times: bool = False):
        """-> (rows int64 [len,S] or None, raw sums int64 [G], seconds per edge or None)."""
        ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
        pe = np.zeros((len(ids), per_edge_slots(self.L, k, self.lib)), dtype=np.int64) if per_edge else None
        sums = np.zeros(global_slots(self.L, k, self.lib), dtype=np.int64)
        sec = np.zeros(len(ids), dtype=np.float64) if times else None
        _check(self.lib.oracle_graph_paper_edges(self.h, k, _p(ids), len(ids), _p(pe), _p(sums), _p(sec), nthreads))
        return pe, sums, sec

    def close(self):
        if getattr(self, "h", None):
            self.lib.oracle_graph_close(self.h)
            self.h = None

    def __del__(self):
        self.close()
