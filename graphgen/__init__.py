"""Seeded synthetic typed graphs shared by the CPU oracle and the GPU path.

This module holds no part of the counting method.  It draws the inputs:
simple undirected graphs (as symmetric CSR with rows sorted by neighbour id)
and node types, from the families the paper uses for its synthetic
experiments (Erdos-Renyi, Chung-Lu, Sec. 8.1 and 8.5) plus a stochastic block
model and ego networks.  Every draw is a function of its seed only
(SplitMix64 seeding xoshiro256**, see graphgen.c).

A graph is a dict: n, m, L, row_ptr (int64[n+1]), col (int32[2m]),
types (uint8[n]), name.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# Fixed seeds of the five standard workloads: 20201029 + k.
SEED_BASE = 20201029


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:5] + ["-fopenmp"] + base[5:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            vp = ctypes.c_void_p
            lib.gg_types_uniform.argtypes = [i64, i32, u64, vp]
            lib.gg_types_zipf.argtypes = [i64, i32, dbl, u64, vp]
            lib.gg_er_edges.argtypes = [i64, i64, u64, vp, vp]
            lib.gg_er_edges.restype = i64
            lib.gg_chung_lu_edges.argtypes = [i64, i64, dbl, dbl, u64, vp, vp]
            lib.gg_chung_lu_weights.argtypes = [i64, dbl, dbl, dbl, vp]
            lib.gg_sbm_edges.argtypes = [i32, vp, vp, i64, u64, vp, vp, vp]
            lib.gg_edges_to_csr.argtypes = [i64, i64, vp, vp, vp, vp]
            lib.gg_ego_network.argtypes = [i64, vp, vp, i32, i64, i64, u64, vp, vp, vp, vp, vp, i64]
            lib.gg_ego_network.restype = i64
            lib.gg_degree_proportional_node.argtypes = [i64, vp, u64]
            lib.gg_degree_proportional_node.restype = i32
            lib.gg_ego_batch_sizes.argtypes = [i64, vp, vp, i64, i64, i64, i64, u64, vp, vp]
            lib.gg_ego_batch_fill.argtypes = [i64, vp, vp, i64, i64, i64, i64, u64, i32, vp, vp, vp, vp, vp]
            lib.gg_unit_from_seed.argtypes = [u64]
            lib.gg_unit_from_seed.restype = dbl
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc < 0:
        raise RuntimeError(f"graphgen: {what} failed (code {rc})")


def csr_from_edges(n: int, eu: np.ndarray, ev: np.ndarray, types: np.ndarray, L: int, name: str) -> dict:
    lib = _load()
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    m = int(eu.shape[0])
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(2 * m, dtype=np.int32)
    _check(lib.gg_edges_to_csr(n, m, _p(eu), _p(ev), _p(row_ptr), _p(col)), "edges_to_csr")
    return {"n": int(n), "m": m, "L": int(L), "row_ptr": row_ptr, "col": col,
            "types": np.ascontiguousarray(types, dtype=np.uint8), "name": name}


def uniform_types(n: int, L: int, seed: int) -> np.ndarray:
    t = np.empty(n, dtype=np.uint8)
    _check(_load().gg_types_uniform(n, L, seed, _p(t)), "types_uniform")
    return t


def zipf_types(n: int, L: int, s: float, seed: int) -> np.ndarray:
    t = np.empty(n, dtype=np.uint8)
    _check(_load().gg_types_zipf(n, L, s, seed, _p(t)), "types_zipf")
    return t


def edge_types(g: dict, X: int, seed: int) -> np.ndarray:
    """One seeded edge type in [0, X) per entry of col, the same on both
    entries of an edge: SplitMix64 (Steele, Lea and Flood 2014) of the pair
    key min(u, v) * n + max(u, v), offset by the seed."""
    rp, n = g["row_ptr"], int(g["n"])
    col = g["col"].astype(np.uint64)
    rows = np.repeat(np.arange(n, dtype=np.uint64), np.diff(rp))
    gamma = 0x9E3779B97F4A7C15
    offset = np.uint64(((seed + 1) * gamma) & 0xFFFFFFFFFFFFFFFF)
    z = np.minimum(rows, col) * np.uint64(n) + np.maximum(rows, col) + offset
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return (z % np.uint64(X)).astype(np.uint8)


def erdos_renyi(n: int, m: int, L: int, seed: int) -> dict:
    """G(n, m): m distinct pairs uniform over all C(n,2); types uniform over L."""
    lib = _load()
    eu = np.empty(m, dtype=np.int32)
    ev = np.empty(m, dtype=np.int32)
    _check(lib.gg_er_edges(n, m, seed, _p(eu), _p(ev)), "er_edges")
    types = uniform_types(n, L, seed ^ 0x7E57)
    return csr_from_edges(n, eu, ev, types, L, f"ER(n={n},m={m},L={L},seed={seed})")


def chung_lu(n: int, m: int, gamma: float, wmax: float, L: int, seed: int,
             type_zipf: float | None = None) -> dict:
    """Chung-Lu graph with exactly m edges; types Zipf(type_zipf) or uniform."""
    lib = _load()
    eu = np.empty(m, dtype=np.int32)
    ev = np.empty(m, dtype=np.int32)
    _check(lib.gg_chung_lu_edges(n, m, gamma, wmax, seed, _p(eu), _p(ev)), "chung_lu_edges")
    if type_zipf is None:
        types = uniform_types(n, L, seed ^ 0x7E57)
    else:
        types = zipf_types(n, L, type_zipf, seed ^ 0x7E57)
    return csr_from_edges(n, eu, ev, types, L,
                          f"CL(n={n},m={m},gamma={gamma},wmax={wmax},L={L},seed={seed})")


def sbm(sizes, affinity, m: int, seed: int) -> dict:
    """Stochastic block model; block b carries node type b."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    B = int(sizes.shape[0])
    aff = np.ascontiguousarray(affinity, dtype=np.float64).reshape(B, B)
    n = int(sizes.sum())
    eu = np.empty(m, dtype=np.int32)
    ev = np.empty(m, dtype=np.int32)
    types = np.empty(n, dtype=np.uint8)
    _check(lib.gg_sbm_edges(B, _p(sizes), _p(aff), m, seed, _p(eu), _p(ev), _p(types)), "sbm_edges")
    return csr_from_edges(n, eu, ev, types, B, f"SBM(sizes={sizes.tolist()},m={m},seed={seed})")


def ego_networks(parent: dict, count: int, n_min: int, n_max: int, m_cap: int, L: int,
                 seed: int, first: int = 0) -> list:
    """Ego networks `first .. first+count-1` of a parent graph.

    Graph g: u ~ U(0,1) from seed+g, target size round(n_min * (n_max/n_min)^u),
    seed node drawn in proportion to degree, breadth-first ball, induced
    subgraph, at most m_cap edges (uniform subset), types uniform over L.
    """
    lib = _load()
    n_p = parent["n"]
    rp, col = parent["row_ptr"], parent["col"]
    mark = np.full(n_p, -1, dtype=np.int32)
    out = []
    for g in range(first, first + count):
        s = seed + g
        u = lib.gg_unit_from_seed(s)
        n_t = int(round(n_min * (n_max / n_min) ** u))
        sn = lib.gg_degree_proportional_node(n_p, _p(rp), s ^ 0x5EED)
        nodes = np.empty(n_t, dtype=np.int32)
        n_out = ctypes.c_int64(0)
        cap = 1 << 16
        while True:
            eu = np.empty(cap, dtype=np.int32)
            ev = np.empty(cap, dtype=np.int32)
            me = lib.gg_ego_network(n_p, _p(rp), _p(col), sn, n_t, m_cap, s ^ 0xD20F, _p(mark),
                                    _p(nodes), ctypes.addressof(n_out), _p(eu), _p(ev), cap)
            if me == -2:
                cap *= 4
                continue
            _check(me, "ego_network")
            break
        nn = int(n_out.value)
        types = uniform_types(nn, L, s ^ 0x7E57)
        out.append(csr_from_edges(nn, eu[:me], ev[:me], types, L, f"ego(g={g},seed={seed})"))
    return out


# ---------------------------------------------------------------- workloads

def workload(name: str) -> dict:
    """The standard seeded workloads, by name.

    er_small   ER G(n=2000, m=10000), L=3 uniform types
    cl_large   Chung-Lu n=2e6, m=2e7, gamma=2.1, max weight 5e4, L=5 Zipf(1.2) types
    sbm_typed  SBM sizes 500k/300k/150k/50k, affinity 1 between / 0.05 within, m=3e7, L=4
    cl_mid     cl_large scaled down 10x: n=2e5, m=2e6, gamma=2.1, max weight 1.2e4, L=5
               Zipf(1.2) types (the size used for profiler captures)
    """
    if name == "er_small":
        return erdos_renyi(2000, 10000, 3, SEED_BASE + 1)
    if name == "cl_large":
        return chung_lu(2_000_000, 20_000_000, 2.1, 5.0e4, 5, SEED_BASE + 2, type_zipf=1.2)
    if name == "cl_mid":
        return chung_lu(200_000, 2_000_000, 2.1, 1.2e4, 5, SEED_BASE + 7, type_zipf=1.2)
    if name == "sbm_typed":
        aff = np.full((4, 4), 1.0)
        np.fill_diagonal(aff, 0.05)
        return sbm([500_000, 300_000, 150_000, 50_000], aff, 30_000_000, SEED_BASE + 3)
    raise KeyError(name)


def ego_parent(seed: int = SEED_BASE + 4) -> dict:
    """Parent graph of the batched workload: Chung-Lu n=4e6, average degree 20
    (m = 4e7), gamma = 2.3, max weight 2e4, L = 6 uniform types."""
    return chung_lu(4_000_000, 40_000_000, 2.3, 2.0e4, 6, seed)


def ego_batch(count: int = 8192, seed: int = SEED_BASE + 4, parent: dict | None = None,
              m_min: int = 100, m_max: int = 400_000, n_max: int = 20_000, L: int = 6) -> dict:
    """The batched workload as one block-diagonal union (dict with node_off).

    Graph g (seed + g): u ~ U(0,1), edge target round(m_min (m_max/m_min)^u)
    (log-uniform), seed node drawn in proportion to degree, breadth-first
    ball grown node by node until the induced subgraph reaches the edge
    target or n_max nodes; L uniform types."""
    lib = _load()
    parent = parent if parent is not None else ego_parent(seed)
    rp, col = parent["row_ptr"], parent["col"]
    n_out = np.zeros(count, dtype=np.int64)
    m_out = np.zeros(count, dtype=np.int64)
    _check(lib.gg_ego_batch_sizes(parent["n"], _p(rp), _p(col), count, m_min, m_max, n_max, seed, _p(n_out),
                                  _p(m_out)), "ego_batch_sizes")
    node_off = np.concatenate([[0], np.cumsum(n_out)]).astype(np.int64)
    nnz_off = np.concatenate([[0], np.cumsum(2 * m_out)]).astype(np.int64)
    n, nnz = int(node_off[-1]), int(nnz_off[-1])
    u_rp = np.empty(n + 1, dtype=np.int64)
    u_col = np.empty(nnz, dtype=np.int32)
    u_ty = np.empty(n, dtype=np.uint8)
    _check(lib.gg_ego_batch_fill(parent["n"], _p(rp), _p(col), count, m_min, m_max, n_max, seed, L, _p(node_off),
                                 _p(nnz_off), _p(u_rp), _p(u_col), _p(u_ty)), "ego_batch_fill")
    u_rp[n] = nnz
    return {"n": n, "m": nnz // 2, "L": L, "row_ptr": u_rp, "col": u_col, "types": u_ty, "node_off": node_off,
            "graph_m": m_out, "graph_n": n_out, "name": f"ego batch of {count} (seed {seed})"}


def split(union: dict, g: int) -> dict:
    """Graph g of a union as a standalone graph (ids relative to its first node)."""
    a, b = int(union["node_off"][g]), int(union["node_off"][g + 1])
    rp = union["row_ptr"][a:b + 1] - union["row_ptr"][a]
    col = union["col"][int(union["row_ptr"][a]):int(union["row_ptr"][b])] - a
    return {"n": b - a, "m": int(rp[-1]) // 2, "L": union["L"], "row_ptr": rp.astype(np.int64),
            "col": col.astype(np.int32), "types": union["types"][a:b].copy(), "name": f"graph {g}"}


def concat(graphs: list) -> dict:
    """Block-diagonal union of graphs with the same L: node_off marks each graph."""
    node_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        node_off[k + 1] = node_off[k] + g["n"]
    nnz = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        nnz[k + 1] = nnz[k] + int(g["row_ptr"][-1])
    rp = np.empty(int(node_off[-1]) + 1, dtype=np.int64)
    col = np.empty(int(nnz[-1]), dtype=np.int32)
    ty = np.empty(int(node_off[-1]), dtype=np.uint8)
    for k, g in enumerate(graphs):
        a, b = int(node_off[k]), int(node_off[k + 1])
        rp[a:b] = g["row_ptr"][:-1] + nnz[k]
        col[nnz[k]:nnz[k + 1]] = g["col"] + a
        ty[a:b] = g["types"]
    rp[-1] = nnz[-1]
    L = graphs[0]["L"] if graphs else 1
    return {"n": int(node_off[-1]), "m": int(nnz[-1]) // 2, "L": L, "row_ptr": rp, "col": col, "types": ty,
            "node_off": node_off, "name": f"union of {len(graphs)} graphs"}
