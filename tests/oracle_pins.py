"""Pin helpers shared by the oracle tests (CPU only).

Each helper states the expected counts of a graph family or an identity
that the mathematics fixes, independently of the oracle's code, so that a
mistake in the oracle fails a check here.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

import graphgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# 4-node orbit numbering (Table 3): g3 4-path end edge, g4 4-path centre edge,
# g5 4-star, g6 4-cycle, g7 tailed-triangle tail, g8 tailed-triangle edge
# opposite the degree-3 node, g9 tailed-triangle edge at the degree-3 node,
# g10 chordal-cycle outer edge, g11 chordal-cycle chord, g12 4-clique.
GRAPHLET_EDGES = {1: 2, 2: 3, 3: 3, 4: 3, 5: 4, 6: 4, 7: 5, 8: 6}


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def graph_from_edges(n, edges, types, L, name="g"):
    e = np.array(sorted((min(a, b), max(a, b)) for a, b in edges), dtype=np.int32).reshape(-1, 2)
    return graphgen.csr_from_edges(n, e[:, 0], e[:, 1], np.array(types, dtype=np.uint8), L, name)


def random_graph(n, p, L, seed):
    rng = np.random.default_rng(seed)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    types = rng.integers(0, L, n)
    return graph_from_edges(n, edges, types, L, f"G({n},{p},L={L},seed={seed})")


# ------------------------------------------------------------ layout, by enumeration

def pairs(L):
    """(t,t') with t <= t' in lexicographic order (itertools order)."""
    return list(itertools.combinations_with_replacement(range(L), 2))


def multisets(L, K):
    """sorted K-multisets over [0,L) in lexicographic order (itertools order)."""
    return list(itertools.combinations_with_replacement(range(L), K))


def per_edge_slot(L, orbit, t, tp=None):
    """slot of (orbit, types) in a per-edge row: orbit 1 (3-path) / 2 (triangle)
    take one type, orbits 3..12 take the unordered pair {t, tp}."""
    if orbit in (1, 2):
        return (orbit - 1) * L + t
    P = L * (L + 1) // 2
    return 2 * L + (orbit - 3) * P + pairs(L).index(tuple(sorted((t, tp))))


def global_slot(L, graphlet, types):
    """slot of (graphlet, type multiset) in the global vector; graphlet 0 is
    the typed edge, 1 the 3-path, 2 the triangle, 3..8 the 4-node graphlets."""
    sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    K = 2 if graphlet == 0 else (3 if graphlet <= 2 else 4)
    return sum(sizes[:graphlet]) + multisets(L, K).index(tuple(sorted(types)))


def global_size(L):
    return math.comb(L + 1, 2) + 2 * math.comb(L + 2, 3) + 6 * math.comb(L + 3, 4)


def edge_list(g):
    """edge ids -> (u, v), u < v, lexicographic."""
    out = []
    rp, col = g["row_ptr"], g["col"]
    for u in range(g["n"]):
        for v in sorted(col[rp[u]:rp[u + 1]]):
            if v > u:
                out.append((u, int(v)))
    return out


# ------------------------------------------------------------- closed forms

def expected_clique(types, L):
    """K_n: every pair adjacent.  Per edge, T^t = all other nodes of type t,
    S_i = S_j = I = empty, so only g2 and g12 (and g11 = 0) are nonzero."""
    n = len(types)
    cnt = np.bincount(types, minlength=L)
    m = n * (n - 1) // 2
    S = 2 * L + 10 * L * (L + 1) // 2
    pe = np.zeros((m, S), dtype=np.int64)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n)]
    for e, (a, b) in enumerate(edges):
        c = cnt.copy()
        c[types[a]] -= 1
        c[types[b]] -= 1
        for t in range(L):
            pe[e, per_edge_slot(L, 2, t)] = c[t]
        for t, tp in pairs(L):
            pe[e, per_edge_slot(L, 12, t, tp)] = math.comb(int(c[t]), 2) if t == tp else int(c[t]) * int(c[tp])
    gl = np.zeros(global_size(L), dtype=np.int64)
    for K, gid in ((2, 0), (3, 2), (4, 8)):
        for ms in multisets(L, K):
            mult = np.bincount(ms, minlength=L)
            gl[global_slot(L, gid, ms)] = int(np.prod([math.comb(int(cnt[t]), int(mult[t])) for t in range(L)]))
    return edges, pe, gl


def expected_star(center_type, leaf_types, L):
    """K_{1,n}: per edge (centre, leaf), S_centre = the other leaves, all
    pairs of them non-adjacent: g1 and g5 only."""
    n = len(leaf_types)
    types = [center_type] + list(leaf_types)
    S = 2 * L + 10 * L * (L + 1) // 2
    pe = np.zeros((n, S), dtype=np.int64)
    edges = [(0, b) for b in range(1, n + 1)]
    for e, (_, b) in enumerate(edges):
        others = [types[x] for x in range(1, n + 1) if x != b]
        for t in others:
            pe[e, per_edge_slot(L, 1, t)] += 1
        for x, y in itertools.combinations(others, 2):
            pe[e, per_edge_slot(L, 5, x, y)] += 1
    gl = np.zeros(global_size(L), dtype=np.int64)
    for _, b in edges:
        gl[global_slot(L, 0, (center_type, types[b]))] += 1
    for x, y in itertools.combinations(leaf_types, 2):
        gl[global_slot(L, 1, (center_type, x, y))] += 1
    for x, y, z in itertools.combinations(leaf_types, 3):
        gl[global_slot(L, 4, (center_type, x, y, z))] += 1
    return types, edges, pe, gl


def expected_cycle(types, L):
    """C_n, n >= 5: per edge (v_k, v_k+1) the 3-paths through v_k-1 and v_k+2,
    4-path ends (v_k-2, v_k-1) and (v_k+2, v_k+3), 4-path centre
    (v_k-1, v_k+2).  For n = 5 the two ends share v_k+3 = v_k-2."""
    n = len(types)
    assert n >= 5
    S = 2 * L + 10 * L * (L + 1) // 2
    edges = sorted((min(k, (k + 1) % n), max(k, (k + 1) % n)) for k in range(n))
    pe = np.zeros((n, S), dtype=np.int64)
    for k in range(n):
        a, b = k, (k + 1) % n
        e = edges.index((min(a, b), max(a, b)))
        ty = lambda x: types[x % n]
        pe[e, per_edge_slot(L, 1, ty(k - 1))] += 1
        pe[e, per_edge_slot(L, 1, ty(k + 2))] += 1
        pe[e, per_edge_slot(L, 3, ty(k - 1), ty(k - 2))] += 1
        pe[e, per_edge_slot(L, 3, ty(k + 2), ty(k + 3))] += 1
        pe[e, per_edge_slot(L, 4, ty(k - 1), ty(k + 2))] += 1
    gl = np.zeros(global_size(L), dtype=np.int64)
    for k in range(n):
        gl[global_slot(L, 0, (types[k], types[(k + 1) % n]))] += 1
        gl[global_slot(L, 1, (types[k], types[(k + 1) % n], types[(k + 2) % n]))] += 1
        gl[global_slot(L, 3, tuple(types[(k + d) % n] for d in range(4)))] += 1
    return edges, pe, gl


def expected_complete_bipartite(a, b):
    """K_{a,b} with node type = side (0 for the a side, 1 for the b side).
    Per edge (l, r): S_l = the other b-1 right nodes, S_r = the other a-1
    left nodes, T = I = empty; every left-right pair is adjacent (4-cycles),
    no same-side pair is (4-stars)."""
    L = 2
    S = 2 * L + 10 * 3
    types = [0] * a + [1] * b
    edges = [(l, a + r) for l in range(a) for r in range(b)]
    pe = np.zeros((len(edges), S), dtype=np.int64)
    for e in range(len(edges)):
        pe[e, per_edge_slot(L, 1, 1)] = b - 1
        pe[e, per_edge_slot(L, 1, 0)] = a - 1
        pe[e, per_edge_slot(L, 6, 0, 1)] = (a - 1) * (b - 1)
        pe[e, per_edge_slot(L, 5, 1, 1)] = math.comb(b - 1, 2)
        pe[e, per_edge_slot(L, 5, 0, 0)] = math.comb(a - 1, 2)
    gl = np.zeros(global_size(L), dtype=np.int64)
    gl[global_slot(L, 0, (0, 1))] = a * b
    gl[global_slot(L, 1, (0, 1, 1))] = a * math.comb(b, 2)
    gl[global_slot(L, 1, (0, 0, 1))] = b * math.comb(a, 2)
    gl[global_slot(L, 5, (0, 0, 1, 1))] = math.comb(a, 2) * math.comb(b, 2)
    gl[global_slot(L, 4, (0, 1, 1, 1))] = a * math.comb(b, 3)
    gl[global_slot(L, 4, (0, 0, 0, 1))] = b * math.comb(a, 3)
    return types, edges, pe, gl


def expected_path(types, L):
    """P_n (nodes 0..n-1 in a line)."""
    n = len(types)
    S = 2 * L + 10 * L * (L + 1) // 2
    edges = [(k, k + 1) for k in range(n - 1)]
    pe = np.zeros((n - 1, S), dtype=np.int64)
    for e, (a, b) in enumerate(edges):
        if a >= 1:
            pe[e, per_edge_slot(L, 1, types[a - 1])] += 1
        if b + 1 <= n - 1:
            pe[e, per_edge_slot(L, 1, types[b + 1])] += 1
        if a >= 2:
            pe[e, per_edge_slot(L, 3, types[a - 1], types[a - 2])] += 1
        if b + 2 <= n - 1:
            pe[e, per_edge_slot(L, 3, types[b + 1], types[b + 2])] += 1
        if a >= 1 and b + 1 <= n - 1:
            pe[e, per_edge_slot(L, 4, types[a - 1], types[b + 1])] += 1
    gl = np.zeros(global_size(L), dtype=np.int64)
    for k in range(n - 1):
        gl[global_slot(L, 0, types[k:k + 2])] += 1
    for k in range(n - 2):
        gl[global_slot(L, 1, types[k:k + 3])] += 1
    for k in range(n - 3):
        gl[global_slot(L, 3, types[k:k + 4])] += 1
    return edges, pe, gl


# ------------------------------------------------------------- untyped identities

def untyped_identities(g, gl_untyped):
    """Standard identities between degree sums and untyped graphlet counts
    (L = 1 global vector: [edges, 3-path, triangle, 4-path, 4-star, 4-cycle,
    tailed-triangle, chordal-cycle, 4-clique]).  Returns (lhs, rhs) pairs."""
    deg = np.diff(g["row_ptr"]).astype(object)
    _, n3p, ntri, np4, nstar, nc4, npaw, ndia, nk4 = [int(x) for x in gl_untyped]
    out = []
    out.append((sum(d * (d - 1) // 2 for d in deg), n3p + 3 * ntri))
    out.append((sum(d * (d - 1) * (d - 2) // 6 for d in deg), nstar + npaw + 2 * ndia + 4 * nk4))
    rp, col = g["row_ptr"], g["col"]
    s = 0
    for u in range(g["n"]):
        for v in col[rp[u]:rp[u + 1]]:
            if v > u:
                s += (deg[u] - 1) * (deg[v] - 1)
    out.append((s - 3 * ntri, np4 + 4 * nc4 + 2 * npaw + 6 * ndia + 12 * nk4))
    return out


# ------------------------------------------- position-aware layout (Sec. 5)
# Numbered shapes: 0 edge; 1 3-path, 0 the centre; 2 triangle; 3 4-path
# 0-1-2-3; 4 4-star, 0 the centre; 5 4-cycle 0-1-2-3-0; 6 tailed triangle, 0
# the degree-3 node, 1 the tail; 7 chordal cycle, 0-1 the chord; 8 4-clique.

BLOCK_EDGES = {0: 1, **GRAPHLET_EDGES}

SHAPES = {0: [(0, 1)], 1: [(0, 1), (0, 2)], 2: [(0, 1), (0, 2), (1, 2)], 3: [(0, 1), (1, 2), (2, 3)],
          4: [(0, 1), (0, 2), (0, 3)], 5: [(0, 1), (1, 2), (2, 3), (3, 0)], 6: [(0, 1), (0, 2), (0, 3), (2, 3)],
          7: [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)], 8: [(a, b) for a in range(4) for b in range(a + 1, 4)]}


def automorphisms(b):
    k = 2 if b == 0 else (3 if b <= 2 else 4)
    E = {frozenset(e) for e in SHAPES[b]}
    return [p for p in itertools.permutations(range(k)) if {frozenset((p[u], p[v])) for u, v in E} == E]


def canonical_classes(L, b):
    """{labelling: rank} for every labelling, ranks by smallest member."""
    k = len(automorphisms(b)[0])
    aut = automorphisms(b)
    canon = {}
    for lab in itertools.product(range(L), repeat=k):
        canon[lab] = min(tuple(lab[p[x]] for x in range(k)) for p in aut)
    reps = sorted(set(canon.values()))
    rank = {r: i for i, r in enumerate(reps)}
    return {lab: rank[c] for lab, c in canon.items()}


def burnside(L):
    """Number of labellings up to automorphism, per block, in closed form."""
    P = L * (L + 1) // 2
    return [P, L * P, math.comb(L + 2, 3), (L ** 4 + L ** 2) // 2, L * math.comb(L + 2, 3),
            (L ** 4 + 2 * L ** 3 + 3 * L ** 2 + 2 * L) // 8, L * L * P, P * P, math.comb(L + 3, 4)]


def pa_sizes(L):
    """Per-edge block sizes O1..O12."""
    P, LL = L * (L + 1) // 2, L * L
    return [2 * L, L, 2 * LL, LL, 2 * P, LL, 2 * P, LL, 2 * LL, 2 * LL, P, P]


def pa_offsets(L):
    return np.concatenate([[0], np.cumsum(pa_sizes(L))])


def slot_instance(L, slot, p_lo, p_hi):
    """(global block, labelling of the numbered shape) of per-edge slot `slot`
    for an edge whose endpoints have types p_lo, p_hi."""
    off = pa_offsets(L)
    o = int(np.searchsorted(off, slot, side="right"))          # 1..12
    r = slot - off[o - 1]
    LL, P = L * L, L * (L + 1) // 2
    pr = pairs(L)
    side = lambda s: (p_lo, p_hi) if s == 0 else (p_hi, p_lo)  # noqa: E731  (that side, the other)
    if o == 1:
        me, other = side(r // L)
        return 1, (me, other, r % L)
    if o == 2:
        return 2, (p_lo, p_hi, r)
    if o == 3:
        me, other = side(r // LL)
        x, y = divmod(r % LL, L)
        return 3, (y, x, me, other)
    if o == 4:
        x, y = divmod(r, L)
        return 3, (x, p_lo, p_hi, y)
    if o == 5:
        me, other = side(r // P)
        t, u = pr[r % P]
        return 4, (me, other, t, u)
    if o == 6:
        x, y = divmod(r, L)
        return 5, (p_lo, p_hi, y, x)
    if o == 7:
        me, other = side(r // P)
        t, u = pr[r % P]
        return 6, (me, other, t, u)
    if o == 8:
        x, y = divmod(r, L)
        return 6, (x, y, p_lo, p_hi)
    if o == 9:
        me, other = side(r // LL)
        x, y = divmod(r % LL, L)
        return 6, (me, y, other, x)
    if o == 10:
        me, other = side(r // LL)
        x, y = divmod(r % LL, L)
        return 7, (me, x, other, y)
    t, u = pr[r]
    return (7 if o == 11 else 8), (p_lo, p_hi, t, u)


def global_slot_pa(L, block, lab, classes=None):
    sizes = burnside(L)
    classes = classes or {}
    if block not in classes:
        classes[block] = canonical_classes(L, block)
    return sum(sizes[:block]) + classes[block][tuple(lab)]


def merge_per_edge(L, pe_pa):
    """Position-aware rows -> typed rows (orbit, unordered pair)."""
    off = pa_offsets(L)
    m = pe_pa.shape[0]
    out = np.zeros((m, 2 * L + 10 * L * (L + 1) // 2), np.int64)
    LL, P = L * L, L * (L + 1) // 2
    pr = pairs(L)
    for t in range(L):
        out[:, per_edge_slot(L, 1, t)] = pe_pa[:, off[0] + t] + pe_pa[:, off[0] + L + t]
        out[:, per_edge_slot(L, 2, t)] = pe_pa[:, off[1] + t]
    for o in range(3, 13):
        for r in range(pa_sizes(L)[o - 1]):
            if o in (5, 7, 11, 12):                     # [side][pair] or [pair]
                t, u = pr[r % P]
            else:                                       # [side][x][y] or [x][y]
                x, y = divmod(r % LL, L)
                t, u = min(x, y), max(x, y)
            out[:, per_edge_slot(L, o, t, u)] += pe_pa[:, off[o - 1] + r]
    return out


def merge_pa_global(L, gl_pa):
    """Position-aware totals -> typed totals (each class to its type multiset)."""
    sizes = burnside(L)
    typed_sizes = [math.comb(L + 1, 2)] + [math.comb(L + 2, 3)] * 2 + [math.comb(L + 3, 4)] * 6
    out = np.zeros(sum(typed_sizes), np.int64)
    s = 0
    for b in range(9):
        K = 2 if b == 0 else (3 if b <= 2 else 4)
        ms_rank = {ms: i for i, ms in enumerate(multisets(L, K))}
        reps = sorted(set(min(tuple(lab[p[x]] for x in range(K)) for p in automorphisms(b))
                          for lab in itertools.product(range(L), repeat=K)))
        for r, rep in enumerate(reps):
            out[sum(typed_sizes[:b]) + ms_rank[tuple(sorted(rep))]] += gl_pa[s + r]
        s += sizes[b]
    return out


# ------------------------------------------------- directed graphs (Sec. 4.8)

def oriented_graph(n, arcs, types, L):
    """Out-neighbour CSR of an oriented graph from its arcs (u, v) = u -> v."""
    rp = np.zeros(n + 1, dtype=np.int64)
    for u, _ in arcs:
        rp[u + 1] += 1
    rp = np.cumsum(rp)
    col = np.zeros(len(arcs), dtype=np.int32)
    fill = rp[:-1].copy()
    for u, v in arcs:
        col[fill[u]] = v
        fill[u] += 1
    return {"n": n, "L": L, "out_row_ptr": rp, "out_col": col, "types": np.asarray(types, dtype=np.uint8),
            "m": len(arcs)}


def random_oriented(n, p, L, seed, tournament=False):
    rng = np.random.default_rng(seed)
    arcs = []
    for a in range(n):
        for b in range(a + 1, n):
            if tournament or rng.random() < p:
                arcs.append((a, b) if rng.random() < 0.5 else (b, a))
    return oriented_graph(n, arcs, rng.integers(0, L, n), L)


def underlying(g):
    """The undirected graph of an oriented graph (symmetric CSR)."""
    arcs = [(u, int(v)) for u in range(g["n"]) for v in g["out_col"][g["out_row_ptr"][u]:g["out_row_ptr"][u + 1]]]
    return graph_from_edges(g["n"], arcs, g["types"], g["L"])


def directed_burnside(L):
    """Connected oriented 3-node graphs with L node types up to isomorphism:
    (1/6)(20 L^3 + 3 * 2 L^2 + 2 * 2 L) -- identity: 20 connected arc
    patterns; a transposition fixes 2 patterns (no arc between the swapped
    nodes, equal arcs to the third) with L^2 typings; a rotation fixes the
    2 cyclic triangles with L typings."""
    return (20 * L**3 + 6 * L**2 + 4 * L) // 6


REVERSE_BLOCK = [1, 0, 3, 2, 7, 6, 5, 4]          # per-edge blocks under reversal of every arc


def directed_class_maps(L, lib=None):
    """For every class: its undirected graphlet (1 path, 2 triangle) and
    sorted type triple, and the class of the reversed configuration."""
    import oracle
    nc = oracle.directed_classes(L, lib)
    und, rev = [None] * nc, [None] * nc
    for t in itertools.product(range(L), repeat=3):
        for a in itertools.product(range(3), repeat=3):
            r = oracle.directed_class(L, t, a, lib)
            if r < 0:
                continue
            arcs = sum(x != 0 for x in a)
            und[r] = (1 if arcs == 2 else 2, tuple(sorted(t)))
            rev[r] = oracle.directed_class(L, t, [(0, 2, 1)[x] for x in a], lib)
    return und, rev


def directed_pins(lib=None):
    """Names of the directed-graphlet pins that fail for an oracle build."""
    import oracle
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except oracle.OracleError:
            failed.append(name + " (error)")

    check("class count = Burnside", lambda: all(oracle.directed_classes(L, lib) == directed_burnside(L)
                                                   for L in range(1, 9)))
    for seed in range(6):
        L = [1, 2, 3][seed % 3]
        g = random_oriented(7 + seed, 0.55, L, 700 + seed)

        def vs_brute(g=g):
            pe, gl = oracle.directed3(g, lib=lib)
            pb, gb = oracle.directed3_brute(g, lib=lib)
            return np.array_equal(pe, pb) and np.array_equal(gl, gb)
        check(f"brute seed={seed}", vs_brute)

        def sums_to_undirected(g=g, L=L):
            pe, gl = oracle.directed3(g, lib=lib)
            u = underlying(g)
            pu, gu = oracle.paper(u, k=3, lib=lib)
            rows = np.concatenate([pe[:, 0:4 * L].reshape(-1, 4, L).sum(1), pe[:, 4 * L:].reshape(-1, 4, L).sum(1)], 1)
            und, _ = directed_class_maps(L, lib)
            glob = np.zeros_like(gu)
            tail_head = gl[:L * L].reshape(L, L)
            for a in range(L):
                for b in range(L):
                    glob[oracle.multiset_rank(L, sorted((a, b)), lib)] += tail_head[a, b]
            off3 = oracle.global_slots(L, 3, lib) - 2 * len(list(itertools.combinations_with_replacement(range(L), 3)))
            n3 = len(list(itertools.combinations_with_replacement(range(L), 3)))
            for r, v in enumerate(gl[L * L:]):
                h, ts = und[r]
                glob[off3 + (h - 1) * n3 + oracle.multiset_rank(L, list(ts), lib)] += v
            return np.array_equal(rows, pu) and np.array_equal(glob, gu)
        check(f"direction sums seed={seed}", sums_to_undirected)

        def reversal(g=g, L=L):
            pe, gl = oracle.directed3(g, lib=lib)
            arcs = [(int(v), u) for u in range(g["n"]) for v in g["out_col"][g["out_row_ptr"][u]:g["out_row_ptr"][u + 1]]]
            h = oriented_graph(g["n"], arcs, g["types"], L)
            pr, gr = oracle.directed3(h, lib=lib)
            want = pe.reshape(-1, 8, L)[:, REVERSE_BLOCK, :].reshape(pe.shape)
            _, rev = directed_class_maps(L, lib)
            wg = np.zeros_like(gl)
            wg[:L * L] = gl[:L * L].reshape(L, L).T.ravel()
            for r, v in enumerate(gl[L * L:]):
                wg[L * L + rev[r]] += v
            return np.array_equal(pr, want) and np.array_equal(gr, wg)
        check(f"reversal seed={seed}", reversal)

    def transitive_tournament():
        n = 9
        g = oriented_graph(n, [(a, b) for a in range(n) for b in range(a + 1, n)], [0] * n, 1)
        pe, gl = oracle.directed3(g, lib=lib)
        src, dst, _ = oracle.directed_edges(g, lib=lib)
        want = np.zeros_like(pe)
        for e, (i, j) in enumerate(zip(src, dst)):
            want[e, 7] = i                 # w < i: w -> i and w -> j
            want[e, 5] = j - i - 1         # i < w < j: i -> w, w -> j
            want[e, 4] = n - 1 - j         # w > j: i -> w, j -> w
        transitive = oracle.directed_class(1, [0, 0, 0], [1, 1, 1], lib)
        wg = np.zeros_like(gl)
        wg[0] = n * (n - 1) // 2
        wg[1 + transitive] = n * (n - 1) * (n - 2) // 6
        return np.array_equal(pe, want) and np.array_equal(gl, wg)
    check("transitive tournament", transitive_tournament)

    def cyclic_triangles():
        # Kendall and Babington Smith: a tournament on n nodes has
        # C(n,3) - sum_v C(out_v, 2) cyclic triangles
        ok = True
        for seed in range(3):
            g = random_oriented(12, 1.0, 1, 800 + seed, tournament=True)
            _, gl = oracle.directed3(g, per_edge=False, lib=lib)
            outd = np.diff(g["out_row_ptr"])
            cyc = oracle.directed_class(1, [0, 0, 0], [1, 2, 1], lib)
            ok &= gl[1 + cyc] == 12 * 11 * 10 // 6 - sum(int(d) * (int(d) - 1) // 2 for d in outd)
        return ok
    check("cyclic triangles of tournaments", cyclic_triangles)

    def stars():
        k = 6
        out = oriented_graph(k + 1, [(0, x) for x in range(1, k + 1)], [0] * (k + 1), 1)
        inn = oriented_graph(k + 1, [(x, 0) for x in range(1, k + 1)], [0] * (k + 1), 1)
        po, go = oracle.directed3(out, lib=lib)
        pi, gi = oracle.directed3(inn, lib=lib)
        out_star = oracle.directed_class(1, [0, 0, 0], [1, 1, 0], lib)   # 0 -> 1, 0 -> 2
        in_star = oracle.directed_class(1, [0, 0, 0], [2, 2, 0], lib)
        return ((po[:, 0] == k - 1).all() and po[:, 1:].sum() == 0 and (pi[:, 1] == k - 1).all()
                and go[1 + out_star] == k * (k - 1) // 2 and gi[1 + in_star] == k * (k - 1) // 2
                and go[1:].sum() == go[1 + out_star] and gi[1:].sum() == gi[1 + in_star])
    check("directed stars", stars)
    return failed


# ------------------------------------------- edge types (Def. 1, Defs. 4-5)

def edge_types_for(g, X, seed):
    """One seeded type in [0, X) per edge, written to both of its entries of col."""
    rng = np.random.default_rng(seed)
    rp, col = g["row_ptr"], g["col"]
    xi = np.zeros(len(col), dtype=np.uint8)
    seen = {}
    for u in range(g["n"]):
        for k in range(rp[u], rp[u + 1]):
            key = (min(u, int(col[k])), max(u, int(col[k])))
            if key not in seen:
                seen[key] = int(rng.integers(0, X))
            xi[k] = seen[key]
    return xi


def edge_types_from(g, fn):
    """Edge types from a function of the edge {u, v} (u < v)."""
    rp, col = g["row_ptr"], g["col"]
    return np.array([fn(min(u, int(col[k])), max(u, int(col[k]))) for u in range(g["n"])
                     for k in range(rp[u], rp[u + 1])], dtype=np.uint8)


def et_offsets(L, X):
    """Starts of the three global blocks: edges, 3-paths, triangles."""
    n2 = len(multisets(L, 2)) * X
    n3 = len(multisets(L, 3)) * len(multisets(X, 2))
    return 0, n2, n2 + n3


def et_merge_to_typed(g, L, X, pe, gl, lib=None):
    """Per-edge rows and totals with the edge types summed out, in the
    typed (node types only) 3-node layout of oracle.paper(k = 3)."""
    import oracle
    P = X * (X + 1) // 2
    rows = np.concatenate([pe[:, :L * X].reshape(-1, L, X).sum(2), pe[:, L * X:].reshape(-1, L, P).sum(2)], 1)
    glob = np.zeros(oracle.global_slots(L, 3, lib), dtype=np.int64)
    o0, o1, o2 = et_offsets(L, X)
    n3 = len(multisets(L, 3))
    glob[:len(multisets(L, 2))] = gl[o0:o1].reshape(-1, X).sum(1)
    glob[len(multisets(L, 2)):len(multisets(L, 2)) + n3] = gl[o1:o2].reshape(n3, -1).sum(1)
    glob[len(multisets(L, 2)) + n3:] = gl[o2:].reshape(n3, -1).sum(1)
    return rows, glob


def edge_typed_pins(lib=None):
    """Names of the edge-typed pins that fail for an oracle build."""
    import oracle
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except oracle.OracleError:
            failed.append(name + " (error)")

    for seed in range(6):
        L, X = [1, 2, 3][seed % 3], [2, 3, 1, 4, 2, 3][seed]
        g = random_graph(8 + seed, 0.5, L, 900 + seed)
        xi = edge_types_for(g, X, 950 + seed)

        def vs_brute(g=g, xi=xi, X=X):
            pe, gl = oracle.edge_typed3(g, xi, X, lib=lib)
            pb, gb = oracle.edge_typed3_brute(g, xi, X, lib=lib)
            return np.array_equal(pe, pb) and np.array_equal(gl, gb)
        check(f"brute seed={seed}", vs_brute)

        def sums_to_typed(g=g, xi=xi, X=X, L=L):
            pe, gl = oracle.edge_typed3(g, xi, X, lib=lib)
            rows, glob = et_merge_to_typed(g, L, X, pe, gl, lib)
            pt, gt = oracle.paper(g, k=3, lib=lib)
            return np.array_equal(rows, pt) and np.array_equal(glob, gt)
        check(f"edge-type sums seed={seed}", sums_to_typed)

    def relabelled_edge_types():
        # a permutation s of the edge types moves path slot (t, x) to (t, s(x))
        # and triangle slot (t, {x, y}) to (t, {s(x), s(y)})
        L, X = 2, 3
        g = random_graph(10, 0.5, L, 977)
        xi = edge_types_for(g, X, 978)
        s = np.array([2, 0, 1], dtype=np.uint8)
        pe, _ = oracle.edge_typed3(g, xi, X, lib=lib)
        pr, _ = oracle.edge_typed3(g, s[xi], X, lib=lib)
        pairs_x = multisets(X, 2)
        want = np.zeros_like(pe)
        for t in range(L):
            for x in range(X):
                want[:, t * X + s[x]] = pe[:, t * X + x]
            for p, (x, y) in enumerate(pairs_x):
                q = pairs_x.index(tuple(sorted((int(s[x]), int(s[y])))))
                want[:, L * X + t * len(pairs_x) + q] = pe[:, L * X + t * len(pairs_x) + p]
        return np.array_equal(pr, want)
    check("edge-type relabelling", relabelled_edge_types)

    def typed_triangle():
        # K3, node types 0 1 1, edge types {0,1}: 0, {0,2}: 1, {1,2}: 2
        g = graph_from_edges(3, [(0, 1), (0, 2), (1, 2)], [0, 1, 1], 2)
        xi = edge_types_from(g, lambda u, v: {(0, 1): 0, (0, 2): 1, (1, 2): 2}[(u, v)])
        pe, gl = oracle.edge_typed3(g, xi, 3, lib=lib)
        L, X, P = 2, 3, 6
        want = np.zeros_like(pe)
        pr = multisets(X, 2)
        want[0, L * X + 1 * P + pr.index((1, 2))] = 1          # edge {0,1}: node 2 (type 1), edges 1 and 2
        want[1, L * X + 1 * P + pr.index((0, 2))] = 1          # edge {0,2}: node 1 (type 1), edges 0 and 2
        want[2, L * X + 0 * P + pr.index((0, 1))] = 1          # edge {1,2}: node 0 (type 0), edges 0 and 1
        o0, o1, o2 = et_offsets(L, X)
        wg = np.zeros_like(gl)
        for (u, v), x in (((0, 1), 0), ((0, 2), 1), ((1, 2), 2)):
            wg[o0 + multisets(L, 2).index(tuple(sorted((int(g["types"][u]), int(g["types"][v]))))) * X + x] += 1
        wg[o2 + multisets(L, 3).index((0, 1, 1)) * len(multisets(X, 3)) + multisets(X, 3).index((0, 1, 2))] = 1
        return np.array_equal(pe, want) and np.array_equal(gl, wg)
    check("typed triangle", typed_triangle)

    def star():
        # K_{1,7}: centre 0, leaves 1..7 of one type, edge types 0 for leaves
        # 1..4 and 1 for leaves 5..7: a leaf's edge of type x sees the other
        # leaves as paths (type 1, their edge type); 3-paths by edge-type
        # pair: C(4,2) {0,0}, 4*3 {0,1}, C(3,2) {1,1}
        g = graph_from_edges(8, [(0, v) for v in range(1, 8)], [0] + [1] * 7, 2)
        xi = edge_types_from(g, lambda u, v: 0 if v <= 4 else 1)
        pe, gl = oracle.edge_typed3(g, xi, 2, lib=lib)
        L, X = 2, 2
        ok = True
        for e, leaf in enumerate(range(1, 8)):
            n0 = 4 - (1 if leaf <= 4 else 0)
            n1 = 3 - (1 if leaf > 4 else 0)
            ok &= pe[e, 1 * X + 0] == n0 and pe[e, 1 * X + 1] == n1 and pe[e].sum() == n0 + n1
        o0, o1, o2 = et_offsets(L, X)
        r3 = multisets(L, 3).index((0, 1, 1)) * len(multisets(X, 2))
        ok &= gl[o1 + r3 + multisets(X, 2).index((0, 0))] == 6
        ok &= gl[o1 + r3 + multisets(X, 2).index((0, 1))] == 12
        ok &= gl[o1 + r3 + multisets(X, 2).index((1, 1))] == 3
        ok &= gl[o1:o2].sum() == 21 and gl[o2:].sum() == 0
        return bool(ok)
    check("star", star)
    return failed
