"""The work units behind bench.py's roofline figures, checked on the CPU
against a plain count from their definitions on small graphs: degree-priority
wedges and (anchor, neighbour) pairs per anchor class, the shorter sides of
the typed intersections, and the triangle / 4-clique sums read from per-edge
rows."""
import importlib.util
import os

import numpy as np
import pytest

import graphgen
from oracle_pins import random_graph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def plain_units(g, light_max, hub_min):
    n, L, rp, col, ty = g["n"], g["L"], g["row_ptr"], g["col"], g["types"]
    adj = [col[rp[x]:rp[x + 1]].tolist() for x in range(n)]
    deg = [len(a) for a in adj]
    prio = lambda x: (deg[x], x)                                  # noqa: E731
    out = {k: 0.0 for k in ("wedges_light", "wedges_heavy", "wedges_hub", "pairs_light", "pairs_heavy",
                            "pairs_hub", "typed_min_sum")}
    out["hubs"] = 0
    for x in range(n):
        # wedges x - v - w with v and w both of lower priority than x
        below = [v for v in adj[x] if prio(v) < prio(x)]
        W = sum(1 for v in below for w in adj[v] if prio(w) < prio(x))
        if W == 0:
            continue
        cls = "light" if W <= light_max else ("heavy" if W <= hub_min else "hub")
        out["wedges_" + cls] += W
        out["pairs_" + cls] += len(below)
        out["hubs"] += cls == "hub"
    for u in range(n):
        for v in adj[u]:
            if v > u:
                out["typed_min_sum"] += sum(min(sum(1 for y in adj[u] if ty[y] == t),
                                                sum(1 for y in adj[v] if ty[y] == t)) for t in range(L))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_kernel_units_match_plain_count(bench, seed):
    g = graphgen.chung_lu(300, 1500, 2.1, 60.0, 3, 40 + seed)
    for light_max, hub_min in ((64, 1 << 16), (4, 40), (1, 2)):
        assert bench.kernel_units(g, light_max, hub_min) == plain_units(g, light_max, hub_min)


def test_kernel_units_on_a_random_graph_with_ties(bench):
    g = random_graph(40, 0.3, 2, 11)                              # many equal degrees: ties broken by id
    assert bench.kernel_units(g, 8, 30) == plain_units(g, 8, 30)


def test_clique_units_read_the_rows(bench):
    torch = pytest.importorskip("torch")
    L, P = 3, 6
    S = 2 * L + 10 * P
    rng = np.random.default_rng(1)
    rows = rng.integers(0, 300, (50, S)).astype(np.int32)
    pe = torch.from_numpy(rows)
    T = rows[:, L:2 * L].astype(np.int64).sum(1)
    K = rows[:, 2 * L + 9 * P:2 * L + 10 * P].astype(np.int64).sum(1)
    big = T > 400
    got = bench.clique_units(pe, L, big_t=400, chunk=7)
    assert got == {"t_small": int(T[~big].sum()), "t_big": int(T[big].sum()), "k_small": int(K[~big].sum()),
                   "k_big": int(K[big].sum()), "edges_big": int(big.sum())}


def test_count_only_split(bench):
    got = bench.count_only(20_000_000, 908.4, 942.7)
    assert got == {"value": round(20_000_000 / 0.9084, 1), "unit": "edges/s", "count_ms": 908.4,
                   "build_and_free_ms": 34.3}
    assert bench.count_only(10, 0.0, 1.0) is None
