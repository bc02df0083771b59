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


# ------------------------------------------------------- CPU-baseline estimator

def test_edge_cost_proxy_is_its_definition(bench):
    g = random_graph(14, 0.4, 3, 71)
    src, dst, proxy = bench.edge_cost_proxy(g)
    import oracle
    s_o, d_o = oracle.edges(g)
    np.testing.assert_array_equal(src, s_o)
    np.testing.assert_array_equal(dst, d_o)
    rp, col = g["row_ptr"], g["col"]
    adj = [col[rp[x]:rp[x + 1]].tolist() for x in range(g["n"])]
    for e, (u, v) in enumerate(zip(src, dst)):
        want = len(adj[u]) + len(adj[v]) + sum(len(adj[w]) for w in adj[u]) + sum(len(adj[w]) for w in adj[v])
        assert proxy[e] == want


def test_oracle_design_partitions_the_edges(bench):
    rng = np.random.default_rng(4)
    proxy = np.exp(rng.normal(10, 2, 50_000))
    strata = bench.oracle_design(proxy, budget_edges=400, heaviest=30, seed=9)
    assert strata[0][0] == "heaviest" and strata[0][1] == 30
    np.testing.assert_array_equal(np.sort(strata[0][2]), np.sort(np.argsort(-proxy)[:30]))
    assert sum(N for _, N, _ in strata) == len(proxy)              # the strata cover every edge once
    for _, N, pick in strata:
        assert 1 <= len(pick) <= N and len(np.unique(pick)) == len(pick)
    again = bench.oracle_design(proxy, budget_edges=400, heaviest=30, seed=9)
    assert all(np.array_equal(a[2], b[2]) for a, b in zip(strata, again))    # seeded


class _FakeOpen:
    """Stands in for oracle.OpenGraph: every edge takes time c * proxy."""

    def __init__(self, proxy, c):
        self.proxy, self.c = proxy, c

    def paper_edges(self, ids, k=4, nthreads=0, per_edge=False, times=False):
        return None, None, self.c * self.proxy[ids]


@pytest.mark.parametrize("thin", [1, 10])
def test_estimator_is_exact_when_time_follows_the_proxy_within_strata(bench, thin):
    # time proportional to the proxy: within a log2 stratum the per-edge
    # times vary, so only the certainty stratum is exact; a constant time
    # per stratum makes the Horvitz-Thompson sum exact
    rng = np.random.default_rng(5)
    proxy = np.floor(2.0 ** rng.uniform(3, 20, 20_000))
    strata = bench.oracle_design(proxy, budget_edges=500, heaviest=50, seed=3)
    bins = np.floor(np.log2(proxy))
    flat = 2.0 ** bins                                              # one value per stratum
    top = strata[0][2]
    flat[top] = proxy[top]
    r = bench.oracle_estimate(_FakeOpen(flat, 1e-6), strata, nthreads=4, thin=thin)
    assert abs(r["work_thread_s"] - 1e-6 * flat.sum()) <= 1e-9 * flat.sum()
    r2 = bench.oracle_estimate(_FakeOpen(proxy, 1e-6), strata, nthreads=4, thin=thin)
    assert abs(r2["work_thread_s"] / (1e-6 * proxy.sum()) - 1) < 0.05    # unbiased up to sampling


def test_w_alg_is_its_definition(bench):
    import math

    import oracle
    g = graphgen.chung_lu(300, 1500, 2.1, 60.0, 3, 12)
    pe, _ = oracle.paper(g, k=3)
    L = g["L"]
    tsize = pe[:, L:2 * L].sum(1)
    rp, col = g["row_ptr"], g["col"]
    adj = [col[rp[x]:rp[x + 1]].tolist() for x in range(g["n"])]
    deg = [len(a) for a in adj]
    lg = [math.ceil(math.log2(d)) if d > 1 else 0 for d in deg]
    src, dst = oracle.edges(g)
    S = 2 * L + 10 * L * (L + 1) // 2
    want = 0
    for e, (i, j) in enumerate(zip(src, dst)):
        U = deg[i] + deg[j] - 2 - int(tsize[e])
        want += 4 * (deg[i] + deg[j])
        for x, other in ((i, j), (j, i)):
            want += 4 * sum(min(deg[w], U * lg[w]) for w in adj[x] if w != other)
    want += 4 * S * len(src)
    got = bench.w_alg_bytes(g, tsize, S)["bytes"]
    assert abs(got - want) <= 1e-9 * want
