"""Host logic that needs no GPU: the server's admission and grouping
decisions, resident-handle eviction, the autotuner's workload signature and
cache, and the shapes of the batched and served input mixes."""
import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")

from paper_2010_14058_gb300 import autotune, serve  # noqa: E402


def req(rid, m, L=3, key=None):
    n = max(10, -(-m // 5))
    return serve.Request(rid, L, np.zeros(n + 1, np.int64), np.zeros(2 * m, np.int32), np.zeros(n, np.uint8),
                         arrival=rid * 1e-3, key=key)


class FakeHandle:
    def __init__(self, nbytes):
        self.device_bytes = nbytes
        self.freed = False

    def free(self):
        self.freed = True


def test_groups_respect_type_count_size_and_budget():
    s = serve.Server(budget_bytes=10 << 30, small_edges=1000, batch_edges=2500, batch_graphs=3)
    pending = [req(0, 500), req(1, 600, L=4), req(2, 700), req(3, 900), req(4, 5000), req(5, 100)]
    g = s._take_group(pending)
    # head's L = 3; L = 4 skipped; 500 + 700 + 900 = 2100 <= 2500; then 3 graphs reached
    assert [r.rid for r in g.reqs] == [0, 2, 3]
    assert [r.rid for r in pending] == [1, 4, 5]
    assert s._in_use == g.nbytes == sum(r.bytes_needed() for r in g.reqs)
    g2 = s._take_group(pending)                          # L = 4 alone (nothing else of its L fits)
    assert [r.rid for r in g2.reqs] == [1]
    g3 = s._take_group(pending)                          # large request: never grouped
    assert [r.rid for r in g3.reqs] == [4]


def test_admission_waits_for_memory():
    big = req(0, 100_000)
    s = serve.Server(budget_bytes=big.bytes_needed() + 1000)
    assert s._take_group([big]) is not None
    pending = [req(1, 100_000)]
    assert s._take_group(pending) is None and len(pending) == 1      # no room until the first finishes
    s._in_use = 0
    assert s._take_group(pending) is not None
    with pytest.raises(ValueError):
        s._take_group([req(2, 10_000_000)])                          # can never fit


def test_resident_hits_and_lru_eviction():
    r1, r2 = req(0, 200_000, key="a"), req(1, 200_000, key="b")
    need = r1.bytes_needed()
    s = serve.Server(budget_bytes=int(2.5 * need), small_edges=1000, resident_bytes=2 * need)
    for r in (r1, r2):                                  # both become resident after running
        g = s._take_group([r])
        s._finish(g, FakeHandle(need))
    assert list(s._resident) == ["a", "b"] and s._in_use == 0
    g = s._take_group([req(2, 200_000, key="a")])       # hit: no reservation, handle handed over
    assert g.handle is not None and g.nbytes == 0 and s._resident["a"].busy
    s._finish(g, g.handle)
    assert not s._resident["a"].busy and list(s._resident) == ["b", "a"]   # "a" is now the newest
    g = s._take_group([req(3, 200_000, key="c")])       # needs room: the oldest idle ("b") goes
    assert g is not None and "b" not in s._resident
    s.close()
    assert not s._resident


def test_summary_percentiles():
    res = [serve.Result(k, np.zeros(3), arrival=0.0, started=0.0, done=(k + 1) / 100, status=0, group_size=1)
           for k in range(100)]
    reqs = [req(k, 1000) for k in range(100)]
    s = serve.summarize(res, reqs)
    assert s["requests"] == 100 and s["edges"] == 100_000
    assert s["p50_ms"] == pytest.approx(505.0) and s["p99_ms"] == pytest.approx(990.1)


def test_autotune_signature_and_cache(tmp_path):
    assert autotune.signature(2_000_000, 20_000_000, 37_312, 5) == "L5-n20-m24-d15-g0"
    path = str(tmp_path / "c.json")
    assert autotune.cached("x", path) is None
    autotune._store("x", {"options": {"ctas_per_sm": 2}}, path)
    autotune._store("y", {"options": {"ctas_per_sm": 4}}, path)
    assert autotune.cached("x", path) == {"ctas_per_sm": 2} and autotune.cached("y", path) == {"ctas_per_sm": 4}
    assert set(autotune.DEFAULTS) == set(autotune.SPACE)


def test_ego_batch_and_request_pool_shapes():
    u = graphgen.ego_batch(24, parent=graphgen.chung_lu(20_000, 200_000, 2.3, 500.0, 6, 5), n_max=2000,
                           m_max=20_000)
    assert len(u["node_off"]) == 25 and u["node_off"][-1] == u["n"] and u["L"] == 6
    assert int(u["graph_m"].sum()) == u["m"] and u["graph_m"].max() <= 20_000
    pool = serve.request_pool(6, seed=3, m_min=100, m_max=5000)
    assert all(100 <= g["m"] <= 5000 and 3 <= g["L"] <= 8 for g in pool)
    tr = serve.poisson_trace(pool, 500.0, 0.2, seed=1)
    assert all(a.arrival < b.arrival for a, b in zip(tr[:-1], tr[1:])) and all(r.key is not None for r in tr)


def test_autotune_descent_with_fake_timings(monkeypatch, tmp_path):
    # a fake measurement: time = sum of per-knob costs; totals fixed
    cost = {"light_edge_max_degree": {32: 3.0, 64: 1.0, 128: 2.0, 256: 2.5},
            "ctas_per_sm": {2: 0.5, 3: 1.0, 4: 2.0}}
    seen = []

    def fake(build, options, L, G, ngraphs, stream, reps):
        seen.append(dict(options))
        return sum(cost[k][v] for k, v in options.items()), np.ones((ngraphs, G), np.int64)

    monkeypatch.setattr(autotune, "_time_count", fake)
    rp = torch.tensor([0, 1, 2], dtype=torch.int64)
    col = torch.tensor([1, 0], dtype=torch.int32)
    ty = torch.zeros(2, dtype=torch.uint8)
    space = {k: sorted(v) for k, v in cost.items()}
    e = autotune.tune(rp, col, ty, 2, space=space, reps=1, path=str(tmp_path / "t.json"), stream=object())
    assert e["options"] == {"light_edge_max_degree": 64, "ctas_per_sm": 2}
    assert e["ms"] == 1.5 and e["default_ms"] == 2.5 + 1.0
    assert len(seen) == 1 + 3 + 2 and len({tuple(sorted(o.items())) for o in seen}) == len(seen)   # no repeats
    assert autotune.cached(e["signature"], str(tmp_path / "t.json")) == e["options"]

    def changing(build, options, L, G, ngraphs, stream, reps):   # a candidate that alters the counts
        return 1.0, np.full((ngraphs, G), options["ctas_per_sm"], np.int64)

    monkeypatch.setattr(autotune, "_time_count", changing)
    with pytest.raises(RuntimeError):
        autotune.tune(rp, col, ty, 2, space={"ctas_per_sm": [2, 3]}, reps=1, store=False, stream=object())
