"""The continuous-batching server: every request's global totals equal the
CPU oracle's (Alg. 1-3 + Lemmas, Sec. 6) and a standalone tg_count of the
same graph (exact integers, tolerance 0), alone and in a mix where requests
of several sizes and type counts are grouped, overlapped on several streams,
admitted under a tight memory budget and counted on resident handles."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402
from paper_2010_14058_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module")
def trace():
    pool = serve.request_pool(24, seed=5, m_min=100, m_max=60_000)
    reqs = serve.poisson_trace(pool, rate_per_s=400.0, duration_s=0.25, seed=11)
    assert len(reqs) > 40
    return reqs


@pytest.fixture(scope="module")
def oracle_totals(trace):
    """Oracle global totals of every distinct graph in the trace, by pool key."""
    out = {}
    for r in trace:
        if r.key not in out:
            g = {"n": r.n, "m": r.m, "L": r.L, "row_ptr": r.row_ptr, "col": r.col, "types": r.types}
            out[r.key] = oracle.paper(g, k=4, per_edge=False)[1]
    return out


def standalone(r):
    h = tg.tg_build(torch.from_numpy(r.row_ptr).cuda(), torch.from_numpy(r.col).cuda(),
                    torch.from_numpy(r.types).cuda(), r.L)
    gl = torch.zeros(tg.tg_layout(r.L, 4)["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, None, gl)
    assert tg.tg_query_status(h) == 0
    h.free()
    return gl.cpu().numpy()


def test_mixed_equals_alone(trace, oracle_totals):
    budget = 3 * max(r.bytes_needed() for r in trace)       # forces waits for memory
    # every request already arrived: the scheduler groups the small ones
    # whatever the GPU's speed (the real-time replays are in the tests below)
    mixed = serve.Server(budget_bytes=budget, workers=4, small_edges=20_000, batch_edges=200_000).run(
        trace, realtime=False)
    alone = serve.Server(budget_bytes=budget, workers=1, batching=False).run(trace, realtime=False)
    assert [r.rid for r in mixed] == [r.rid for r in trace]
    assert any(r.group_size > 1 for r in mixed)             # micro-batches were formed
    for a, b, r in zip(mixed, alone, trace):
        assert a.status == 0 and b.status == 0
        np.testing.assert_array_equal(a.totals, b.totals)
    for r in trace[:12]:
        np.testing.assert_array_equal(mixed[r.rid].totals, standalone(r))
    for a, r in zip(mixed, trace):                           # every served result is the oracle's
        np.testing.assert_array_equal(a.totals, oracle_totals[r.key])


def test_summary(trace):
    res = serve.Server(workers=2).run(trace)
    s = serve.summarize(res, trace)
    assert s["requests"] == len(trace) and s["p99_ms"] >= s["p50_ms"] > 0


def test_resident_handles(trace, oracle_totals):
    # graphs above 5,000 edges stay on the device after their first request;
    # repeats are counted on those handles, with the same totals
    srv = serve.Server(budget_bytes=4 << 30, workers=3, small_edges=5_000, batch_edges=200_000,
                       resident_bytes=1 << 30)
    res = srv.run(trace)
    alone = serve.Server(workers=1, batching=False).run(trace, realtime=False)
    srv.close()
    assert sum(r.resident for r in res) > 0
    for a, b, r in zip(res, alone, trace):
        assert a.status == 0
        np.testing.assert_array_equal(a.totals, b.totals)
        np.testing.assert_array_equal(a.totals, oracle_totals[r.key])
