"""The diagnostic work counters (tg_set_work_counting / tg_get_work): they
change no count, and the hub pass's wedge counter equals the degree-priority
wedges of the hub anchors computed on the host from their definition (the
anchors u with more than hub_min_wedges wedges u - v - w, v and w of lower
(degree, id) priority than u; Sec. 4's 4-cycle search restated with a
degree order)."""
import importlib.util
import os

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_for_work", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def run(g, options, counting):
    rp, col, ty = tg.to_device(g)
    h = tg.tg_build(rp, col, ty, g["L"], options=options)
    lay = tg.tg_layout(g["L"], 4)
    pe = torch.zeros((h.m, lay["per_edge_slots"]), dtype=torch.int32, device="cuda")
    gl = torch.zeros(lay["global_slots"], dtype=torch.int64, device="cuda")
    if counting:
        tg.tg_set_work_counting(h, True)
    tg.tg_count(h, 4, pe, gl)
    assert tg.tg_query_status(h) == 0
    work = tg.tg_get_work(h) if counting else None
    h.free()
    return pe, gl, work


@pytest.mark.parametrize("hub_min", [1 << 10, 1 << 12])
def test_work_counting_changes_nothing_and_counts_hub_wedges(bench, hub_min):
    g = graphgen.chung_lu(20000, 150000, 2.1, 2500.0, 4, 77)
    opts = {"hub_min_wedges": hub_min}
    pe0, gl0, _ = run(g, opts, False)
    pe1, gl1, work = run(g, opts, True)
    assert torch.equal(pe0, pe1) and torch.equal(gl0, gl1)
    units = bench.kernel_units(g, 64, hub_min)
    assert units["hubs"] > 0
    assert work["hub_wedges"] == int(units["wedges_hub"])
    # one update per (wedge, type) and per (item, round, type) at most
    assert 0 < work["hub_slot_updates"] <= 2 * g["L"] * work["hub_wedges"]
    assert work["hub_fill_cycles"] > 0 and work["hub_read_cycles"] > 0
    assert work["clique_probes"] + work["clique_big_probes"] > 0
