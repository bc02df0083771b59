"""The autotuner: every candidate's counts equal the defaults' (it raises
otherwise), the chosen options give the oracle's totals, and the cache
round-trips by workload signature."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402
from paper_2010_14058_gb300 import autotune  # noqa: E402


def test_tune_keeps_counts_and_caches(tmp_path):
    g = graphgen.chung_lu(3000, 20000, 2.1, 900.0, 4, 21, type_zipf=1.2)
    rp, col, ty = tg.to_device(g)
    space = {"light_edge_max_degree": [32, 256], "hub_min_wedges": [300, 1 << 16], "ctas_per_sm": [2, 4]}
    path = str(tmp_path / "tune.json")
    entry = autotune.tune(rp, col, ty, g["L"], space=space, reps=1, path=path)
    new_values = sum(len([v for v in vals if v != autotune.DEFAULTS[k]]) for k, vals in space.items())
    assert len(entry["trials"]) == 1 + new_values                 # defaults, then each other value once
    assert autotune.cached(entry["signature"], path) == entry["options"]
    h = tg.tg_build(rp, col, ty, g["L"], options=entry["options"])
    gl = torch.zeros(tg.tg_layout(g["L"], 4)["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, None, gl)
    assert tg.tg_query_status(h) == 0
    h.free()
    np.testing.assert_array_equal(gl.cpu().numpy(), oracle.paper(g)[1])


def test_tune_batch():
    graphs = [graphgen.chung_lu(400 + 50 * x, 2500 + 300 * x, 2.2, 120.0, 3, 40 + x) for x in range(6)]
    u = graphgen.concat(graphs)
    rp, col, ty = (torch.as_tensor(u[k], device="cuda") for k in ("row_ptr", "col", "types"))
    space = {"light_anchor_max_wedges": [64, 1024], "ctas_per_sm": [2]}
    entry = autotune.tune(rp, col, ty, 3, node_off=u["node_off"], space=space, reps=1, store=False)
    new_values = sum(len([v for v in vals if v != autotune.DEFAULTS[k]]) for k, vals in space.items())
    assert entry["ngraphs"] == 6 and len(entry["trials"]) == 1 + new_values


def test_tune_intersection_modes_per_bucket():
    # the per-bucket intersection choice (binary search / merge / cost model)
    # never changes a count; the tuned choice gives the oracle's totals
    g = graphgen.chung_lu(4000, 40000, 2.1, 1500.0, 3, 23, type_zipf=1.2)
    rp, col, ty = tg.to_device(g)
    space = {f"isect_bucket_{b}": [1, 2, 3] for b in range(4)}
    entry = autotune.tune(rp, col, ty, g["L"], space=space, reps=1, store=False)
    assert len(entry["trials"]) == 1 + 4 * 2
    assert 0 <= entry["options"]["isect_modes"] < 256
    h = tg.tg_build(rp, col, ty, g["L"], options=entry["options"])
    gl = torch.zeros(tg.tg_layout(g["L"], 4)["global_slots"], dtype=torch.int64, device="cuda")
    tg.tg_count(h, 4, None, gl)
    assert tg.tg_query_status(h) == 0
    h.free()
    np.testing.assert_array_equal(gl.cpu().numpy(), oracle.paper(g)[1])
