"""The GPU range counter of shard.py: three weighted edge ranges counted one
after another on one handle, their raw sums added as the all-reduce would,
equal the oracle's totals; the per-edge rows land in their own rows."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402
from paper_2010_14058_gb300 import shard  # noqa: E402


def test_ranges_sum_to_whole_graph():
    g = graphgen.chung_lu(3000, 20000, 2.1, 900.0, 4, 23, type_zipf=1.2)
    L, m = g["L"], g["m"]
    h = tg.tg_build(*tg.to_device(g), L)
    pe = torch.zeros((m, tg.tg_layout(L, 4)["per_edge_slots"]), dtype=torch.int32, device="cuda")
    count = shard.gpu_range_counter(h, per_edge_out=pe)
    raw = sum(count(b, e) for b, e in shard.edge_ranges(m, 3, shard.edge_weights(g["row_ptr"], g["col"])))
    pe_o, gl_o = oracle.paper(g)
    np.testing.assert_array_equal(tg.tg_finalize_global(L, 4, 1, raw), gl_o)
    np.testing.assert_array_equal(pe.cpu().numpy().view(np.uint32).astype(np.int64), pe_o)
    h.free()
