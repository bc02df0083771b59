"""The two forms of the set of T in the 4-clique scans, bit-exact against the
oracle (Alg. 3's 4-clique branch through the per-edge rows, Table 3's g12).

Internal ids are (degree, id) ranks.  The scans keep the members of T within
a window of B ids below T's largest member as a bitmap (B = 2^15 for the
CTA-per-edge kernel, 2^13 for the warp-per-edge one) and the members below
the window in a hash set; an edge with more than a quarter of its members
below the window keeps all of them in the hash set, in shared memory or, past
its capacity, in the CTA's global slice.  The graph below puts members of
degree 3-5 below 40,000 filler nodes of degree 6 and members of degree ~300
above them, so that each form is taken by one edge:

  (a, b): |T| = 1,200, 200 below the window        CTA kernel, bitmap + hash
  (c, d): |T| = 4,500, 3,500 below                 CTA kernel, hash in the global slice
  (e, f): |T| = 120, 20 below                      warp kernel, bitmap + hash
  (g, h): |T| = 90, 60 below                       warp kernel, hash

Low members are joined in a path and each to one high member, so the
4-cliques through these edges pair low with low (hash lookups), low with high
and high with high (window lookups).
"""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import gpu_count

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_14058_gb300 as tg  # noqa: E402


def edge_id(g, u, v):
    """Edge id of {u, v}: rank of (min, max) among the pairs u < v in caller ids."""
    u, v = min(u, v), max(u, v)
    rp, col = g["row_ptr"], g["col"]
    upper = np.array([np.count_nonzero(col[rp[x]:rp[x + 1]] > x) for x in range(u)], dtype=np.int64).sum()
    row = np.sort(col[rp[u]:rp[u + 1]])
    row = row[row > u]
    k = int(np.searchsorted(row, v))
    assert k < len(row) and row[k] == v
    return int(upper + k)


def build():
    rng = np.random.default_rng(20201029)
    sizes = {"L1": 200, "L2": 3500, "L3": 20, "L4": 60}
    nxt = 0
    low = {}
    for k, s in sizes.items():                                # low members first: lowest ranks among equals
        low[k] = np.arange(nxt, nxt + s)
        nxt += s
    nf = 40_000
    F = np.arange(nxt, nxt + nf)
    nxt += nf
    H = np.arange(nxt, nxt + 1000)
    nxt += 1000
    a, b, c, d, e, f, g_, h = range(nxt, nxt + 8)
    n = nxt + 8
    edges = []
    for s in (1, 2, 3):                                       # fillers: circulant of degree 6
        edges.append(np.stack([F, F[(np.arange(nf) + s) % nf]], 1))
    iu, ju = np.triu_indices(len(H), 1)
    keep = rng.random(len(iu)) < 0.3
    edges.append(np.stack([H[iu[keep]], H[ju[keep]]], 1))
    for (x, y), hs, lk in (((a, b), H, "L1"), ((c, d), H, "L2"), ((e, f), H[:100], "L3"), ((g_, h), H[100:130], "L4")):
        members = np.concatenate([hs, low[lk]])
        edges.append(np.array([[x, y]]))
        edges.append(np.stack([np.full(len(members), x), members], 1))
        edges.append(np.stack([np.full(len(members), y), members], 1))
        lm = low[lk]
        edges.append(np.stack([lm[:-1], lm[1:]], 1))          # a path through the low members
        edges.append(np.stack([lm, rng.choice(hs, len(lm))], 1))   # each joined to one high member
    E = np.concatenate(edges).astype(np.int64)
    E = np.sort(E, axis=1)
    E = np.unique(E, axis=0)
    types = rng.integers(0, 3, n).astype(np.uint8)
    gr = graphgen.csr_from_edges(n, E[:, 0].astype(np.int32), E[:, 1].astype(np.int32), types, 3,
                                 "4-clique set forms")
    return gr, low, H, (a, b, c, d, e, f, g_, h)


def test_window_and_hash_forms_match_oracle():
    g, low, H, (a, b, c, d, e, f, g_, h) = build()
    deg = np.diff(g["row_ptr"])
    assert deg[low["L2"]].max() <= 5 and deg[H].min() > 6   # low below the fillers, high above
    pairs = [(a, b), (c, d), (e, f), (g_, h), (a, int(H[0])), (c, int(low["L2"][7])), (int(H[3]), int(H[500])),
             (int(low["L2"][10]), int(low["L2"][11])), (e, int(low["L3"][4])), (g_, int(H[110]))]
    pairs = [(u, v) for u, v in pairs if v in set(g["col"][g["row_ptr"][u]:g["row_ptr"][u + 1]].tolist())]
    ids = np.array([edge_id(g, u, v) for u, v in pairs])
    pe, gl, st = gpu_count(g)
    assert st == 0, tg.STATUS[st]
    rows_o, _ = oracle.paper_edges(g, ids)
    np.testing.assert_array_equal(pe[ids], rows_o)
    lay = tg.tg_layout(g["L"], 4)
    g12 = lay["orbit_offset"][12]
    P = g["L"] * (g["L"] + 1) // 2
    assert (pe[ids[:4], g12:g12 + P].sum(axis=1) > 0).all()   # every probed big/small edge has 4-cliques
    # |T| of the four edges, from their triangle slots
    T = pe[ids[:4], g["L"]:2 * g["L"]].sum(axis=1)
    assert list(T) == [1200, 4500, 120, 90]
