"""Multi-rank counting of one graph on CPU: two gloo ranks split the edge
ids, each counts its range (here with the oracle's per-edge routine standing
in for the GPU range counter), the raw sums meet in one all-reduce, and
tg_finalize_global must give the oracle's whole-graph totals."""
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir, weighted):
    import torch.distributed as dist
    from paper_2010_14058_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    g = graphgen.chung_lu(700, 4000, 2.1, 120.0, 3, 17, type_zipf=1.2)
    w = shard.edge_weights(g["row_ptr"], g["col"]) if weighted else None
    tot = shard.count_sharded(lambda b, e: oracle.paper_edges(g, np.arange(b, e))[1], g["L"], g["m"], rank, world,
                              weights=w)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), tot)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("weighted", [False, True])
def test_two_gloo_ranks_match_whole_graph(tmp_path, weighted):
    import torch.multiprocessing as mp

    from paper_2010_14058_gb300 import build
    build.build()                                   # the ranks call tg_finalize_global
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path), weighted), nprocs=2, join=True,
                       start_method="spawn")
    g = graphgen.chung_lu(700, 4000, 2.1, 120.0, 3, 17, type_zipf=1.2)
    want = oracle.paper(g)[1]
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"r{r}.npy"), want)


def test_edge_ranges_cover_and_balance():
    from paper_2010_14058_gb300 import shard
    for m, world in [(0, 3), (10, 1), (10, 4), (1001, 7)]:
        rs = shard.edge_ranges(m, world)
        assert rs[0][0] == 0 and rs[-1][1] == m
        assert all(a[1] == b[0] for a, b in zip(rs[:-1], rs[1:]))
    w = np.array([100.0] + [1.0] * 99)
    rs = shard.edge_ranges(100, 2, w)
    assert rs[0] == (0, 1) and rs[1] == (1, 100)            # the heavy edge alone on rank 0
    g = graphgen.chung_lu(300, 1500, 2.1, 60.0, 2, 3)
    ew = shard.edge_weights(g["row_ptr"], g["col"])
    assert ew.shape == (g["m"],) and ew.min() >= 2
