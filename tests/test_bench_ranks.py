"""bench.py's multi-rank path on the host (two gloo ranks): replicas over
colourings get disjoint colourings that together are the stream's first
world * B, and the step time reported is the largest rank's."""
import os
import socket

import numpy as np

import sg2v_inputs as si

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys

    import torch
    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(torch, 1.5 + rank, dist)
        cols = bench.rank_colourings(300, 7, 3, rank, seed=4)
        np.save(os.path.join(out_dir, f"cols{rank}.npy"), cols)
        with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert float(open(tmp_path / f"max{r}.txt").read()) == 2.5
    c0, c1 = np.load(tmp_path / "cols0.npy"), np.load(tmp_path / "cols1.npy")
    assert np.array_equal(np.concatenate([c0, c1]), si.colourings(300, 7, 6, seed=4))
    assert not any(np.array_equal(a, b) for a in c0 for b in c1)


def test_one_process_is_unchanged():
    import sys

    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    import bench

    assert bench.max_over_ranks(torch, 3.25, None) == 3.25
    assert np.array_equal(bench.rank_colourings(100, 5, 4, 0, seed=1), si.colourings(100, 5, 4, seed=1))
