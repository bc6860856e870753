"""The multi-rank bench path on the CPU (gloo, world size 2): each rank
renders its own camera set over its own copy of the bricks (replicas, no
data-path collective); the whole-job figures are the max over ranks of the
timed intervals and the sum over ranks of the samples."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank timings and work counts, as run_ours produces them
        times = [10.0 + rank, 4.0 + 2 * rank, 6.0 - rank]
        counts = [1000 * (rank + 1), 700 * (rank + 1), 3]
        dist.barrier()
        t, c = bench.reduce_over_ranks(dist, torch.device("cpu"), times, counts)
        cams = bench._cameras(bench.CONFIGS["batched"], rank)
        eyes = np.array([c_.eye for c_ in cams])
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), t=np.array(t), c=np.array(c), eyes=eyes)
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        r0, r1 = (np.load(os.path.join(d, "rank%d.npz" % r)) for r in (0, 1))
    # every rank sees the same whole-job figures
    np.testing.assert_array_equal(r0["t"], r1["t"])
    np.testing.assert_array_equal(r0["c"], r1["c"])
    np.testing.assert_array_equal(r0["t"], [11.0, 6.0, 6.0])        # max over ranks
    np.testing.assert_array_equal(r0["c"], [3000.0, 2100.0, 6.0])   # sum over ranks
    # replicas render different camera sets (seeded by rank), 16 each
    assert r0["eyes"].shape == (16, 3) and r1["eyes"].shape == (16, 3)
    assert not np.allclose(r0["eyes"], r1["eyes"])


def test_single_process_reduce_is_identity():
    t, c = bench.reduce_over_ranks(None, None, [1.5, 2.5], [7, 9])
    assert t == [1.5, 2.5] and c == [7, 9]
    # the cameras of one rank are deterministic
    a = bench._cameras(bench.CONFIGS["diff"], 1)
    b = bench._cameras(bench.CONFIGS["diff"], 1)
    assert [x.eye for x in a] == [x.eye for x in b]
