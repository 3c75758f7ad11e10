"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank solves its
own seeded batch, so the only cross-rank step is the reduction of the timing and
the counts (max of the step times, sum of the solved counts and rates), and the
reference arm prints on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 + r ms over the timed steps, 100 + r solved, 1000 + r solved/s end to end
        res = bench.combine_ranks(dist, world, 10.0 + rank, 100.0 + rank, 1000.0 + rank)
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_combine_ranks_over_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        total_ms, solved, e2e = out[r]
        assert total_ms == 11.0            # the slowest rank sets the job time
        assert solved == 201.0             # every rank's solved trajectories count
        assert e2e == 2001.0               # whole-job end-to-end rate


def test_single_rank_is_the_identity_and_shards_differ():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2408_10731_b300 import scenes
    assert bench.combine_ranks(None, 1, 3.5, 7, 9.0) == (3.5, 7.0, 9.0)
    a, b = scenes.config2(0, n_scenes=2), scenes.config2(1, n_scenes=2)  # ranks 0 and 1
    assert not np.array_equal(a.centers, b.centers) and not np.array_equal(a.xi0, b.xi0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(seed=0, steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
