"""The multi-GPU replica bookkeeping on CPU: two gloo ranks each time a different
(seeded) hologram workload, the slowest rank's time sets the whole-job throughput, and
every rank sees the same aggregate (the benchmark's max-over-ranks protocol)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2511_15022_gb300 import inputs
    from paper_2511_15022_gb300.replicas import (aggregate_throughput, max_over_ranks,
                                                 rank_info, replica_seed)
    ri = rank_info()
    dist.init_process_group("gloo", rank=ri.rank, world_size=ri.world)
    w = inputs.small_256()
    p = inputs.params_for(w, seed=replica_seed(w.seed, ri.rank))
    dist.barrier()
    ms = [100.0 + 50.0 * ri.rank, 120.0 - 10.0 * ri.rank]   # per-rank times (fake)
    mx = max_over_ranks(ms)
    out[ri.rank] = (float(p["theta"][0]), mx, aggregate_throughput(10, ri.world, mx[0]),
                    ri.is_root)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_share_the_max_time():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    assert res[0][0] != res[1][0]                      # different holograms per rank
    assert res[0][1] == res[1][1] == [150.0, 120.0]    # element-wise max over ranks
    assert res[0][2] == res[1][2] == pytest.approx(2 * 10 / 0.150)
    assert res[0][3] and not res[1][3]


def test_single_process_needs_no_group():
    from paper_2511_15022_gb300.replicas import aggregate_throughput, max_over_ranks
    assert max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert aggregate_throughput(5, 1, 500.0) == pytest.approx(10.0)
