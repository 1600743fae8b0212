"""The multi-rank bench path on CPU: two gloo ranks on 127.0.0.1. Environments never interact, so
ranks share nothing but the timing reduction: each rank simulates its own envs from its own seed,
and the slowest rank's time sets the whole-job throughput."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2108_10470_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_time = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(my_time, world, "cpu")
    w = W.ant_workload(8)
    root, dof, acts = W.seeded_inputs(w, bench.rank_seed(rank), 2)
    out[rank] = (t, float(dof[:, 0].sum()), bench.weak_value(world, 8, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_use_distinct_seeds():
    world = 2
    port = free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0            # max over ranks
    assert res[0][1] != res[1][1]                    # each rank has its own environments
    assert np.isclose(res[0][2], 2 * 8 * 10 / 2.0)   # whole-job env-steps/s
