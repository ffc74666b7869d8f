"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own stream.

Every rank gets distinct seeds (independent problems: weak scaling, no collective on the data
path); the reported time is the slowest rank's, and the whole-job rate counts the units of all
ranks over that time.  The per-rank work here is the CPU oracle on a small stream, so the test
needs no GPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _solve(data_seed, sketch_seed):
    from oracle.rid import OnlineRID, RIDConfig
    from workloads import config1_matrix
    A = config1_matrix(data_seed, m=512, n=40, r=12)
    o = OnlineRID(RIDConfig(m=512, k=8, s=35, h=12, seed=sketch_seed))
    o.ingest(A)
    J, _ = o.finalize()
    return tuple(int(j) for j in J)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    data_seed, sketch_seed = bench.rank_seeds(rank)
    J = _solve(data_seed, sketch_seed)
    ms = 10.0 * (rank + 1)                      # a stand-in time per rank
    t_max = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.whole_job_rate(world, 40, t_max)
    out[rank] = (data_seed, sketch_seed, t_max, rate, J)
    dist.destroy_process_group()


def test_two_gloo_ranks_independent_streams_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] != r1[0] and r0[1] != r1[1]          # distinct seeds: independent problems
    assert r0[2] == r1[2] == 20.0                     # both ranks report the slowest rank's time
    assert np.isclose(r0[3], 2 * 40 / 0.020)          # units of all ranks over that time
    import bench
    for rank, r in ((0, r0), (1, r1)):                 # each rank solved its own problem
        assert tuple(bench.rank_seeds(rank)) == r[:2]
        assert r[4] == _solve(*r[:2])
