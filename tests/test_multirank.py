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


def _row_shard_worker(rank, world, port, bounds, out):
    """One rank of the row-sharded design: it holds coordinates [lo, hi) of every snapshot,
    sketches them with Omega's columns lo..hi-1 (Omega is keyed by the global coordinate, so no
    rank needs another's part of it), and the partial sketches, squared norms and basis Grams are
    summed across ranks."""
    import torch
    from oracle import philox
    from workloads import config1_matrix
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = config1_matrix(3, m=1000, n=30, r=12)
    lo, hi = bounds[rank], bounds[rank + 1]
    part = philox.omega_block("rademacher", 5, np.arange(35 + 12), lo, hi) @ A[lo:hi]
    nrm = np.sum(A[lo:hi] ** 2, axis=0)
    J = np.array([2, 7, 11, 19])
    gram = A[lo:hi, J].T @ A[lo:hi, J]
    buf = torch.from_numpy(np.concatenate([part.ravel(), nrm, gram.ravel()]))
    dist.all_reduce(buf)
    out[rank] = buf.numpy().copy()
    dist.destroy_process_group()


def test_row_sharded_partial_sketches_sum_to_the_full_sketch():
    """The row-sharded multi-GPU design, with gloo ranks standing in for GPUs: one all-reduce of
    the (s + h) x b partial sketches and norms, and one of the basis-Gram partials, give the
    single-process sketch, ||a_j||^2 and A_J^T A_J, and every rank holds the same sums bit for
    bit, so the batch step that follows runs identically on each rank."""
    from oracle.rid import OnlineRID, RIDConfig
    from workloads import config1_matrix
    world = 2
    bounds = [0, 437, 1000]                           # an uneven split of m = 1000
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_row_shard_worker, args=(world, port, bounds, out), nprocs=world, join=True)
    A = config1_matrix(3, m=1000, n=30, r=12)
    o = OnlineRID(RIDConfig(m=1000, k=8, s=35, h=12, seed=5))
    o.ingest(A)
    rows, n = 35 + 12, 30
    J = np.array([2, 7, 11, 19])
    for rank in range(world):
        got = out[rank]
        S = got[:rows * n].reshape(rows, n)
        nrm = got[rows * n:rows * n + n]
        gram = got[rows * n + n:].reshape(4, 4)
        assert np.abs(S - o.S).max() <= 1e-12 * np.abs(o.S).max()
        assert np.abs(nrm.sum() - o.fro2) <= 1e-13 * o.fro2
        assert np.abs(gram - A[:, J].T @ A[:, J]).max() <= 1e-13 * np.abs(gram).max()
    assert np.array_equal(out[0], out[1])             # every rank holds the same sums
