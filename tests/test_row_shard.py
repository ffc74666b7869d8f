"""Row-sharded streams: the library's exchange points, exercised with two shards on one GPU.

Each shard is a handle holding an uneven block of the rows of every snapshot (row_offset a
multiple of 128), driven from its own host thread on its own CUDA stream, and given an allreduce
callback.  The callback exchanges through the host: it waits for its stream, copies its partial
buffer out, meets the other shards at a barrier, and every shard writes back the partials added in
shard order (so all shards receive the same bits).  No kernel of one handle waits for the other's.
The library calls the callback after each sketch group (partial sketch, then partial norms) and
in each batch step (the block of partial basis-Gram entries); everything else is replicated.

Checks: both shards return the same J and P, bit for bit; they equal those of an unsharded handle
on the whole rows (FP64: P within 1e-10 relative -- the sketch sums are added in another order;
indices equal, the decision margins on this stream being far from 1e-10); each shard's basis
columns are its rows of the selected snapshots; the sketch equals the oracle's (Omega keyed by
the global row) within 1e-12; with the tensor-core BF16x2 path, the shards agree with each other
bit for bit and with the unsharded handle's sketch within the BF16x2 bar 2e-5 ||a||_2.
"""
import ctypes
import ctypes.util
import os
import threading

import numpy as np
import pytest

from oracle.rid import OnlineRID as Oracle, RIDConfig

pytestmark = pytest.mark.gpu


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so", ctypes.util.find_library("cudart") or "",
                 "/usr/local/cuda/lib64/libcudart.so"):
        if not name:
            continue
        try:
            lib = ctypes.CDLL(name)
            lib.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            lib.cudaStreamSynchronize.argtypes = [ctypes.c_void_p]
            return lib
        except OSError:
            continue
    pytest.skip("libcudart not found")


class HostExchange:
    """allreduce for two shards in one process: host copies and a barrier."""

    def __init__(self, rid, nshards=2):
        self.rt = _cudart()
        self.barrier = threading.Barrier(nshards, timeout=120)
        self.parts = [None] * nshards
        self.calls = [0] * nshards
        self.fns = [rid.RID_ALLREDUCE_FN(self._make(i)) for i in range(nshards)]

    def _make(self, shard):
        def fn(buf, count, stream, user):
            try:
                rt = self.rt
                if rt.cudaStreamSynchronize(ctypes.c_void_p(stream)) != 0:
                    return 1
                host = np.empty(count, dtype=np.float64)
                if rt.cudaMemcpy(ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(buf), host.nbytes, 2) != 0:
                    return 2
                self.parts[shard] = host
                self.barrier.wait()
                total = self.parts[0].copy()
                for part in self.parts[1:]:     # shard order: the same bits on every shard
                    total += part
                self.barrier.wait()
                if rt.cudaMemcpy(ctypes.c_void_p(buf), ctypes.c_void_p(total.ctypes.data), total.nbytes, 1) != 0:
                    return 3
                self.calls[shard] += 1
                return 0
            except Exception:                  # never let an exception cross the C boundary
                self.barrier.abort()
                return 4
        return fn


def _run_shards(A, splits, k, s, h, dtype, sketch, block, seed):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A.shape
    npd = np.float64 if dtype == "f64" else np.float32
    X = torch.from_numpy(np.ascontiguousarray(A.T.astype(npd))).cuda()      # row j = snapshot j
    torch.cuda.synchronize()
    ex = HostExchange(rid, len(splits) - 1)
    out = [None] * (len(splits) - 1)
    errs = []

    def shard(i):
        try:
            r0, r1 = splits[i], splits[i + 1]
            st = torch.cuda.Stream()
            g = rid.OnlineRID(m=r1 - r0, k=k, s=s, h=h, dtype=dtype, sketch=sketch, seed=seed, n_max=n,
                              stream=st, row_offset=r0, m_global=m, allreduce=ex.fns[i])
            for j0 in range(0, n, block):
                g.ingest(X[j0:j0 + block, r0:r1])
            J, P = g.finalize()
            out[i] = (J, P, g.state(0), g.basis(), g.state(3))
            g.close()
        except Exception as e:                   # reported by the main thread
            errs.append(e)
            ex.barrier.abort()

    th = [threading.Thread(target=shard, args=(i,)) for i in range(len(splits) - 1)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    assert not errs, errs
    return out, ex


@pytest.mark.parametrize("seed", [0, 1])
def test_two_fp64_shards_match_whole_handle_and_oracle(seed):
    from paper_2405_16076_gb300 import rid
    from workloads import config1_matrix
    A = config1_matrix(seed)                           # 4096 x 256
    m, n = A.shape
    k, s, h = 20, 83, 30
    splits = [0, 1536, m]                              # uneven, offset a multiple of 128
    out, ex = _run_shards(A, splits, k, s, h, "f64", "native", 7, seed)
    (J0, P0, S0, B0, F0), (J1, P1, S1, B1, F1) = out
    assert np.array_equal(J0, J1) and np.array_equal(P0, P1) and np.array_equal(S0, S1)
    assert ex.calls[0] == ex.calls[1] > 0
    whole = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f64", seed=seed, n_max=n)
    import torch
    Xw = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j0 in range(0, n, 7):
        whole.ingest(Xw[j0:j0 + 7])
    Jw, Pw = whole.finalize()
    Sw = whole.state(0)
    whole.close()
    o = Oracle(RIDConfig(m=m, k=k, s=s, h=h, seed=seed))
    o.ingest(A)
    assert np.abs(S0 - o.S).max() <= 1e-12 * np.abs(o.S).max()
    assert np.abs(S0 - Sw).max() <= 1e-12 * np.abs(Sw).max()
    assert abs(F0[0] - o.fro2) <= 1e-13 * o.fro2
    assert np.array_equal(J0, Jw)
    assert np.linalg.norm(P0 - Pw) <= 1e-10 * np.linalg.norm(Pw)
    for i, j in enumerate(J0):                         # each shard keeps its own rows of the basis
        if j >= 0:
            assert np.array_equal(B0[:, i], A[splits[0]:splits[1], j])
            assert np.array_equal(B1[:, i], A[splits[1]:splits[2], j])


def test_three_bf16x2_shards_agree():
    from paper_2405_16076_gb300 import rid
    rng = np.random.default_rng(4)
    m, n = 200_000, 48
    A = (rng.standard_normal((m, 8)) @ rng.standard_normal((8, n)) + 0.05 * rng.standard_normal((m, n)))
    A = A.astype(np.float32)
    k, s, h = 12, 51, 30
    splits = [0, 60_032, 130_048, m]                   # offsets multiples of 128
    ex_out, ex = _run_shards(A, splits, k, s, h, "f32", "bf16x2", 8, 5)
    J0, P0, S0 = ex_out[0][:3]
    for J, P, S, _, _ in ex_out[1:]:
        assert np.array_equal(J, J0) and np.array_equal(P, P0) and np.array_equal(S, S0)
    import torch
    whole = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f32", sketch="bf16x2", seed=5, n_max=n)
    Xw = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j0 in range(0, n, 8):
        whole.ingest(Xw[j0:j0 + 8])
    whole.finalize()
    Sw = whole.state(0)
    whole.close()
    norms = np.linalg.norm(A.astype(np.float64), axis=0)
    assert (np.abs(S0 - Sw) / norms[None, :]).max() <= 2e-5


def test_shard_configuration_checks():
    from paper_2405_16076_gb300 import rid
    ex = HostExchange(rid)
    with pytest.raises(rid.RIDError):                  # offset not a multiple of 128
        rid.OnlineRID(m=1000, k=5, s=23, h=30, dtype="f64", row_offset=100, m_global=2000, allreduce=ex.fns[0])
    with pytest.raises(rid.RIDError):                  # m_global too small
        rid.OnlineRID(m=1000, k=5, s=23, h=30, dtype="f64", row_offset=128, m_global=1000, allreduce=ex.fns[0])
    with pytest.raises(rid.RIDError):                  # an offset without an exchange
        rid.OnlineRID(m=1000, k=5, s=23, h=30, dtype="f64", row_offset=128, m_global=2000)
