"""rid_batch_ingest: many independent streams in one call (configuration C5 shapes, scaled down).

Each handle runs the same kernels in the same order whether its columns come through
rid_batch_ingest or rid_ingest, so J and P must agree exactly with the one-by-one runs,
also when every handle has its own CUDA stream and they run concurrently.
"""
import ctypes

import numpy as np
import pytest

from workloads import ImagingStream


def _mk(rid, m, k, seed, stream):
    return rid.OnlineRID(m=m, k=k, s=4 * k + 3, h=30, dtype="f32", sketch="bf16x2", n_max=256, seed=seed,
                         stream=stream)


@pytest.mark.gpu
def test_batch_ingest_matches_individual_runs():
    import torch
    from paper_2405_16076_gb300 import rid
    rng = np.random.default_rng(7)
    specs = []
    for i in range(5):
        m = int(2 ** rng.uniform(14, 17))
        k = int(rng.choice([5, 10, 15]))
        n = int(rng.integers(40, 90))
        specs.append((m, k, n, 100 + i))
    data = []
    for (m, k, n, seed) in specs:
        gen = ImagingStream(seed=seed, m=m, n=n, device="cuda")
        data.append(gen.block(0, n))                                       # row j = snapshot j
    torch.cuda.synchronize()

    streams = [torch.cuda.Stream() for _ in specs]
    batched = [_mk(rid, m, k, seed, st) for (m, k, n, seed), st in zip(specs, streams)]
    b = 8
    nmax = max(n for (_, _, n, _) in specs)
    for j0 in range(0, nmax, b):
        hs, blocks = [], []
        for hd, X, (m, k, n, seed) in zip(batched, data, specs):
            if j0 < n:
                hs.append(hd)
                blocks.append(X[j0:min(n, j0 + b)])
        rid.batch_ingest(hs, blocks)
    res_b = [hd.finalize() for hd in batched]

    for (m, k, n, seed), X, (Jb, Pb) in zip(specs, data, res_b):
        one = _mk(rid, m, k, seed, None)
        for j0 in range(0, n, b):
            one.ingest(X[j0:min(n, j0 + b)])
        Jo, Po = one.finalize()
        assert np.array_equal(Jb, Jo)
        assert np.array_equal(Pb, Po)
        one.close()
    for hd in batched:
        hd.close()


@pytest.mark.gpu
def test_batch_ingest_rejects_null_handle():
    from paper_2405_16076_gb300 import rid
    cols = (ctypes.c_void_p * 1)(None)
    ld = (ctypes.c_int64 * 1)(10)
    nc = (ctypes.c_int32 * 1)(1)
    hs = (ctypes.c_void_p * 1)(None)
    assert rid.rid_batch_ingest(hs, 1, cols, ld, nc, 1) == rid.RID_EINVAL


@pytest.mark.gpu
def test_graph_captured_streams_match_eager_runs():
    """rid_reset, rid_batch_ingest of device columns and the asynchronous device finalize of
    several streams, captured into one CUDA graph: every replay reproduces the eager run's J and
    P exactly."""
    import torch
    from paper_2405_16076_gb300 import rid
    specs = [(20000, 10, 70, 200), (35001, 5, 45, 201), (16384, 15, 61, 202)]
    data = [ImagingStream(seed=seed, m=m, n=n, device="cuda").block(0, n) for (m, k, n, seed) in specs]
    streams = [torch.cuda.Stream() for _ in specs]
    hs = [rid.OnlineRID(m=m, k=k, s=4 * k + 3, h=30, dtype="f32", sketch="bf16x2", n_max=n, seed=seed,
                        stream=st, defer=True) for (m, k, n, seed), st in zip(specs, streams)]
    outs = [(torch.zeros(k, dtype=torch.int64, device="cuda"), torch.zeros((n, k), dtype=torch.float64, device="cuda"))
            for (m, k, n, seed) in specs]
    b = 8
    nmax = max(n for (_, _, n, _) in specs)

    def run(sync):
        for hd in hs:
            hd.reset()
        for j0 in range(0, nmax, b):
            sel = [(hd, X[j0:j0 + b]) for hd, X, (m, k, n, seed) in zip(hs, data, specs) if j0 < n]
            rid.batch_ingest([x[0] for x in sel], [x[1] for x in sel])
        for hd, (J, P) in zip(hs, outs):
            hd.finalize_device(J, P, sync=sync)

    run(True)
    torch.cuda.synchronize()
    ref = [(J.clone(), P.clone()) for J, P in outs]
    for hd in hs:
        hd.reset()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
        fork = torch.cuda.Event()
        fork.record(cap)
        for st in streams:
            st.wait_event(fork)
        run(False)
        for st in streams:
            e = torch.cuda.Event()
            e.record(st)
            cap.wait_event(e)
    for _ in range(2):
        for J, P in outs:
            J.zero_()
            P.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for (J, P), (Jr, Pr) in zip(outs, ref):
            assert torch.equal(J, Jr)
            assert torch.equal(P, Pr)
    for hd in hs:
        hd.sync()                                  # no device error behind the replays
        hd.close()
