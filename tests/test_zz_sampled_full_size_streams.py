"""Parity at the full size of the 64-stream batched workload, in the benchmark's launch
configuration.

The workload: the 64 streams of ``workloads.batched_streams_spec(seed=0)`` (m log-uniform in
[2^16, 2^21], n in [100, 1000], k in {10, 30, 60}, s = 4k + 3, h = 30, half imaging- and half
flow-shaped, FP32 data, BF16x2 sketches), each handle on its own CUDA stream with device input
grouped up to 64 columns, stepped together through rid_batch_ingest in blocks of 8 -- the eager
form of the benchmark's step (its CUDA-graph replays reproduce these results exactly, which
``test_batch_ingest`` checks).  Checks:

* every stream: valid distinct indices, ||A_obs||^2 within 1e-6 of the FP64 sum, the basis
  columns bit-exact copies of the snapshots J names, the committed P equal to candidate q*;
* three streams -- the smallest imaging stream (m = 68,963: ragged against every tile), the
  smallest flow stream, and the largest stream (m = 2,076,971) -- run again alone through
  rid_ingest give the same J and P bit for bit;
* the two small streams' whole sketches (all s + h rows, every snapshot) against the oracle's
  Omega times the data in FP64, bar 2e-5 ||a_j||_2 (the small tensor-core parity test's bar);
  the large stream's sketch at sampled rows for sampled snapshots, and for every snapshot
  through a seeded +-1 combination (bar 2e-5 of the combined norm), as in the channel-flow module;
* the last batch's Algorithm 4 candidate of these three streams against the oracle's
  Algorithm 4 on the GPU's own sketch, where the basis is well enough conditioned for the two to
  be comparable (kappa <= 1e3, bar 1e-10 kappa).
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import philox
from oracle.rid import coeff_alg4

pytestmark = pytest.mark.gpu

BAR = 2e-5
H = 30
BLOCK = 8


def _sum_sq(X, rows=25):
    """sum of squares of the snapshots (rows of X) in FP64, a few rows at a time"""
    tot = 0.0
    for j0 in range(0, X.shape[0], rows):
        tot += float(X[j0:j0 + rows].double().square().sum().item())
    return tot


def _handle(rid, sp, stream):
    k = sp["k"]
    return rid.OnlineRID(m=sp["m"], k=k, s=4 * k + 3, h=H, dtype="f32", sketch="bf16x2", n_max=sp["n"],
                         seed=sp["seed"], stream=stream, defer=True, group_max=64)


@pytest.fixture(scope="module")
def streams_run():
    import torch
    from paper_2405_16076_gb300 import rid
    from workloads import ImagingStream, LowRankStream, batched_streams_spec

    torch.cuda.empty_cache()
    dev = torch.device("cuda", 0)
    spec = batched_streams_spec(seed=0, nstreams=64)
    data = []
    for sp in spec:
        gen = (ImagingStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device=dev) if sp["kind"] == "imaging"
               else LowRankStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device=dev))
        X = torch.empty((sp["n"], sp["m"]), dtype=torch.float32, device=dev)    # row j = snapshot j
        for j0 in range(0, sp["n"], 100):
            gen.block(j0, min(100, sp["n"] - j0), out=X[j0:j0 + 100])
        data.append(X)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(device=dev) for _ in spec]
    hs = [_handle(rid, sp, st) for sp, st in zip(spec, streams)]
    nmax = max(sp["n"] for sp in spec)
    for j0 in range(0, nmax, BLOCK):
        sel = [(hd, X[j0:j0 + BLOCK]) for hd, X, sp in zip(hs, data, spec) if j0 < sp["n"]]
        rid.batch_ingest([x[0] for x in sel], [x[1] for x in sel])
    res = [hd.finalize() for hd in hs]
    img = [i for i, sp in enumerate(spec) if sp["kind"] == "imaging"]
    flow = [i for i, sp in enumerate(spec) if sp["kind"] == "flow"]
    chosen = [min(img, key=lambda i: spec[i]["m"]), min(flow, key=lambda i: spec[i]["m"]),
              max(range(len(spec)), key=lambda i: spec[i]["m"])]
    run = dict(torch=torch, rid=rid, spec=spec, data=data, hs=hs, res=res, chosen=chosen)
    yield run
    for hd in hs:
        hd.close()
    run.clear()
    del data
    torch.cuda.empty_cache()


def test_streams_full_size_properties_of_every_stream(streams_run):
    r = streams_run
    torch, rid = r["torch"], r["rid"]
    assert len(r["spec"]) == 64
    for sp, X, hd, (J, P) in zip(r["spec"], r["data"], r["hs"], r["res"]):
        m, n, k = sp["m"], sp["n"], sp["k"]
        act = J >= 0
        assert act.any()
        Ja = J[act]
        assert Ja.min() >= 0 and Ja.max() < n and len(np.unique(Ja)) == len(Ja), sp
        ref = _sum_sq(X)
        fro2 = hd.state(rid.RID_STATE_FRO2)[0]
        assert abs(fro2 - ref) <= 1e-6 * ref, (sp, fro2, ref)
        B = torch.empty((k, m), dtype=torch.float32, device=X.device)
        rid._check(rid.rid_get_basis(hd.h, ctypes.c_void_p(B.data_ptr()), m, 1), hd.h)
        for i in range(k):
            if J[i] >= 0:
                assert torch.equal(B[i].view(torch.int32), X[int(J[i])].view(torch.int32)), (sp, i)
        del B
        cand = hd.candidates(n)
        _, _, q = hd.error_estimate()
        assert 4 <= q <= 7
        assert np.array_equal(P[act], cand[q - 4][:int(act.sum())]), sp
        assert not P[~act].any() and np.isfinite(P).all(), sp


def test_streams_full_size_batched_equals_individual(streams_run):
    r = streams_run
    rid = r["rid"]
    for i in r["chosen"]:
        sp, X = r["spec"][i], r["data"][i]
        one = _handle(rid, sp, None)
        for j0 in range(0, sp["n"], BLOCK):
            one.ingest(X[j0:j0 + BLOCK])
        J1, P1 = one.finalize()
        one.close()
        Jb, Pb = r["res"][i]
        assert np.array_equal(J1, Jb) and np.array_equal(P1, Pb), sp


def test_streams_full_size_sketches_against_oracle(streams_run):
    r = streams_run
    torch = r["torch"]
    small, large = r["chosen"][:2], r["chosen"][2]
    for i in small:
        sp, X, hd = r["spec"][i], r["data"][i], r["hs"][i]
        m, n, s = sp["m"], sp["n"], 4 * sp["k"] + 3
        A = X.double().cpu().numpy().T                                   # m x n
        Om = philox.omega_block("rademacher", sp["seed"], np.arange(s + H), 0, m)
        ref = Om @ A
        S = hd.state(0)
        assert S.shape == ref.shape
        err = np.abs(S - ref) / np.linalg.norm(A, axis=0)[None, :]
        assert err.max() <= BAR, (sp, err.max())
    sp, X, hd = r["spec"][large], r["data"][large], r["hs"][large]
    m, n, s = sp["m"], sp["n"], 4 * sp["k"] + 3
    S = hd.state(0)
    rows = np.array([0, s - 1, s, s + H - 1])
    cols = [0, 63, 64, n // 2, n - 1]
    c = np.random.default_rng(2407).choice([-1.0, 1.0], size=n)
    V = np.empty((m, len(cols) + 1))
    for q, j in enumerate(cols):
        V[:, q] = X[j].double().cpu().numpy()
    cd = torch.from_numpy(c).to(X.device)
    V[:, -1] = np.concatenate([(cd @ X[:, c0:c0 + (1 << 18)].double()).cpu().numpy()
                               for c0 in range(0, m, 1 << 18)])
    ref = np.zeros((len(rows), V.shape[1]))
    for i0 in range(0, m, 1 << 20):
        i1 = min(m, i0 + (1 << 20))
        ref += philox.omega_block("rademacher", sp["seed"], rows, i0, i1) @ V[i0:i1]
    err = np.abs(S[np.ix_(rows, cols)] - ref[:, :-1]) / np.linalg.norm(V[:, :-1], axis=0)[None, :]
    assert err.max() <= BAR, err
    assert np.abs(S[rows] @ c - ref[:, -1]).max() <= BAR * math.sqrt(_sum_sq(X))


def test_streams_full_size_algorithm4_on_gpu_sketch(streams_run):
    r = streams_run
    for i in r["chosen"]:
        sp, hd = r["spec"][i], r["hs"][i]
        J, _ = r["res"][i]
        n, s = sp["n"], 4 * sp["k"] + 3
        act = np.nonzero(J >= 0)[0]
        SA = hd.state(0)[:s] / math.sqrt(s)
        SJ = SA[:, J[act]]
        got = hd.candidates(n)[0][:len(act)]
        assert np.isfinite(got).all()
        kap = np.linalg.cond(SJ)
        if kap <= 1e3:
            P4 = coeff_alg4(SJ, SA)
            assert np.linalg.norm(got - P4) <= 1e-10 * max(1.0, kap) * np.linalg.norm(P4), (sp, kap)
