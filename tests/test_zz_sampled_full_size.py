"""Parity at the full size of the channel-flow stream, in the benchmark's launch configuration.

The stream: m = 3 x 192 x 129 x 192 = 14,266,368 coordinates, n = 1000 snapshots ingested in
blocks of 8 from device memory (grouped up to 64 columns per sketch launch), k = t = 100, s = 403
sketch rows, h = 50 NA-Hutch++ probe rows, FP32 data, BF16x2 tensor-core sketches, the data and
sketch seeds of the benchmark's first rank.  The oracle cannot run this stream inside a test (its
sketch alone is 453 x 14.3 M Philox draws per snapshot), so the GPU's results are checked where the
oracle computes them one by one, and by properties that hold at any size:

* sampled sketch entries -- the first and last sketch rows and the first and last probe rows, for
  snapshots in the first and last groups and batches -- against the oracle's rows of Omega times
  the snapshot, in FP64; bar 2e-5 ||a_j||_2, the bar of the small tensor-core parity test (the
  BF16x2 split leaves a residual of at most 2^-16 of each value; the FP32 accumulation adds far
  less);
* the same rows for every snapshot at once, through a seeded +-1 combination c of the snapshots:
  S[R] c = Omega[R] (A c) by linearity; the per-snapshot errors are independent and add in
  quadrature, so the bar is 2e-5 (sum_j ||a_j||^2)^(1/2).  A dropped 64-coordinate tile of one
  snapshot moves the combination by ~2e-3 ||a_j||, well above it;
* ||A_obs||^2 within 1e-6 of the FP64 sum of the snapshots' squared norms;
* the basis columns are bit-exact copies of the snapshots that J names, J holds distinct snapshot
  indices, and empty slots are zero;
* the last batch's Algorithm 4 candidate equals the oracle's Algorithm 4 on the GPU's own sketch
  within 1e-10 kappa (both solve in FP64), and the committed P is the candidate q*, row for row;
* the NA-Hutch++ estimate (Algorithm 8) of the committed result lies within 15 % of its exact
  error ||A - A_J P||_F / ||A||_F, evaluated in FP64.

The module runs after the earlier GPU modules (file order): it holds about 90 GB of device memory
while it runs.
"""
import ctypes
import math

import numpy as np
import pytest

import bench
from oracle import philox
from oracle.rid import coeff_alg4

pytestmark = pytest.mark.gpu

SKETCH_BAR = 2e-5


def _sum_sq(X, rows=25):
    tot = 0.0
    for j0 in range(0, X.shape[0], rows):
        tot += float(X[j0:j0 + rows].double().square().sum().item())
    return tot


@pytest.fixture(scope="module")
def channel_run():
    import torch
    from paper_2405_16076_gb300 import rid
    from workloads import ChannelFlowStream

    cfg = bench.CONFIGS["channel"]
    data_seed, sketch_seed = bench.rank_seeds(0)
    dev = torch.device("cuda", 0)
    n, b, k, s, h = cfg["n"], cfg["b"], cfg["k"], cfg["s"], cfg["h"]
    gen = ChannelFlowStream(seed=data_seed, nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], n=n, device=dev)
    m = gen.m
    X = torch.empty((n, m), dtype=torch.float32, device=dev)       # row j = snapshot j
    for j0 in range(0, n, 50):
        gen.block(j0, min(50, n - j0), out=X[j0:j0 + 50])
    torch.cuda.synchronize()
    st = torch.cuda.Stream(device=dev)
    g = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f32", sketch="bf16x2", n_max=n, seed=sketch_seed,
                      stream=st, defer=True, group_max=64)
    for j0 in range(0, n, b):
        g.ingest(X[j0:j0 + b])
    J, P = g.finalize()
    run = dict(torch=torch, rid=rid, X=X, g=g, J=J, P=P, m=m, n=n, k=k, s=s, h=h, seed=sketch_seed,
               fro2=_sum_sq(X))
    yield run
    g.close()
    run.clear()
    del X
    torch.cuda.empty_cache()


def test_full_size_norms_copies_and_indices(channel_run):
    r = channel_run
    torch, rid, X, g, J = r["torch"], r["rid"], r["X"], r["g"], r["J"]
    m, n, k = r["m"], r["n"], r["k"]
    assert m == 14266368 and J.shape == (k,)
    act = J >= 0
    assert act.any()
    Ja = J[act]
    assert Ja.min() >= 0 and Ja.max() < n and len(np.unique(Ja)) == len(Ja)
    fro2 = g.state(rid.RID_STATE_FRO2)[0]
    assert abs(fro2 - r["fro2"]) <= 1e-6 * r["fro2"], (fro2, r["fro2"])
    B = torch.empty((k, m), dtype=torch.float32, device=X.device)   # row i = basis column i
    rid._check(rid.rid_get_basis(g.h, ctypes.c_void_p(B.data_ptr()), m, 1), g.h)
    for i in range(k):
        if J[i] >= 0:
            assert torch.equal(B[i].view(torch.int32), X[int(J[i])].view(torch.int32)), i
        else:
            assert not bool(B[i].any()), i


def test_full_size_sampled_sketch_against_oracle(channel_run):
    r = channel_run
    torch, X, g = r["torch"], r["X"], r["g"]
    m, n, s, h = r["m"], r["n"], r["s"], r["h"]
    S = g.state(0)                                   # (s + h) x n, unit-variance Omega rows
    assert S.shape == (s + h, n)
    rows = np.array([0, s - 1, s, s + h - 1])
    cols = [0, 63, 64, 517, n - 1]
    c = np.random.default_rng(2405).choice([-1.0, 1.0], size=n)
    V = np.empty((m, len(cols) + 1))
    for q, j in enumerate(cols):
        V[:, q] = X[j].double().cpu().numpy()
    cd = torch.from_numpy(c).to(X.device)
    v = torch.empty(m, dtype=torch.float64, device=X.device)
    step = 1 << 18
    for c0 in range(0, m, step):
        v[c0:c0 + step] = cd @ X[:, c0:c0 + step].double()
    V[:, -1] = v.cpu().numpy()
    ref = np.zeros((len(rows), V.shape[1]))
    chunk = 1 << 20
    for i0 in range(0, m, chunk):
        i1 = min(m, i0 + chunk)
        ref += philox.omega_block("rademacher", r["seed"], rows, i0, i1) @ V[i0:i1]
    norms = np.linalg.norm(V[:, :-1], axis=0)
    err = np.abs(S[np.ix_(rows, cols)] - ref[:, :-1]) / norms[None, :]
    assert err.max() <= SKETCH_BAR, err
    comb = S[rows] @ c
    bar = SKETCH_BAR * math.sqrt(r["fro2"])
    assert np.abs(comb - ref[:, -1]).max() <= bar, (comb - ref[:, -1], bar)


def test_full_size_algorithm4_commit_and_estimate(channel_run):
    r = channel_run
    torch, X, g, J, P = r["torch"], r["X"], r["g"], r["J"], r["P"]
    n, s = r["n"], r["s"]
    S = g.state(0)
    act = np.nonzero(J >= 0)[0]
    na = len(act)
    SA = S[:s] / math.sqrt(s)
    SJ = SA[:, J[act]]
    cand = g.candidates(n)                           # (4, t, n), rows = active slots in slot order
    P4 = coeff_alg4(SJ, SA)
    got = cand[0][:na]
    kap = np.linalg.cond(SJ)
    if kap <= 1e3:
        assert np.linalg.norm(got - P4) <= 1e-10 * max(1.0, kap) * np.linalg.norm(P4), kap
    else:
        # near the rank tolerance of the BF16x2 sketch the two least-squares solutions may differ
        # in directions the sketch does not determine; their residuals still agree
        res_g = np.linalg.norm(SJ @ got - SA)
        res_o = np.linalg.norm(SJ @ P4 - SA)
        assert res_g <= res_o * (1.0 + 1e-2) + 1e-12 * np.linalg.norm(SA), (kap, res_g, res_o)
    sq, fro_est, q = g.error_estimate()
    assert 4 <= q <= 7
    assert P.shape == (r["k"], n)
    assert np.array_equal(P[act], cand[q - 4][:na])
    assert not P[J < 0].any()
    Jd = torch.from_numpy(J).to(X.device)
    Pd = torch.from_numpy(np.ascontiguousarray(P.T)).to(X.device)
    err, fro2 = bench.id_error_device(X, Jd, Pd)
    assert abs(fro2 - r["fro2"]) <= 1e-9 * r["fro2"]
    est = fro_est[0] / math.sqrt(fro2)
    assert abs(est - err) <= 0.15 * err, (est, err, q)
