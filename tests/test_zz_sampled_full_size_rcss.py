"""Algorithm 1 (online CSS by residual-based sampling, Sec. 2.2.1) at the full size of the
channel-flow stream, in the benchmark's launch configuration.

The stream: m = 3 x 192 x 129 x 192 = 14,266,368 coordinates, n = 1000 snapshots from device
memory in blocks of 8, FP32 data, k = 100 with the subset capped at k columns (Sec. 4.1), xi =
||A - A_k||_F^2 (the smallest value the guarantee allows; every snapshot of this stream then has
p >= 1), the benchmark's data seed and its sketch seed for the uniforms.  The oracle cannot take
the whole stream inside a test, so the GPU's results are checked where the oracle computes them
one by one, and by properties that hold at any size:

* the oracle's decision code replayed on the GPU's own p (keep draws, sigma, steps, the cap)
  reproduces the GPU's selection and sigma exactly -- both take the same FP64 comparisons;
* the GPU's basis is orthonormal and spans C_pre (FP32 storage, two rounds of Gram-Schmidt);
* p of sampled snapshots decided after the basis stopped growing, by the oracle's formula
  (residual formed explicitly, FP64) on the GPU's final basis, within 1e-5 k ||a||^2 / xi (the
  FP32 products over runs of 128 coordinates and the basis' departure from orthonormality).

The module runs after the other full-size modules (file order): it holds about 70 GB of device
memory while it runs.
"""
import ctypes

import numpy as np
import pytest

import bench
from oracle.residual_css import probability, replay

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcss_run():
    import torch
    from paper_2405_16076_gb300 import rid
    from workloads import ChannelFlowStream

    cfg = bench.CONFIGS["channel"]
    data_seed, sketch_seed = bench.rank_seeds(0)
    dev = torch.device("cuda", 0)
    n, b, k = cfg["n"], cfg["b"], cfg["k"]
    gen = ChannelFlowStream(seed=data_seed, nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], n=n, device=dev)
    m = gen.m
    X = torch.empty((n, m), dtype=torch.float32, device=dev)       # row j = snapshot j
    for j0 in range(0, n, 50):
        gen.block(j0, min(50, n - j0), out=X[j0:j0 + 50])
    G = torch.zeros((n, n), dtype=torch.float64, device=dev)
    for c0 in range(0, m, 1 << 16):
        Xc = X[:, c0:c0 + (1 << 16)]
        G += (Xc @ Xc.T).double()
    ev = torch.linalg.eigvalsh(G.cpu()).flip(0)
    xi = float(ev[k:].sum())
    st = torch.cuda.Stream(device=dev)
    g = rid.ResidualCSS(m, k, xi, seed=sketch_seed, data_dtype=rid.RID_F32, cap=k, stop_at_cap=True,
                        cuda_stream=st.cuda_stream)
    for j0 in range(0, n, b):
        g.ingest(X[j0:j0 + b])
    sel, sigma, nb = g.selection()
    p = g.probabilities()
    Q = torch.empty((max(nb, 1), m), dtype=torch.float32, device=dev)   # row i = basis vector i
    if nb:
        rid._check(rid.rid_rcss_basis(g.h, ctypes.c_void_p(Q.data_ptr()), m, 1))
    run = dict(torch=torch, X=X, Q=Q[:nb], sel=sel, sigma=sigma, nb=nb, p=p, m=m, n=n, k=k, xi=xi,
               seed=sketch_seed)
    yield run
    g.close()
    run.clear()
    del X, Q
    torch.cuda.empty_cache()


def test_full_size_rcss_decisions_replay_exactly(rcss_run):
    r = rcss_run
    assert r["m"] == 14266368 and len(r["p"]) == r["n"]
    sel, sigma, steps = replay(r["p"], r["seed"], limit=r["k"])
    np.testing.assert_array_equal(r["sel"], sel)
    assert r["sigma"] == sigma
    assert len(sel) == r["k"]                        # the cap was reached
    assert np.all(r["p"] >= 0)


def test_full_size_rcss_basis_orthonormal_and_spans_c_pre(rcss_run):
    r = rcss_run
    torch, X, Q, nb = r["torch"], r["X"], r["Q"], r["nb"]
    _, _, steps = replay(r["p"], r["seed"], limit=r["k"])
    pre = [j for j in r["sel"] if j <= max(steps)]
    assert 0 < nb <= len(pre)
    Gq = torch.zeros((nb, nb), dtype=torch.float64, device=X.device)
    C = torch.zeros((nb, len(pre)), dtype=torch.float64, device=X.device)
    nrm = torch.zeros(len(pre), dtype=torch.float64, device=X.device)
    idx = torch.tensor(pre, device=X.device)
    for c0 in range(0, r["m"], 1 << 18):
        Qc = Q[:, c0:c0 + (1 << 18)].double()
        Sc = X[idx, c0:c0 + (1 << 18)].double()
        Gq += Qc @ Qc.T
        C += Qc @ Sc.T
        nrm += Sc.square().sum(dim=1)
    dev = (Gq - torch.eye(nb, dtype=torch.float64, device=X.device)).abs().max().item()
    assert dev <= 1e-4, dev
    # ||a - Q Q^T a||^2 = ||a||^2 - ||Q^T a||^2 for an orthonormal Q (to the deviation above)
    res = (nrm - C.square().sum(dim=0)).clamp(min=0) / nrm
    assert res.max().item() <= 1e-3, res.max().item()


def test_full_size_rcss_sampled_p_against_oracle(rcss_run):
    r = rcss_run
    torch, X, Q = r["torch"], r["X"], r["Q"]
    _, _, steps = replay(r["p"], r["seed"], limit=r["k"])
    # the basis stops growing at the step that holds the k-th selection
    last = min(j for j in steps if j >= r["sel"][-1])
    cand = [last + 1, (last + 1 + r["n"] - 1) // 2, r["n"] - 1]
    Qh = Q.cpu().numpy().astype(np.float64).T       # m x nb
    for j in cand:
        a = X[j].double().cpu().numpy()
        po = probability(a, Qh, r["k"], r["xi"])
        scale = r["k"] * float(a @ a) / r["xi"]
        assert abs(r["p"][j] - po) <= 1e-5 * scale, (j, r["p"][j], po, scale)
