"""The optional right sketch Y = sum_j a_j omega_j^T (m x l; not part of the paper's method).

GPU against the oracle on the same seeded stream: FP64 within 1e-12 of max|Y| (the same
additions in the same snapshot order, fused multiply-adds on the GPU); FP32 data within
1e-5 x (|A| |W|) entrywise: on the native path the bound of n FP32 roundings of the running sums;
on tensor-core handles (a +-1 W) the BF16x2 split leaves at most 2^-18 of each value per term
(3.8e-6) and each group's FP32 accumulation and its FP32 addition to Y add rounding of the same
order, within the same bound.  Also: l > 256 (two column blocks), reset, checkpoint and
restore, and the error for a handle without a right sketch.
"""
import numpy as np
import pytest

from oracle import philox
from oracle.rid import OnlineRID as Oracle, RIDConfig

pytestmark = pytest.mark.gpu


def _stream(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 6)) @ rng.standard_normal((6, n)) + 0.1 * rng.standard_normal((m, n))
    return A


def _gpu(A, dtype, sketch, omega, l, seed, block=8, **kw):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A.shape
    g = rid.OnlineRID(m=m, k=10, s=43, h=30, dtype=dtype, sketch=sketch, omega=omega, seed=seed, n_max=n,
                      right_l=l, **kw)
    X = torch.from_numpy(np.ascontiguousarray(A.T, dtype=np.float64 if dtype == "f64" else np.float32)).cuda()
    for j0 in range(0, n, block):
        g.ingest(X[j0:j0 + block])
    return g, X


@pytest.mark.parametrize("omega", ["rademacher", "gaussian"])
def test_right_sketch_fp64_matches_oracle(omega):
    A = _stream(5003, 70, 1)
    o = Oracle(RIDConfig(m=5003, k=10, s=43, h=30, omega_kind=omega, seed=4, right_l=21))
    o.ingest(A)
    g, _ = _gpu(A, "f64", "native", omega, 21, 4)
    Y = g.right_sketch()
    assert Y.shape == o.Y.shape
    assert np.abs(Y - o.Y).max() <= 1e-12 * np.abs(o.Y).max()
    g.close()


@pytest.mark.parametrize("sketch,m", [("native", 70001), ("bf16x2", 70001), ("bf16x2", 70000)])
def test_right_sketch_fp32_within_rounding(sketch, m):
    # m = 70000 keeps every column 16-byte aligned (vector loads; the last tile is partial)
    A = _stream(m, 90, 2).astype(np.float32).astype(np.float64)
    l = 300                                           # two blocks of sketch columns
    o = Oracle(RIDConfig(m=A.shape[0], k=10, s=43, h=30, seed=9, right_l=l))
    o.ingest(A)
    g, _ = _gpu(A, "f32", sketch, "rademacher", l, 9, block=16)
    Y = g.right_sketch().astype(np.float64)
    W = philox.omega_block("rademacher", 9, np.arange(l), 0, A.shape[1], right=True).T
    bound = 1e-5 * (np.abs(A) @ np.abs(W))
    assert np.all(np.abs(Y - o.Y) <= bound + 1e-30)
    g.close()


def test_right_sketch_reset_checkpoint_and_errors():
    from paper_2405_16076_gb300 import rid
    A = _stream(3001, 60, 3)
    o = Oracle(RIDConfig(m=3001, k=10, s=43, h=30, seed=5, right_l=13))
    o.ingest(A)
    g, X = _gpu(A[:, :25], "f64", "native", "rademacher", 13, 5)
    state = g.checkpoint()
    g2 = rid.OnlineRID(m=3001, k=10, s=43, h=30, dtype="f64", seed=5, n_max=60, right_l=13)
    g2.restore(state)
    import torch
    X2 = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j0 in range(25, 60, 8):
        g2.ingest(X2[j0:min(60, j0 + 8)])
    assert np.abs(g2.right_sketch() - o.Y).max() <= 1e-12 * np.abs(o.Y).max()
    g2.reset()
    assert np.all(g2.right_sketch() == 0.0)
    g3 = rid.OnlineRID(m=3001, k=10, s=43, h=30, dtype="f64", seed=5, n_max=60)
    with pytest.raises(rid.RIDError):
        g3.right_sketch()
    for h in (g, g2, g3):
        h.close()
