"""Gradient mode (Sec. 3.4, Eqs. 38-43) and sketches of more than 512 rows on the tensor cores.

The tensor-core ingest holds at most 512 test-matrix rows in one CTA's TMEM, so a longer sketch is
taken in row slices (one pass over the columns each), and gradient mode sketches the stacked
gradient field G a -- materialized per group by the stencil, in the same FP32 arithmetic as the
native path -- with the gradient test matrix Omega_g.  The oracle computes Omega a, Omega_g (G a)
and the norms in FP64 on the same counter-based entries.

Bars, from the BF16x2 split (|a - hi - lo| <= 2^-16 |a|, FP32 accumulation): plain sketch entries
within 2e-5 ||a||_2; leverage sketch entries (Omega a + Omega_g G a) within 2e-5 (||a||_2 +
||G a||_2), where G a itself is rounded to FP32 (relative 2^-24 per entry); ||A_obs||^2 and the
leverage norm within 1e-6 relative (compensated FP32 sums).  Slot copies bit-exact.
"""
import numpy as np
import pytest

from oracle.gradient import grid_gradient_operator
from oracle.rid import OnlineRID as Oracle, RIDConfig
from test_parity_grad import grid_stream

pytestmark = pytest.mark.gpu


def _gpu(A32, k, s, h, sketch, seed, block=8, **kw):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A32.shape
    g = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f32", sketch=sketch, seed=seed, n_max=n, **kw)
    X = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda()
    for j0 in range(0, n, block):
        g.ingest(X[j0:j0 + block])
    J, P = g.finalize()
    return g, J, P


@pytest.mark.parametrize("sketch", ["bf16x2", "bf16"])
def test_tc_gradient_mode_against_oracle(sketch):
    nx, ny, nfields, n = 96, 64, 3, 40
    A = grid_stream(nx, ny, nfields, n, 5).astype(np.float32)
    m = A.shape[0]
    k, s, h, seed = 10, 43, 30, 2
    G = grid_gradient_operator((nx, ny), nfields=nfields)
    o = Oracle(RIDConfig(m=m, k=k, s=s, h=h, seed=seed, grad_op=G))
    o.ingest(A.astype(np.float64))
    g, J, P = _gpu(A, k, s, h, sketch, seed, grad_dims=2, nx=nx, ny=ny, nfields=nfields)
    from paper_2405_16076_gb300 import rid
    S = g.state(rid.RID_STATE_SKETCH)
    L = g.state(rid.RID_STATE_SKETCH_LEV)
    A64 = A.astype(np.float64)
    na = np.linalg.norm(A64, axis=0)
    ng = np.linalg.norm(G @ A64, axis=0)
    bar = 2e-5 if sketch == "bf16x2" else 1e-2
    assert (np.abs(S - o.S) / na[None, :]).max() <= bar
    assert (np.abs(L - o.S_lev) / (na + ng)[None, :]).max() <= bar
    fro = g.state(rid.RID_STATE_FRO2)
    assert abs(fro[0] - o.fro2) <= 1e-6 * o.fro2
    assert abs(fro[1] - o.fro2_lev) <= 1e-6 * o.fro2_lev
    B = g.basis()
    for i, j in enumerate(J):
        if j >= 0:
            assert np.array_equal(B[:, i], A[:, j])
    assert np.isfinite(P).all()
    if sketch == "bf16x2":
        # the native FP32 path on the same stream takes the same decisions
        g2, J2, _ = _gpu(A, k, s, h, "native", seed, grad_dims=2, nx=nx, ny=ny, nfields=nfields)
        assert np.array_equal(J, J2)


def test_tc_sketch_of_more_than_512_rows():
    """s + h = 653 (the ignition configuration's sizes) in two row slices of one pass each."""
    rng = np.random.default_rng(9)
    m, n = 70_003, 40
    A = (rng.standard_normal((m, 8)) @ rng.standard_normal((8, n)) + 0.05 * rng.standard_normal((m, n)))
    A = A.astype(np.float32)
    k, s, h, seed = 150, 603, 50, 4
    o = Oracle(RIDConfig(m=m, k=k, s=s, h=h, seed=seed))
    o.ingest(A.astype(np.float64))
    g, J, P = _gpu(A, k, s, h, "bf16x2", seed)
    S = g.state(0)
    norms = np.linalg.norm(A.astype(np.float64), axis=0)
    assert (np.abs(S - o.S) / norms[None, :]).max() <= 2e-5
    fro = g.state(3)
    assert abs(fro[0] - o.fro2) <= 1e-6 * o.fro2
