"""Block-scaled E4M3 tensor-core ingest (FP32 data, FP8 / FP8x2 sketches) against the FP64 oracle.

The oracle writes out the FP8 form's arithmetic (``oracle/fp8.py``): each column is split into
blocks of 32 coordinates, each block scaled by the smallest power of two that keeps its largest
magnitude within 448, rounded to E4M3 (nearest, ties to even); FP8x2 adds the block-scaled E4M3
image of the residual.  The sketch of the quantized data, Omega (hi + lo), is then exact
arithmetic on the same +-1 Omega.  The GPU sums those products in FP32 on the tensor cores
(per CTA over its coordinate range, then in FP64 across CTAs), so its entries must match the
oracle's quantized sketch to FP32 accumulation accuracy: bar 1e-5 ||a||_2 per entry, far below
the quantization error itself (2^-8 relative per coordinate for FP8x2, 2^-4 for FP8), so a wrong
scale, rounding or Omega entry fails it.  Against the unquantized FP64 sketch, FP8x2 entries
carry an error of standard deviation ~2^-8 / sqrt(3) ||a||_2 ~ 2.3e-3 ||a||_2: bar 2e-2 ||a||_2
(about 9 sigma).  Slot copies bit-exact; squared norms from the FP32 data within 1e-6.
"""
import numpy as np
import pytest

from oracle import fp8 as ofp8
from oracle import philox
from oracle.rid import OnlineRID as Oracle, RIDConfig

pytestmark = pytest.mark.gpu

BLOCK = 32


def _mats(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 10)) @ np.diag(0.8 ** np.arange(10)) @ rng.standard_normal((10, n))
    A += 0.05 * rng.standard_normal((m, n))
    # a spread of magnitudes across coordinate blocks, so that the block scales differ
    A *= np.exp2(np.floor(8 * np.sin(np.arange(m) / 997.0)))[:, None]
    return A.astype(np.float32)


def _run_gpu(A32, k, s, h, sketch, block=8, defer=True, offset=0, seed=3):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A32.shape
    g = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f32", sketch=sketch, seed=seed, defer=defer)
    flat = torch.zeros(n * m + offset + 64, dtype=torch.float32, device="cuda")
    X = flat[offset:offset + n * m].view(n, m)
    X.copy_(torch.from_numpy(np.ascontiguousarray(A32.T)))
    for j0 in range(0, n, block):
        g.ingest(X[j0:j0 + block])
    J, P = g.finalize()
    return g, J, P


def _quantized_sketch(A32, rows, seed, two_terms):
    A = A32.astype(np.float64)
    if two_terms:
        hi, lo = ofp8.split_x2(A, BLOCK)
        Q = hi + lo
    else:
        Q = ofp8.quantize_blocked(A, BLOCK)
    Om = philox.omega_block("rademacher", seed, np.arange(rows), 0, A.shape[0])
    return Om @ Q


@pytest.mark.parametrize("sketch", ["fp8x2", "fp8"])
@pytest.mark.parametrize("m,n,k,s,h", [
    (100003, 45, 12, 51, 30),     # one N tile (81 rows -> 96), ragged m, tail batch
    (50000, 130, 100, 403, 50),   # two N tiles (453 rows -> 256 + 208)
    (777, 20, 5, 23, 30),         # m below one 128-coordinate chunk plus a partial one
])
def test_fp8_sketch_against_oracle(sketch, m, n, k, s, h):
    A = _mats(m, n, m + 3 * n)
    g, J, P = _run_gpu(A, k, s, h, sketch)
    S_g = g.state(0)
    norms = np.linalg.norm(A.astype(np.float64), axis=0)
    S_q = _quantized_sketch(A, s + h, 3, sketch == "fp8x2")
    err_q = np.abs(S_g - S_q) / norms[None, :]
    assert err_q.max() <= 1e-5, err_q.max()
    o = Oracle(RIDConfig(m=m, k=k, s=s, h=h, seed=3))
    o.ingest(A.astype(np.float64))
    if sketch == "fp8x2":
        assert (np.abs(S_g - o.S) / norms[None, :]).max() <= 2e-2
    fro = g.state(3)
    assert abs(fro[0] - o.fro2) <= 1e-6 * o.fro2
    B = g.basis()
    for i, j in enumerate(J):
        if j >= 0:
            assert np.array_equal(B[:, i], A[:, j])
    assert P.shape == (k, n) and np.isfinite(P).all()


def test_fp8_group_and_alignment_invariance():
    """A column's FP8x2 sketch does not depend on its group or on its pointer's alignment."""
    A = _mats(70001, 40, 7)
    k, s, h = 10, 43, 30
    g1, J1, P1 = _run_gpu(A, k, s, h, "fp8x2", block=8, defer=False)
    g2, J2, P2 = _run_gpu(A, k, s, h, "fp8x2", block=8, defer=True)
    g3, J3, P3 = _run_gpu(A, k, s, h, "fp8x2", block=3, defer=False, offset=1)
    S1, S2, S3 = g1.state(0), g2.state(0), g3.state(0)
    # a column's partial sums depend only on the coordinate range of each CTA (fixed by m and the
    # batch's CTA count), not on the other columns of its group: bit-identical
    assert np.array_equal(S1, S2) and np.array_equal(S1, S3)
    assert np.array_equal(J1, J2) and np.array_equal(J1, J3)
    assert np.array_equal(P1, P2) and np.array_equal(P1, P3)


def test_fp8_rejects_too_many_rows():
    from paper_2405_16076_gb300 import rid
    with pytest.raises(rid.RIDError):
        rid.OnlineRID(m=1000, k=100, s=403, h=100, dtype="f32", sketch="fp8x2")
