"""Algorithm 1 (online CSS by residual-based sampling, Sec. 2.2.1) on the GPU against the oracle.

Every decision is a comparison of a uniform with p_a, of p_a with 1, or of sigma with 1; where the
oracle's value lies within the GPU path's rounding of such a threshold, both answers are right,
so the comparison runs up to the first such near tie (whose position is checked to leave most of
the stream), and after it checks only that the GPU's selection is valid.
"""
import numpy as np
import pytest

from oracle.residual_css import ResidualCSS as Oracle, uniform
from workloads import config1_matrix

gpu = pytest.mark.gpu


def _lib():
    torch = pytest.importorskip("torch")
    from paper_2405_16076_gb300 import rid
    return torch, rid


def first_near_tie(o, A, k, xi, rel):
    """Index of the first column whose decision lies within rel * k ||a||^2 / xi of a threshold
    (u against min(p, 1), p against 1, sigma against 1) in the oracle's run, else n."""
    sigma, since = 0.0, 0
    for j in range(A.shape[1]):
        scale = k * float(A[:, j] @ A[:, j]) / xi
        tol = rel * max(scale, 1e-300)
        p = o.p[j]
        u = uniform(o.seed, j)
        if abs(u - min(p, 1.0)) <= tol or abs(p - 1.0) <= tol:
            return j
        if p < 1.0:
            sigma += p
            since += 1
            if abs(sigma - 1.0) <= tol * since:      # the p errors summed since the last reset
                return j
        if p >= 1.0 or sigma >= 1.0:
            sigma, since = 0.0, 0
    return A.shape[1]


def run_gpu(A, k, xi, seed, dtype, blocks=None, on_device=True, cap=512, limit=None):
    torch, rid = _lib()
    m, n = A.shape
    g = rid.ResidualCSS(m, k, xi, seed=seed, data_dtype=rid.RID_F64 if dtype == np.float64 else rid.RID_F32,
                        cap=limit or cap, stop_at_cap=limit is not None)
    X = np.asfortranarray(A.astype(dtype))
    cuts = [0] + list(np.cumsum(blocks or [n]))
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        if on_device:
            g.ingest(torch.from_numpy(X[:, a:b].T.copy()).cuda())
        else:
            g.ingest(np.asfortranarray(X[:, a:b]))
    sel, sigma, nb = g.selection()
    p = g.probabilities()
    Q = g.basis()
    g.close()
    return sel, sigma, nb, p, Q


def check(A, k, xi, seed, dtype, rel, min_frac=0.5, limit=None, **kw):
    o = Oracle(A.shape[0], k, xi, seed, limit=limit)
    o.ingest(A.astype(dtype).astype(np.float64))
    sel, sigma, nb, p, Q = run_gpu(A, k, xi, seed, dtype, limit=limit, **kw)
    n = A.shape[1]
    t = first_near_tie(o, A.astype(dtype).astype(np.float64), k, xi, rel)
    assert t >= min_frac * n, f"near tie at column {t} of {n}"
    assert len(p) == n
    scale = k * np.einsum("ij,ij->j", A, A) / xi
    op = np.array(o.p)
    np.testing.assert_array_less(np.abs(p[:t] - op[:t]), rel * scale[:t] + 1e-300)
    osel = o.selection()
    np.testing.assert_array_equal(sel[sel < t], osel[osel < t])
    if t == n:
        np.testing.assert_array_equal(sel, osel)
        assert nb == o.Q.shape[1]
        assert abs(sigma - o.sigma) <= rel * max(scale.max(), 1.0) * n
        if nb:
            # same span, orthonormal
            np.testing.assert_allclose(Q.astype(np.float64).T @ Q.astype(np.float64), np.eye(nb),
                                       atol=1e3 * np.finfo(dtype).eps)
            P1 = Q.astype(np.float64) @ Q.astype(np.float64).T
            P2 = o.Q @ o.Q.T
            assert np.abs(P1 - P2).max() <= 1e3 * np.finfo(dtype).eps
    assert np.all(np.diff(sel) > 0) and (len(sel) == 0 or (sel[0] >= 0 and sel[-1] < n))
    return sel, o


@gpu
def test_rcss_fp64_parity_low_rank_plus_noise():
    """m = 3000 (23 runs of 128 and a ragged tail), 400 columns of rank 40 plus noise; xi is half
    of k times the median squared column norm, so the first column ends a step at once (p >= 1)
    and the later ones by residual mass (sigma >= 1): 89 selected over 68 steps."""
    A = config1_matrix(5, m=3000, n=400, r=40, noise_var=1e-7)
    k = 10
    xi = 0.5 * k * float(np.median(np.einsum("ij,ij->j", A, A)))
    sel, o = check(A, k, xi, 7, np.float64, rel=1e-12, min_frac=1.0)
    assert len(o.steps) >= 30 and 30 <= len(sel) <= 200
    assert any(o.p[j] >= 1.0 for j in o.steps) and any(o.p[j] < 1.0 for j in o.steps)


@gpu
def test_rcss_fp64_parity_ragged_blocks_and_host_input():
    """Blocks of 1, 63, 64, 65 and the rest, from host memory: the decisions do not depend on how
    the stream is cut nor on where the columns live.  p agrees to rounding only: after a step's end
    the dots of the new basis vector with the rest of a block are thin products, summed in another
    order than the block's first dots."""
    A = config1_matrix(6, m=1000, n=300, r=25, noise_var=1e-7)
    k = 8
    xi = 0.5 * k * float(np.median(np.einsum("ij,ij->j", A, A)))
    ref = run_gpu(A, k, xi, 3, np.float64)
    cut = run_gpu(A, k, xi, 3, np.float64, blocks=[1, 63, 64, 65, 107], on_device=False)
    np.testing.assert_array_equal(ref[0], cut[0])
    scale = k * np.einsum("ij,ij->j", A, A) / xi
    np.testing.assert_array_less(np.abs(ref[3] - cut[3]), 1e-12 * scale)
    assert abs(ref[1] - cut[1]) <= 1e-12 * scale.max() * A.shape[1] and ref[2] == cut[2]
    check(A, k, xi, 3, np.float64, rel=1e-12, min_frac=1.0, blocks=[1, 63, 64, 65, 107])


@gpu
def test_rcss_fp32_parity_prefix():
    """FP32 data: products in FP32 over runs of 128, basis in FP32."""
    A = config1_matrix(5, m=3000, n=400, r=40, noise_var=1e-7).astype(np.float32).astype(np.float64)
    k = 10
    xi = 0.5 * k * float(np.median(np.einsum("ij,ij->j", A, A)))
    check(A, k, xi, 11, np.float32, rel=1e-5, min_frac=0.5)


@gpu
def test_rcss_rank_r_stream_greedy_and_exact_span():
    """Rank 7 stream with xi far below its energy: the first maximal independent set in arrival
    order is selected, the basis spans the stream's range, and the dependent columns that join
    C_cur within a step add no direction."""
    rng = np.random.default_rng(4)
    B = rng.standard_normal((700, 7))
    A = B @ rng.standard_normal((7, 90))
    A[:, 3] = A[:, 1] * 2.0          # an exact repeat
    xi = 1e-4 * 5 * float(np.min(np.einsum("ij,ij->j", A, A)))
    sel, o = check(A, 5, xi, 2, np.float64, rel=1e-12, min_frac=1.0)
    ranks = [np.linalg.matrix_rank(A[:, :j + 1]) for j in range(A.shape[1])]
    greedy = [j for j in range(A.shape[1]) if ranks[j] > (ranks[j - 1] if j else 0)]
    np.testing.assert_array_equal(sel, greedy)


@gpu
def test_rcss_stop_at_k_columns():
    """The experiments' treatment (Sec. 4.1): the subset stops growing at k columns; the stream
    goes on (p, sigma and the steps) against the basis of those k."""
    A = config1_matrix(5, m=3000, n=400, r=40, noise_var=1e-7)
    k = 10
    xi = 0.5 * k * float(np.median(np.einsum("ij,ij->j", A, A)))
    sel, o = check(A, k, xi, 7, np.float64, rel=1e-12, min_frac=1.0, limit=k)
    assert len(sel) == k and o.Q.shape[1] == k


@gpu
def test_rcss_huge_xi_selects_nothing():
    A = config1_matrix(9, m=500, n=120, r=10, noise_var=1e-2)
    xi = 1e12 * float(np.linalg.norm(A) ** 2)
    sel, sigma, nb, p, _ = run_gpu(A, 4, xi, 1, np.float64)
    assert len(sel) == 0 and nb == 0
    assert abs(sigma - p.sum()) <= 1e-12 * p.sum()


@gpu
def test_rcss_capacity_and_arguments():
    torch, rid = _lib()
    rng = np.random.default_rng(1)
    A = rng.standard_normal((64, 40))
    g = rid.ResidualCSS(64, 5, 1e-9, cap=8)          # every independent column is kept: 8 fit
    with pytest.raises(rid.RIDError) as e:
        g.ingest(A)
    assert e.value.code == rid.RID_EINVAL
    g.close()
    h = rid.ctypes.c_void_p()
    assert rid.rid_rcss_init(rid.ctypes.byref(h), 0, 5, 1.0, 0, rid.RID_F64, 8, 0, None) == rid.RID_EINVAL
    assert rid.rid_rcss_init(rid.ctypes.byref(h), 10, 5, 0.0, 0, rid.RID_F64, 8, 0, None) == rid.RID_EINVAL
    assert rid.rid_rcss_init(rid.ctypes.byref(h), 10, 5, 1.0, 0, rid.RID_F64, 5000, 0, None) == rid.RID_EINVAL
    assert rid.rid_rcss_init(rid.ctypes.byref(h), 10, 5, 1.0, 0, 7, 8, 0, None) == rid.RID_EINVAL
