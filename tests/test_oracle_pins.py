"""Pins for the CPU oracle: closed forms, brute force, invariants and published values.

Each test fixes a property that the paper or the mathematics determines
independently of the oracle's own code, chosen so that a plausible slip in the
oracle (a dropped 1/s scale, a transposed operand, a wrong sign, a wrong index
set) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import philox, offline
from oracle.gradient import grid_gradient_operator
from oracle.rid import (RIDConfig, OnlineRID, coeff_alg4, coeff_alg5, coeff_alg6,
                        coeff_alg7, css_update, na_hutchpp_sq_error, refill_scale,
                        sketched_ridge_scores, streaming_lambda)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32(*v[:4], v[4], v[5])
        assert [int(o) for o in out] == v[6:]


def test_rademacher_bit_layout_and_moments():
    seed = 12345
    blk = philox.rademacher_block(seed, [3, 7], 0, 512)
    k0, k1 = philox.seed_key(seed)
    # entry (row 7, coordinate 300): block 2, position 44 -> word 1, e = 12 (even, pair 6) -> bit 9;
    # coordinate 301 (e = 13, odd, pair 6) -> bit 25
    w = philox.philox4x32(2, 7, philox.TAG_RADEMACHER, 0, k0, k1)
    assert blk[1, 300] == (-1.0 if (int(w[1]) >> 9) & 1 else 1.0)
    assert blk[1, 301] == (-1.0 if (int(w[1]) >> 25) & 1 else 1.0)
    # every bit of the 128-bit block is used exactly once per 128 coordinates
    one = philox.rademacher_block(seed, [7], 256, 384)[0]
    bits = [(int(w[q]) >> b) & 1 for q in range(4) for b in range(32)]
    assert sorted((one < 0).astype(int).tolist()) == sorted(bits)
    big = philox.rademacher_block(seed, np.arange(64), 0, 4096)
    assert set(np.unique(big)) == {-1.0, 1.0}
    assert abs(big.mean()) < 4 / math.sqrt(big.size)
    # distinct rows are uncorrelated: E[w_r w_q] = delta_rq
    C = big @ big.T / big.shape[1]
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() < 5 / math.sqrt(big.shape[1])


def test_gaussian_moments():
    g = philox.gauss_block(7, np.arange(16), 0, 8192)
    x = g.ravel()
    n = x.size
    assert abs(x.mean()) < 4 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 0.1


def test_uniform53_exact_and_range():
    u = philox.uniform(99, np.arange(4), np.arange(1000)[:, None], 0)
    assert (u >= 0).all() and (u < 1).all()
    k0, k1 = philox.seed_key(99)
    w = philox.philox4x32(5, 3, philox.TAG_UNIFORM, 2, k0, k1)
    ref = ((int(w[0]) >> 5) * 2 ** 26 + (int(w[1]) >> 6)) / 2 ** 53
    assert float(philox.uniform(99, 2, 5, 3)) == ref


# ---------------------------------------------------------------- ridge leverage (Eqs. 16, 23)
def test_ridge_scores_orthogonal_closed_form():
    """For orthogonal columns with norms sigma_j, Eq. 16 gives sigma_j^2/(sigma_j^2 + lambda)."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 6)))
    sig = np.array([3.0, 2.0, 1.0, 0.5, 0.1, 0.01])
    A = Q * sig
    lam = 0.3
    ref = sig ** 2 / (sig ** 2 + lam)
    np.testing.assert_allclose(offline.ridge_leverage_scores(A, lam), ref, rtol=1e-12)
    # Eq. 23 with the identity as the (scaled) sketch reduces to Eq. 16
    np.testing.assert_allclose(sketched_ridge_scores(A @ A.T, lam, A), ref, rtol=1e-12)


def test_ridge_score_trace_identity_and_monotonicity():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((10, 7)) @ np.diag([5, 3, 2, 1, .5, .2, .1])
    lam = 0.4
    tau = offline.ridge_leverage_scores(A, lam)
    mu = np.linalg.eigvalsh(A @ A.T)
    assert abs(tau.sum() - np.sum(mu / (mu + lam))) < 1e-12
    b = rng.standard_normal(10)
    tau2 = offline.ridge_leverage_scores(np.column_stack([A, b]), lam)
    assert (tau2[:7] <= tau + 1e-15).all()      # Lemma 1 (monotonicity)


def test_streaming_lambda_identity_sketch_is_tail_over_k():
    """With the identity sketch, (||A||^2 - ||S_k||^2)/k equals ||A - A_k||_F^2/k (Eckart-Young)."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((15, 9))
    k = 4
    lam = streaming_lambda(A @ A.T, float(np.sum(A * A)), k)
    assert abs(lam - offline.tail_energy(A, k) / k) < 1e-12 * np.sum(A * A)


# ---------------------------------------------------------------- CPQR ID (Eqs. 5-11) and coefficient updates
def test_cpqr_id_is_least_squares_and_exact_for_rank_k():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 30))
    J, P = offline.cpqr_id(A, 5)
    np.testing.assert_allclose(P[:, J], np.eye(5), atol=1e-12)
    assert offline.id_error(A, J, P) < 1e-12 * np.linalg.norm(A)
    B = A + 1e-3 * rng.standard_normal(A.shape)
    J, P = offline.cpqr_id(B, 5)
    Pls = np.linalg.lstsq(B[:, J], B, rcond=None)[0]
    np.testing.assert_allclose(P, Pls, atol=1e-9)


def test_coefficient_updates_with_identity_sketch_equal_exact_least_squares():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 20))
    J = np.array([3, 9, 11, 17])
    Pls = np.linalg.lstsq(A[:, J], A, rcond=None)[0]
    G = A[:, J].T @ A[:, J]
    np.testing.assert_allclose(coeff_alg4(A[:, J], A), Pls, atol=1e-12)
    np.testing.assert_allclose(coeff_alg5(G, A[:, J], A), Pls, atol=1e-11)
    # Algorithm 6 with every row replaced is Algorithm 4; with none replaced it keeps P_prev
    Pprev = rng.standard_normal((4, 20))
    np.testing.assert_allclose(coeff_alg6(A[:, J], A, Pprev, np.zeros(4, bool)), Pls, atol=1e-12)
    np.testing.assert_array_equal(coeff_alg6(A[:, J], A, Pprev, np.ones(4, bool)), Pprev)
    # mixed case: kept rows are unchanged; the new rows satisfy the normal equations of the residual
    kept = np.array([True, False, True, False])
    P6 = coeff_alg6(A[:, J], A, Pprev, kept)
    np.testing.assert_array_equal(P6[kept], Pprev[kept])
    Anew = A[:, J[~kept]]
    np.testing.assert_allclose(Anew.T @ (A - A[:, J] @ P6), 0, atol=1e-10)
    # Algorithm 7: T = A_J^+ A_Jprev; same basis gives T = I
    np.testing.assert_allclose(coeff_alg7(A[:, J], A[:, J], Pprev), Pprev, atol=1e-12)
    # a permuted previous basis is mapped back by the permutation
    perm = np.array([2, 0, 3, 1])
    np.testing.assert_allclose(coeff_alg7(A[:, J], A[:, J[perm]], Pprev), np.eye(4)[:, perm] @ Pprev, atol=1e-12)


# ---------------------------------------------------------------- NA-Hutch++ (Eqs. 33-37)
def _hutch_fixture(seed=5, m=60, n=25, t=4, h=36):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 6)) @ rng.standard_normal((6, n)) + 0.1 * rng.standard_normal((m, n))
    J = np.array([1, 7, 12, n - 2])
    P = np.linalg.lstsq(A[:, J], A, rcond=None)[0] + 0.05 * rng.standard_normal((t, n))
    Om = rng.standard_normal((h, m))
    return A, J, P, Om


def test_hutchpp_sketch_form_equals_dense_form():
    """Eq. 37 (sketches only) equals Eqs. 34-35 applied to the explicit B = A (A_J P)^T."""
    A, J, P, Om = _hutch_fixture()
    AJ = A[:, J]
    G = AJ.T @ AJ
    split = ((0, 6), (6, 18), (18, 36))
    H = Om @ A
    fro2 = float(np.sum(A * A))
    e2 = na_hutchpp_sq_error(H, H[:, J], P, G, fro2, split)
    B = A @ (AJ @ P).T
    cross = offline.na_hutchpp_trace(B, Om[0:6], Om[6:18], Om[18:36])
    ref = fro2 - 2 * cross + np.trace(G @ P @ P.T)
    assert abs(e2 - ref) < 1e-10 * fro2
    # Eq. 36 itself: the expansion is an identity for the exact trace
    exact = np.linalg.norm(A - AJ @ P) ** 2
    assert abs(fro2 - 2 * np.trace(B) + np.trace(G @ P @ P.T) - exact) < 1e-10 * fro2


def test_hutchpp_reduces_to_hutchinson_without_control_variate():
    A, J, P, Om = _hutch_fixture()
    AJ = A[:, J]
    G = AJ.T @ AJ
    fro2 = float(np.sum(A * A))
    e2 = na_hutchpp_sq_error(Om @ A, (Om @ A)[:, J], P, G, fro2, ((0, 0), (0, 0), (0, 36)))
    B = A @ (AJ @ P).T
    ref = fro2 - 2 * offline.hutchinson_trace(B, Om) + np.trace(G @ P @ P.T)
    assert abs(e2 - ref) < 1e-10 * fro2


def test_hutchpp_exact_when_reconstruction_is_exact_and_rank_small():
    """A = A_J P of rank r <= c1 h: B is symmetric of rank r, B~ = B and the estimate is exact (0)."""
    rng = np.random.default_rng(6)
    m, n, r = 80, 30, 4
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    J = np.array([0, 5, 9, 14])
    P = np.linalg.lstsq(A[:, J], A, rcond=None)[0]
    G = A[:, J].T @ A[:, J]
    Om = rng.standard_normal((48, m))
    H = Om @ A
    e2 = na_hutchpp_sq_error(H, H[:, J], P, G, float(np.sum(A * A)), ((0, 8), (8, 24), (24, 48)))
    assert abs(e2) < 1e-9 * np.sum(A * A)


def test_hutchpp_unbiased_over_probe_draws():
    """E[e2] = ||A - A_J P||_F^2 for fixed (A, J, P) over independent probe rows."""
    A, J, P, _ = _hutch_fixture(seed=8, m=40, n=20, h=30)
    AJ = A[:, J]
    G = AJ.T @ AJ
    fro2 = float(np.sum(A * A))
    exact = np.linalg.norm(A - AJ @ P) ** 2
    split = ((0, 5), (5, 15), (15, 30))
    vals = []
    for seed in range(3000):
        Om = philox.rademacher_block(seed, np.arange(30), 0, A.shape[0])
        H = Om @ A
        vals.append(na_hutchpp_sq_error(H, H[:, J], P, G, fro2, split))
    vals = np.array(vals)
    se = vals.std() / math.sqrt(len(vals))
    assert abs(vals.mean() - exact) < 4 * se


# ---------------------------------------------------------------- column subset selection
def test_css_update_probabilities():
    """Drop with probability 1 - tau/tau_old; refill with probability tau^D * scale (clipped)."""
    cfg = RIDConfig(m=10, k=4, s=7, seed=0)
    scale = refill_scale(cfg)
    JC = np.array([10, 11, 12, 13])
    tau_old = np.array([0.5, 0.5, 0.5, 0.5])
    tau_C = np.array([0.5, 0.4, 0.25, 0.1])          # drop probabilities 0, .2, .5, .8
    JD = [20, 21, 22, 23]
    tau_D = np.array([0.3, 0.3, 0.3, 0.3]) / scale    # refill probability 0.3 per candidate
    drops = np.zeros(4)
    first = np.zeros(4)
    N = 4000
    for seed in range(N):
        cfg.seed = seed
        newJ, newtau = css_update(cfg, 0, JC, tau_old, tau_C, JD, tau_D)
        dropped = newJ != JC
        drops += dropped
        if newJ[3] == 20:
            first[3] += 1
        assert len(set(int(j) for j in newJ if j >= 0)) == int((newJ >= 0).sum())
        kept = ~dropped
        np.testing.assert_array_equal(newtau[kept], tau_C[kept])
    p = np.array([0.0, 0.2, 0.5, 0.8])
    assert drops[0] == 0
    se = np.sqrt(p * (1 - p) / N) + 1e-9
    assert (np.abs(drops / N - p) < 4 * se + 1e-12).all()
    # slot 3 is dropped w.p. 0.8 and then takes candidate 20 w.p. 0.3, unless slot 1 or 2
    # (dropped w.p. 0.2 and 0.5) took it first: candidates already in C are skipped
    q = 0.8 * 0.3 * (1 - 0.2 * 0.3) * (1 - 0.5 * 0.3)
    assert abs(first[3] / N - q) < 4 * math.sqrt(q * (1 - q) / N)


def test_css_update_proportional_refill():
    """R7p: a refilled slot takes buffered column r with probability tau^D_r / sum tau^D over the
    columns not already in C (here every refill probability is clipped to 1, the case in which
    R7 would always take the first column); the refill decision itself is R7's."""
    cfg = RIDConfig(m=10, k=4, s=7, seed=0, refill="proportional")
    scale = refill_scale(cfg)
    JC = np.array([10, -1, 12, 13])                  # slot 1 empty: always refilled
    tau_old = np.array([0.5, 1.0, 0.5, 0.5])
    tau_C = np.array([0.5, 1.0, 0.5, 0.5])           # no drops
    JD = [20, 21, 22, 23]
    w = np.array([1.0, 2.0, 3.0, 4.0])
    tau_D = w * (2.0 / scale)                        # p = min(2 w, 1) = 1 for every candidate
    N = 6000
    counts = np.zeros(4)
    for seed in range(N):
        cfg.seed = seed
        newJ, newtau = css_update(cfg, 0, JC, tau_old, tau_C, JD, tau_D)
        r = JD.index(int(newJ[1]))
        counts[r] += 1
        assert newtau[1] == tau_D[r]
        np.testing.assert_array_equal(newJ[[0, 2, 3]], JC[[0, 2, 3]])
    p = w / w.sum()
    chi2 = float((((counts - N * p) ** 2) / (N * p)).sum())
    assert chi2 < 16.3, (counts, chi2)               # chi-square, 3 degrees of freedom, p ~ 0.001
    # the first-success reading on the same draws always takes the first column
    cfg.refill = "first"
    for seed in range(50):
        cfg.seed = seed
        assert css_update(cfg, 0, JC, tau_old, tau_C, JD, tau_D)[0][1] == 20
    # a column already in C is never drawn again: two empty slots receive distinct columns
    cfg.refill = "proportional"
    JC2 = np.array([-1, -1, 12, 13])
    for seed in range(300):
        cfg.seed = seed
        newJ = css_update(cfg, 0, JC2, tau_old, tau_C, JD, tau_D)[0]
        assert newJ[0] != newJ[1] and newJ[0] in JD and newJ[1] in JD


def test_refill_scale_formula():
    cfg = RIDConfig(m=10, k=20, s=83, eps=0.5, delta=0.05)
    assert abs(refill_scale(cfg) - (20 * math.log(20) + 20 * math.log(20.0) / 0.5) / 20) < 1e-12


# ---------------------------------------------------------------- whole stream (Algorithm 3)
def test_stream_exact_rank_r_reconstruction():
    """Rank r < t data: Algorithms 4 and 7 reproduce A; the chosen error estimate is ~0 with c1 h >= r."""
    rng = np.random.default_rng(9)
    m, n, r, k = 400, 70, 5, 8
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    cfg = RIDConfig(m=m, k=k, s=4 * k + 3, h=60, seed=2)
    o = OnlineRID(cfg)
    o.ingest(A)
    J, P = o.finalize()
    act = o._last_active
    assert np.linalg.norm(A - A[:, J[act]] @ o._last_candidates[0]) < 1e-11 * np.linalg.norm(A)
    assert np.linalg.norm(A - A[:, J[act]] @ o._last_candidates[3]) < 1e-10 * np.linalg.norm(A)
    est, q = o.error_estimates()
    assert abs(est[0]) < 1e-9 * np.sum(A * A)
    assert offline.id_error(A, J, P) < 1e-6 * np.linalg.norm(A) or q in (5, 6)


def test_stream_large_sketch_approaches_unsketched_quantities():
    """s >> t: the scaled sketch Gram matches A A^T in trace and top-k energy, and Algorithm 5
    approaches exact least squares (both fail by a factor ~s if the 1/s scale of R1 is dropped)."""
    rng = np.random.default_rng(10)
    m, n, k = 300, 24, 6
    A = rng.standard_normal((m, 10)) @ np.diag(2.0 ** -np.arange(10)) @ rng.standard_normal((10, n))
    A += 0.01 * rng.standard_normal((m, n))
    s = 3000
    cfg = RIDConfig(m=m, k=k, s=s, h=0, seed=1)
    o = OnlineRID(cfg)
    o.ingest(A[:, :k * 3])
    A18 = A[:, :18]
    fro2 = float(np.sum(A18 ** 2))
    M = o.SSt / s
    assert abs(np.trace(M) - fro2) < 4 * math.sqrt(2.0 / s) * fro2
    mu = np.linalg.eigvalsh(M)[::-1]
    topk = fro2 - offline.tail_energy(A18, k)
    assert abs(mu[:k].sum() - topk) < 0.1 * topk
    rec = o.history[-1]
    assert abs(rec.lam - max((fro2 - mu[:k].sum()) / k, 1e-12 * fro2 / k)) < 1e-9 * fro2
    act = o._last_active
    J = o.JC[act]
    P5 = o._last_candidates[1]
    Pls = np.linalg.lstsq(A[:, J], A18, rcond=None)[0]
    assert np.linalg.norm(A[:, J] @ (P5 - Pls)) < 0.1 * np.linalg.norm(A18)


def test_stream_first_batch_fills_slots_in_order_when_probabilities_saturate():
    rng = np.random.default_rng(11)
    m, k = 200, 5
    A = rng.standard_normal((m, 5))
    cfg = RIDConfig(m=m, k=k, s=23, h=12, c_const=1e6, seed=4)
    o = OnlineRID(cfg)
    o.ingest(A)
    np.testing.assert_array_equal(o.JC, np.arange(5))


def test_stream_tail_batch_and_p_width():
    rng = np.random.default_rng(12)
    m, k, n = 150, 4, 23
    A = rng.standard_normal((m, n))
    cfg = RIDConfig(m=m, k=k, s=19, h=12, seed=3)
    o = OnlineRID(cfg)
    o.ingest(A)
    assert len(o.history) == n // k
    J, P = o.finalize()
    assert len(o.history) == n // k + 1
    assert P.shape == (k, n)
    assert ((J >= -1) & (J < n)).all()
    assert (P[J < 0] == 0).all()


# ---------------------------------------------------------------- simplex gradient (Eqs. 38-43)
def test_gradient_interior_is_central_difference_and_linear_exact():
    nx, ny = 7, 5
    G = grid_gradient_operator((nx, ny))
    x = np.arange(nx)[None, :].repeat(ny, 0).ravel()    # x fastest
    y = np.arange(ny)[:, None].repeat(nx, 1).ravel()
    f = np.sin(0.7 * x) + np.cos(0.3 * y) * x
    g = G @ f
    gx, gy = g[: nx * ny].reshape(ny, nx), g[nx * ny:].reshape(ny, nx)
    F = f.reshape(ny, nx)
    np.testing.assert_allclose(gx[:, 1:-1], (F[:, 2:] - F[:, :-2]) / 2, atol=1e-12)
    np.testing.assert_allclose(gy[1:-1, :], (F[2:, :] - F[:-2, :]) / 2, atol=1e-12)
    np.testing.assert_allclose(gx[:, 0], F[:, 1] - F[:, 0], atol=1e-12)       # one-sided at the boundary
    lin = 2.0 * x - 3.0 * y + 1.0
    gl = G @ lin
    np.testing.assert_allclose(gl[: nx * ny], 2.0, atol=1e-12)
    np.testing.assert_allclose(gl[nx * ny:], -3.0, atol=1e-12)
    G2 = grid_gradient_operator((nx, ny), nfields=2)
    assert G2.shape == (2 * 2 * nx * ny, 2 * nx * ny)
    np.testing.assert_allclose(G2 @ np.concatenate([f, lin]),
                               np.concatenate([gx.ravel(), lin * 0 + 2.0, gy.ravel(), lin * 0 - 3.0]), atol=1e-12)


# ---------------------------------------------------------------- optional right sketch
@pytest.mark.parametrize("kind", ["rademacher", "gaussian"])
def test_right_sketch_is_unbiased_for_the_column_gram(kind):
    """E[Y Y^T] = l A A^T for unit-variance i.i.d. omega_j (JL-type sketch): the mean over
    independent seeds lies within 5 standard errors entrywise; a dropped or doubled scale, or
    omega vectors shared between snapshots, break it."""
    from oracle.rid import right_sketch
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 5))
    l, nseed = 8, 1500
    acc = np.zeros((6, 6))
    acc2 = np.zeros((6, 6))
    for seed in range(nseed):
        Y = right_sketch(A, l, kind, 1000 + seed)
        g = Y @ Y.T / l
        acc += g
        acc2 += g * g
    mean = acc / nseed
    se = np.sqrt(np.maximum(acc2 / nseed - mean ** 2, 1e-30) / nseed)
    assert np.all(np.abs(mean - A @ A.T) <= 5 * se + 1e-12)


def test_right_sketch_captures_the_range_and_is_block_invariant():
    """With l >= rank(A) Gaussian omega_j, range(Y) = range(A) (A = Q Q^T A for the
    orthonormal basis Q of Y), and streaming the columns in any blocks gives the same Y as
    the whole matrix (omega_j is keyed by the global snapshot index j)."""
    from oracle.rid import right_sketch
    rng = np.random.default_rng(5)
    m, n, r = 40, 30, 4
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    Y = right_sketch(A, 7, "gaussian", 11)
    U, sv, _ = np.linalg.svd(Y, full_matrices=False)
    Q = U[:, sv > 1e-10 * sv[0]]
    assert np.linalg.norm(A - Q @ (Q.T @ A)) <= 1e-12 * np.linalg.norm(A)
    o = OnlineRID(RIDConfig(m=m, k=5, s=23, h=12, omega_kind="gaussian", seed=11, right_l=7))
    o.ingest(A[:, :3])
    o.ingest(A[:, 3:4])
    o.ingest(A[:, 4:])
    assert np.allclose(o.Y, Y, rtol=0, atol=1e-12 * np.abs(Y).max())
    L = philox.omega_block("gaussian", 11, np.arange(7), 0, n)           # the left-sketch stream
    R = philox.omega_block("gaussian", 11, np.arange(7), 0, n, right=True)
    assert not np.allclose(L, R)                                         # independent streams


# ---------------------------------------------------------------- gradient-augmented coefficients (Sec. 3.4)
def _grid_case(seed=0, nx=6, ny=5, n=12):
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    A = np.stack([(np.cos(2 * np.pi * (rng.integers(1, 3) * x + rng.integers(0, 2) * y) + rng.uniform(0, 6))
                   + 0.1 * rng.standard_normal((ny, nx))).reshape(-1) for _ in range(n)], axis=1)
    G = grid_gradient_operator((nx, ny))
    return A, G


def test_gradient_coefficients_with_identity_sketch_solve_the_augmented_problem():
    """With Omega = sqrt(s) I the sketched quantities are the exact ones: P(lam) is the least-
    squares solution of the stacked system [A_J; sqrt(lam) G^p A_J] X = [A; sqrt(lam) G^p A]
    (lstsq, another route), C(lam) A = A_J P(lam) (the identity the paper states for C), and at
    lam -> 0 C is the orthogonal projector onto range(A_J): tr(I - C) = m - |J|."""
    from oracle import gcv
    A, Gop = _grid_case()
    m = A.shape[0]
    Gs = gcv.split_gradient(Gop, m)
    J = [0, 3, 7, 9]
    SJ, GJ, G = A[:, J], [Gp @ A[:, J] for Gp in Gs], [Gp @ A for Gp in Gs]
    K = [Gp.toarray() for Gp in Gs]
    for lam in (1e-3, 0.3, 7.0):
        P = gcv.p_of_lambda(SJ, A, GJ, G, lam)
        stack_l = np.vstack([SJ] + [math.sqrt(lam) * g for g in GJ])
        stack_r = np.vstack([A] + [math.sqrt(lam) * g for g in G])
        P_ls = np.linalg.lstsq(stack_l, stack_r, rcond=None)[0]
        assert np.allclose(P, P_ls, rtol=1e-9, atol=1e-11)
        C = gcv.c_matrix(SJ, GJ, K, lam)
        assert np.allclose(C @ A, SJ @ P, rtol=1e-9, atol=1e-11)
    C0 = gcv.c_matrix(SJ, GJ, K, 1e-14)
    assert abs(np.trace(C0) - len(J)) < 1e-8
    Q, _ = np.linalg.qr(SJ)
    proj_res = np.sum((A - Q @ (Q.T @ A)) ** 2)
    assert abs(gcv.gcv(SJ, A, GJ, K, 1e-14) - proj_res / (m - len(J)) ** 2) < 1e-8 * proj_res


def test_golden_section_finds_known_minima():
    from oracle import gcv
    assert abs(gcv.golden_section(lambda t: (t - 0.7) ** 2 + 1.0) - 0.7) < 1e-3
    assert abs(gcv.golden_section(lambda t: math.exp(t) - 2.0 * t) - math.log(2.0)) < 1e-3
    assert abs(gcv.golden_section(lambda t: abs(t + 2.5)) + 2.5) < 1e-3


def test_stream_keeps_gradient_sketches_and_small_lambda_gives_algorithm_4():
    """The streamed Omega G^p a_j equal Omega G^p A column by column, and with lam -> 0 the
    augmented solution is the plain sketched least squares of Algorithm 4 (Eq. 24)."""
    from oracle import gcv
    A, Gop = _grid_case(1, n=20)
    m = A.shape[0]
    o = OnlineRID(RIDConfig(m=m, k=4, s=19, h=12, seed=2, grad_op=Gop, grad_coeff=True))
    o.ingest(A[:, :7])
    o.ingest(A[:, 7:])
    Om = o.omega()[:19]
    for p, Gp in enumerate(gcv.split_gradient(Gop, m)):
        assert np.allclose(o.SG[p], Om @ (Gp @ A), rtol=1e-12, atol=1e-12)
    J, P = o.finalize()
    act = J >= 0
    S = o.S[:19] / math.sqrt(19)
    G = [o.SG[p] / math.sqrt(19) for p in range(2)]
    Pz = gcv.p_of_lambda(S[:, J[act]], S, [g[:, J[act]] for g in G], G, 1e-13)
    assert np.allclose(Pz, coeff_alg4(S[:, J[act]], S), rtol=1e-7, atol=1e-9)
    lam, Pg, g = o.gradient_coefficients()
    assert 1e-3 <= lam <= 1e3 and np.isfinite(g) and Pg.shape == (4, 20)


def test_truncated_svd_error_closed_form():
    """Eckart-Young: with A = U diag(sigma) V^T (orthonormal U, V) the best rank-k error is the
    norm of the trailing singular values."""
    from oracle.offline import truncated_svd_error
    rng = np.random.default_rng(21)
    U, _ = np.linalg.qr(rng.standard_normal((40, 9)))
    V, _ = np.linalg.qr(rng.standard_normal((15, 9)))
    sig = np.array([9.0, 5.0, 4.0, 2.0, 1.0, 0.5, 0.25, 0.125, 0.0625])
    A = U @ np.diag(sig) @ V.T
    for k in (0, 1, 4, 9):
        want = math.sqrt(np.sum(sig[k:] ** 2) / np.sum(sig ** 2))
        assert abs(truncated_svd_error(A, k) - want) <= 1e-13


def test_stream_exact_rank_r_with_shared_probe_rows():
    """The paper-literal probe mode (h = 0: NA-Hutch++ draws its rows from the left sketch itself,
    split c1 s / c2 s / rest): with rank r < t data Algorithm 4 reproduces A and the chosen
    estimate is ~0, as with independent probe rows."""
    rng = np.random.default_rng(19)
    m, n, r, k = 400, 70, 5, 8
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    o = OnlineRID(RIDConfig(m=m, k=k, s=4 * k + 3, h=0, seed=6))
    assert o.cfg.probe_split() == ((0, 5), (5, 16), (16, 35))
    o.ingest(A)
    J, P = o.finalize()
    act = o._last_active
    assert np.linalg.norm(A - A[:, J[act]] @ o._last_candidates[0]) < 1e-11 * np.linalg.norm(A)
    est, q = o.error_estimates()
    assert abs(est.min()) < 1e-9 * np.sum(A * A)


# ---------------------------------------------------------------- FP8 (E4M3) block-scaled operands
def test_e4m3_grid_from_the_bit_definition():
    from oracle import fp8
    g = fp8.e4m3_grid()
    pos = g[g > 0]
    assert len(pos) == 126                              # 7 subnormals, 14 x 8 normals, 7 in the top binade
    assert pos.min() == 2.0 ** -9 and pos.max() == 448.0
    assert 2.0 ** -6 in pos and (1 + 7 / 8) * 2.0 ** 7 in pos and 480.0 not in pos
    assert np.all(np.diff(g) > 0)


def test_e4m3_rounding_is_nearest_with_ties_to_even_and_saturates():
    from oracle import fp8
    g = fp8.e4m3_grid()
    assert np.array_equal(fp8.e4m3_round(g), g) and np.array_equal(fp8.e4m3_round(-g), -g)
    # brute force: the nearest grid value; at a midpoint, the one whose mantissa (index) is even
    rng = np.random.default_rng(8)
    mids = (g[1:] + g[:-1]) / 2
    x = np.concatenate([rng.uniform(0, 448, 4000), 2.0 ** rng.uniform(-12, 8.8, 4000), mids])
    got = fp8.e4m3_round(x)
    for xi, gi in zip(x, got):
        d = np.abs(g - min(xi, 448.0))
        cand = np.nonzero(d == d.min())[0]
        want = g[cand[0]] if len(cand) == 1 else g[[c for c in cand if c % 2 == 0][0]]
        assert gi == want, (xi, gi, want)
    assert fp8.e4m3_round(0.1) == 0.1015625                   # 1.625 x 2^-4
    assert fp8.e4m3_round(1.0625) == 1.0 and fp8.e4m3_round(1.1875) == 1.25   # ties to even
    assert fp8.e4m3_round(2.0 ** -10) == 0.0 and fp8.e4m3_round(3 * 2.0 ** -11) == 2.0 ** -9
    assert fp8.e4m3_round(500.0) == 448.0 and fp8.e4m3_round(-1e6) == -448.0


def test_block_scales_are_the_smallest_powers_of_two_that_avoid_saturation():
    from oracle import fp8
    rng = np.random.default_rng(9)
    a = rng.standard_normal((100, 5)) * 10.0 ** rng.uniform(-6, 6, 5)
    a[32:64, 2] = 0.0                                   # an all-zero block
    a[5, 4] = 448.0 * 2.0 ** -20                        # a block maximum exactly on the bound
    s = fp8.block_scales(a, 32)
    for b0 in range(0, 100, 32):
        blk, sb = a[b0:b0 + 32], s[b0:b0 + 32]
        assert np.all(sb == sb[0])                      # one scale per block and column
        amax = np.abs(blk).max(axis=0)
        x = np.log2(sb[0])
        assert np.all(x == np.round(x))                 # powers of two
        nz = amax > 0
        assert np.all(amax[nz] / sb[0][nz] <= 448.0) and np.all(amax[nz] / (sb[0][nz] / 2) > 448.0)
        assert np.all(sb[0][~nz] == 1.0)


def test_fp8x2_split_error_bound_and_sketch():
    """Each stage rounds to 3 fraction bits (relative error <= 2^-4 for normal values), so
    |a - hi - lo| <= 2^-8 |a| plus the subnormal spacing of the second stage; the split's
    sketch is the sketch of hi + lo, and its error is the sketch of that residual."""
    from oracle import fp8
    rng = np.random.default_rng(10)
    m, n, block = 1000, 6, 32
    a = rng.standard_normal((m, n)) * np.exp(rng.standard_normal((m, n)))
    hi, lo = fp8.split_x2(a, block)
    s1, s2 = fp8.block_scales(a, block), fp8.block_scales(a - hi, block)
    g = fp8.e4m3_grid()
    assert np.isin(np.abs(hi / s1), g).all() and np.isin(np.abs(lo / s2), g).all()   # block-scaled E4M3 terms
    err = np.abs(a - hi - lo)
    assert np.all(err <= 2.0 ** -8 * np.abs(a) + 2.0 ** -10 * s2 + 1e-300)
    r = a - hi                                          # each stage: 3 fraction bits at its own scale
    assert np.all(np.abs(r - lo) <= 2.0 ** -4 * np.abs(r) + 2.0 ** -10 * s2)
    assert np.all(np.abs(a - hi) <= 2.0 ** -4 * np.abs(a) + 2.0 ** -10 * fp8.block_scales(a, block))
    om = philox.rademacher_block(3, np.arange(20), 0, m)
    S = fp8.sketch_fp8x2(om, a, block)
    assert np.allclose(S, om @ (hi + lo), rtol=0, atol=1e-12 * np.abs(om @ a).max())
    assert np.abs(S - om @ a).max() <= 2.0 ** -8 * np.abs(om).max() * np.abs(a).sum(axis=0).max() * 1.01


def _stream_with_history(seed, refill="first"):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((300, 8)) @ rng.standard_normal((8, 60)) + 0.05 * rng.standard_normal((300, 60))
    cfg = RIDConfig(m=300, k=10, s=23, h=9, seed=seed, refill=refill)
    o = OnlineRID(cfg)
    o.ingest(A)
    J, P = o.finalize()
    return A, cfg, o, J, P


@pytest.mark.parametrize("refill", ["first", "proportional"])
def test_resync_to_own_decisions_changes_nothing(refill):
    """Re-synchronising the selection to the oracle's own per-step slot contents records no
    differing decision and reproduces J, P and the estimates exactly."""
    A, cfg, o, J, P = _stream_with_history(3, refill)
    o2 = OnlineRID(cfg)
    o2.resync = {r.batch: r.JC for r in o.history}
    o2.ingest(A)
    J2, P2 = o2.finalize()
    assert o2.flips == []
    assert np.array_equal(J, J2) and np.array_equal(P, P2)
    assert np.array_equal(o.error_estimates()[0], o2.error_estimates()[0])


def test_resync_reports_the_planted_prune_and_refill_differences():
    """A planted difference in the target (a kept slot pruned; a refill with another buffered
    column) is reported as the decision that differs, with that decision's own margin, the step
    takes the target's slot contents, and the later steps run on them."""
    A, cfg, o, J, P = _stream_with_history(5)
    hist = {r.batch: r.JC.copy() for r in o.history}
    b = 2                                            # a step with earlier basis elements
    prev = hist[b - 1]
    kept_slots = [i for i in range(cfg.t) if prev[i] >= 0 and hist[b][i] == prev[i]]
    assert kept_slots
    i = kept_slots[0]
    target = hist[b].copy()
    target[i] = -1                                   # plant: slot i pruned instead of kept
    o3 = OnlineRID(cfg)
    o3.resync = {k: v for k, v in hist.items() if k < b}
    o3.resync[b] = target                            # the later steps decide on the synced state
    o3.ingest(A)
    o3.finalize()
    # the keep-or-prune draw of slot i differs; the slot's refill scan, which then runs on the
    # pruned slot, may differ from the planted empty slot too -- nothing else does
    assert (o3.flips[0][0], o3.flips[0][1], o3.flips[0][2]) == (b, i, "prune")
    assert all(f[0] == b and f[1] == i for f in o3.flips) and len(o3.flips) <= 2
    assert o3.history[b].JC[i] == -1
    assert o3.flips[0][3] > 0.0
    # a different refill: slot j refilled with another of the step's buffered columns
    refilled = [j for j in range(cfg.t) if hist[b][j] >= 0 and hist[b][j] != prev[j]]
    if refilled:
        j = refilled[0]
        batch_cols = set(range(b * cfg.t, (b + 1) * cfg.t))
        others = sorted(batch_cols - set(int(x) for x in hist[b]))
        target2 = hist[b].copy()
        target2[j] = others[0]
        o4 = OnlineRID(cfg)
        o4.resync = {k: v for k, v in hist.items() if k < b}
        o4.resync[b] = target2
        o4.ingest(A)
        o4.finalize()
        assert (b, j, "refill") in [(f[0], f[1], f[2]) for f in o4.flips]
        assert o4.history[b].JC[j] == others[0]


# ---------------------------------------------------------------- Algorithm 1 (residual CSS)
from oracle.residual_css import ResidualCSS


def _rank_stream(m, n, r, seed, dependent_every=3):
    """Columns that are either a new random direction or a combination of earlier columns."""
    rng = np.random.default_rng(seed)
    cols, independent = [], []
    for j in range(n):
        if j % dependent_every == dependent_every - 1 and cols:
            c = np.stack(cols, axis=1) @ rng.standard_normal(len(cols))
        elif len(independent) < r:
            c = rng.standard_normal(m)
            independent.append(j)
        else:
            c = np.stack(cols, axis=1) @ rng.standard_normal(len(cols))
        cols.append(c)
    return np.stack(cols, axis=1), independent


def test_residual_css_tiny_xi_selects_the_greedy_independent_columns():
    """With xi far below every nonzero residual, p >= 1 for each column outside the span (selected
    and added at once) and p ~ 0 for the columns inside it: the selection is the first maximal
    independent set in arrival order, checked by brute-force rank counts."""
    A, _ = _rank_stream(60, 40, 9, 3)
    o = ResidualCSS(60, k=5, xi=1e-20 * np.linalg.norm(A) ** 2, seed=1)
    o.ingest(A)
    brute = []
    for j in range(A.shape[1]):
        if np.linalg.matrix_rank(A[:, brute + [j]], tol=1e-8 * np.linalg.norm(A)) > len(brute):
            brute.append(j)
    assert list(o.selection()) == brute
    assert len(brute) == 9


def test_residual_css_huge_xi_selects_nothing_and_never_updates():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((50, 30))
    o = ResidualCSS(50, k=4, xi=1e9 * 4 * np.linalg.norm(A) ** 2, seed=3)
    o.ingest(A)
    assert len(o.selection()) == 0 and o.steps == []
    assert abs(o.sigma - sum(o.p)) <= 1e-15 * max(sum(o.p), 1e-300)


def test_residual_css_first_column_kept_with_probability_p():
    """The first column meets an empty C_pre: p = k ||a||^2 / xi, set to 0.3; over 4000 seeds it is
    kept with frequency 0.3 (4 sigma of the binomial)."""
    a = np.random.default_rng(5).standard_normal((20, 1))
    k = 3
    xi = k * float(a[:, 0] @ a[:, 0]) / 0.3
    hits = 0
    for seed in range(4000):
        o = ResidualCSS(20, k=k, xi=xi, seed=seed)
        o.ingest(a)
        assert abs(o.p[0] - 0.3) <= 1e-12
        hits += len(o.selection())
    assert abs(hits / 4000 - 0.3) <= 4 * np.sqrt(0.3 * 0.7 / 4000)


def test_residual_css_residual_mass_and_forced_updates():
    """Orthonormal columns with p = 0.4 each: sigma reaches 1.2 at the third, which ends the step;
    a column with p >= 1 ends a step at once and is always kept."""
    m = 8
    E = np.eye(m)
    k = 2
    xi = k / 0.4                                   # p = k ||e||^2 / xi = 0.4 outside span(C_pre)
    o = ResidualCSS(m, k=k, xi=xi, seed=7)
    o.ingest(E[:, :3])
    assert o.steps == [2] and o.sigma == 0.0
    o.ingest(E[:, 3:4])
    assert abs(o.sigma - 0.4) <= 1e-15
    o.ingest(3.0 * E[:, 4:5])                      # p = 2 * 9 / 5 = 3.6 >= 1
    assert o.steps == [2, 4] and 4 in o.selection() and o.sigma == 0.0


def test_residual_css_recovers_a_rank_r_stream():
    """A rank-5 stream with xi far below its energy: every column outside the span ends a step,
    so span(C) is the stream's range: ||A - Q Q^T A|| at rounding level."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((200, 5)) @ rng.standard_normal((5, 300))
    o = ResidualCSS(200, k=5, xi=1e-8 * np.linalg.norm(A) ** 2, seed=2)
    o.ingest(A)
    Q = o.Q
    assert Q.shape[1] == 5
    assert np.linalg.norm(A - Q @ (Q.T @ A)) <= 1e-10 * np.linalg.norm(A)
    assert np.abs(Q.T @ Q - np.eye(5)).max() <= 1e-12


def test_residual_css_limit_stops_the_selection_only():
    """With a limit of k columns (the experiments' treatment), the selection is the unlimited run's
    first k columns as long as the two runs agree -- they do up to the step that holds the k-th
    selection, and p is identical up to and including it -- and never more than k."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((80, 25)) @ rng.standard_normal((25, 120))
    xi = 0.2 * 6 * float(np.median(np.einsum("ij,ij->j", A, A)))
    free = ResidualCSS(80, k=6, xi=xi, seed=4)
    free.ingest(A)
    capped = ResidualCSS(80, k=6, xi=xi, seed=4, limit=6)
    capped.ingest(A)
    sel = free.selection()
    assert len(sel) > 6
    np.testing.assert_array_equal(capped.selection(), sel[:6])
    # the k-th selection's step: both runs took the same decisions through its end
    end = min(j for j in free.steps if j >= sel[5])
    np.testing.assert_array_equal(capped.p[:end + 1], free.p[:end + 1])
    assert len(capped.selection()) == 6 and len(capped.p) == 120


def test_residual_selector_feeds_algorithm1_subset_to_the_coefficient_updates():
    """The online rows with Algorithm 1 as the selector: the final basis is Algorithm 1's subset
    (capped at t columns) in slot order, and on an exact rank-6 stream whose subset spans the range
    the chosen coefficients reconstruct it to rounding."""
    from oracle.rid import OnlineRID, RIDConfig
    rng = np.random.default_rng(3)
    m, n, r, k = 300, 60, 6, 8
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    xi = 1e-4 * k * float(np.min(np.einsum("ij,ij->j", A, A)))
    cfg = RIDConfig(m=m, k=k, s=4 * k + 3, h=12, lambda_mode="fixed", lambda_fixed=1e-6, seed=1,
                    selector="residual", rcss_xi=xi, rcss_seed=5)
    o = OnlineRID(cfg)
    o.ingest(A)
    J, P = o.finalize()
    ref = ResidualCSS(m, k, xi, 5, limit=k)
    ref.ingest(A)
    act = J >= 0
    np.testing.assert_array_equal(J[act], ref.selection())
    assert np.all(J[~act] == -1) and act.sum() == 6
    assert np.linalg.norm(A - A[:, J[act]] @ P[act]) <= 1e-12 * np.linalg.norm(A)


def test_residual_css_replay_reproduces_the_run():
    """The decision steps replayed on a run's own p give back its selection, sigma and steps (the
    full-size GPU check relies on this)."""
    from oracle.residual_css import replay
    rng = np.random.default_rng(9)
    A = rng.standard_normal((60, 30)) @ rng.standard_normal((30, 150))
    xi = 0.3 * 5 * float(np.median(np.einsum("ij,ij->j", A, A)))
    for limit in (None, 7):
        o = ResidualCSS(60, 5, xi, 2, limit=limit)
        o.ingest(A)
        sel, sigma, steps = replay(o.p, 2, limit=limit)
        np.testing.assert_array_equal(sel, o.selection())
        assert sigma == o.sigma and steps == o.steps
