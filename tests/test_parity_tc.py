"""Tensor-core ingest (FP32 data, BF16 / BF16x2 sketches) against the FP64 oracle.

Bars, from the arithmetic: BF16x2 splits each FP32 value a = hi + lo with
|a - hi - lo| <= 2^-16 |a|, so a sketch entry sum_i (+-a_i) carries an error of
at most 2^-16 ||a||_1 and, with independent signs, about 2^-16 ||a||_2 / sqrt(3);
FP32 accumulation adds ~1e-6 ||a||_2.  The bar is 2e-5 ||a||_2 per entry.  BF16
rounds each value to 8 significant bits (|error| <= 2^-9 |a|, RMS 2^-9/sqrt(3) |a|), so
an entry's error has standard deviation ~1.1e-3 ||a||_2; over thousands of entries the
maximum reaches 4-6 sigma: bar 1e-2 ||a||_2 (about 9 sigma).
The copy into the buffer slot must be bit-exact; squared norms within 1e-6.
"""
import numpy as np
import pytest

from oracle.rid import OnlineRID as Oracle, RIDConfig

pytestmark = pytest.mark.gpu


def _mats(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 10)) @ np.diag(0.8 ** np.arange(10)) @ rng.standard_normal((10, n))
    A += 0.05 * rng.standard_normal((m, n))
    return A.astype(np.float32)


def _run_gpu(A32, k, s, h, sketch, block=8, defer=False, group_max=0, offset=0, seed=3):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A32.shape
    g = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype="f32", sketch=sketch, seed=seed, defer=defer,
                      group_max=group_max)
    flat = torch.zeros(n * m + offset + 64, dtype=torch.float32, device="cuda")
    X = flat[offset:offset + n * m].view(n, m)
    X.copy_(torch.from_numpy(np.ascontiguousarray(A32.T)))
    for j0 in range(0, n, block):
        g.ingest(X[j0:j0 + block])
    J, P = g.finalize()
    return g, J, P, X


def _oracle(A32, k, s, h, seed=3):
    o = Oracle(RIDConfig(m=A32.shape[0], k=k, s=s, h=h, seed=seed))
    o.ingest(A32.astype(np.float64))
    return o


@pytest.mark.parametrize("sketch,bar", [("bf16x2", 2e-5), ("bf16", 1e-2)])
@pytest.mark.parametrize("m,n,k,s,h", [
    (100003, 45, 12, 51, 30),     # one N tile (81 rows -> 96), ragged m, tail batch
    (50000, 130, 100, 403, 50),   # two N tiles (453 rows -> 256 + 208)
])
def test_tc_sketch_against_oracle(sketch, bar, m, n, k, s, h):
    A = _mats(m, n, m + n)
    o = _oracle(A, k, s, h)
    g, J, P, X = _run_gpu(A, k, s, h, sketch, defer=True)
    S_g = g.state(0)
    norms = np.linalg.norm(A.astype(np.float64), axis=0)
    err = np.abs(S_g - o.S) / norms[None, :]
    assert err.max() <= bar, err.max()
    fro = g.state(3)
    assert abs(fro[0] - o.fro2) <= 1e-6 * o.fro2
    # the buffered/basis columns are exact copies of the input
    B = g.basis()
    for i, j in enumerate(J):
        if j >= 0:
            assert np.array_equal(B[:, i], A[:, j])
    assert P.shape == (k, n) and np.isfinite(P).all()


def test_tc_group_size_and_alignment_invariance():
    """The sketch of a column does not depend on which group it was read with, nor on the
    alignment of its pointer (vector or scalar loads)."""
    A = _mats(70001, 40, 7)
    k, s, h = 10, 43, 30
    g1, J1, P1, _ = _run_gpu(A, k, s, h, "bf16x2", block=8, defer=False)
    g2, J2, P2, _ = _run_gpu(A, k, s, h, "bf16x2", block=8, defer=True, group_max=64)
    g3, J3, P3, _ = _run_gpu(A, k, s, h, "bf16x2", block=3, defer=False, offset=1)
    S1, S2, S3 = g1.state(0), g2.state(0), g3.state(0)
    assert np.array_equal(S1, S2)
    assert np.array_equal(S1, S3)
    assert np.array_equal(J1, J2) and np.array_equal(P1, P2)


def test_tc_host_input_matches_device_input():
    import torch
    from paper_2405_16076_gb300 import rid
    A = _mats(30000, 25, 9)
    k, s, h = 8, 35, 12
    g1, J1, P1, _ = _run_gpu(A, k, s, h, "bf16x2", defer=True)
    g = rid.OnlineRID(m=A.shape[0], k=k, s=s, h=h, dtype="f32", sketch="bf16x2", seed=3)
    rows = np.ascontiguousarray(A.T)
    for j0 in range(0, A.shape[1], 5):
        g.ingest(rows[j0:j0 + 5])
    J2, P2 = g.finalize()
    assert np.array_equal(g1.state(0), g.state(0))
    assert np.array_equal(J1, J2) and np.array_equal(P1, P2)


def test_tc_small_m_single_column_groups():
    A = _mats(200, 30, 5)          # fewer coordinates than one chunk pair per SM
    k, s, h = 5, 23, 12
    o = _oracle(A, k, s, h)
    g, J, P, _ = _run_gpu(A, k, s, h, "bf16x2", block=1)
    err = np.abs(g.state(0) - o.S) / np.linalg.norm(A.astype(np.float64), axis=0)[None, :]
    assert err.max() <= 2e-5


def test_tc_batch_step_candidates_on_gpu_sketch():
    """Batch-step parity on identical inputs: the oracle's Algorithms 4 and 5 evaluated on the
    GPU's own sketch and basis.  Algorithm 4 uses only the FP64 sketch (bar 1e-10 x kappa);
    Algorithm 5 also uses the basis Gram, computed on tensor cores from the BF16x2 split
    (per-term error <= ~2^-16 |a_i b_i|, FP32 accumulation): bar 1e-5 x kappa(G)."""
    import math
    from oracle.rid import coeff_alg4, coeff_alg5
    A = _mats(50000, 64, 21)
    k, s, h = 16, 67, 30
    g, J, P, _ = _run_gpu(A, k, s, h, "bf16x2", defer=True)
    n = A.shape[1]
    cand = g.candidates(n)
    S = g.state(0)
    act = J >= 0
    Ja = J[act]
    SA = S[:s] / math.sqrt(s)
    SJ = SA[:, Ja]
    A64 = A.astype(np.float64)
    G = A64[:, Ja].T @ A64[:, Ja]
    na = int(act.sum())
    P4 = coeff_alg4(SJ, SA)
    P5 = coeff_alg5(G, SJ, SA)
    kap = np.linalg.cond(SJ)
    assert np.linalg.norm(cand[0][:na] - P4) <= 1e-10 * max(1.0, kap) * np.linalg.norm(P4)
    kapG = np.linalg.cond(G)
    assert np.linalg.norm(cand[1][:na] - P5) <= 1e-5 * max(1.0, kapG) * np.linalg.norm(P5)


def test_tc_batch_step_alg6_alg7_hutch_on_gpu_state():
    """Batch-step parity of the rest of the step on identical inputs: the oracle's Algorithms 6 and
    7 and Algorithm 8's four estimates, evaluated on the GPU's own sketch, basis, previous basis and
    previous coefficients (read from a second handle stopped after the previous batch step: both
    run the same deterministic stream).  Algorithm 6 uses only the FP64 sketch (bar 1e-10 x
    kappa(Omega A_J)); Algorithm 7 goes through the tensor-core basis Gram (bar 1e-5 x kappa(G),
    as Algorithm 5).  The estimates: the oracle's Eqs. 36-37 on the GPU's candidates, the GPU's
    ||A_obs||^2 and the pseudo-inverse cutoff of the reduced-precision sketch (sk_rel = 2e-5); the
    GPU's Gram enters tr(G P P^T), so the bar is 1e-9 ||A_obs||^2 plus 5e-5 x the candidate's energy
    sum_j sum_a G_aa P_aj^2 (ten times the Gram's relative accuracy)."""
    import math
    from oracle.rid import coeff_alg4, coeff_alg6, coeff_alg7, na_hutchpp_sq_error
    A = _mats(50000, 64, 21)
    k, s, h = 16, 67, 30
    n = A.shape[1]
    gp, Jp, Pp, _ = _run_gpu(A[:, :n - k], k, s, h, "bf16x2", defer=True)   # stops after batch 2
    g, J, P, _ = _run_gpu(A, k, s, h, "bf16x2", defer=True)
    n_prev = n - k
    cand = g.candidates(n)
    S = g.state(0)
    fro = g.state(3)[0]
    est_g = g.error_estimate()[0][1:5]
    A64 = A.astype(np.float64)
    act = np.nonzero(J >= 0)[0]
    Ja = J[act]
    na = len(act)
    SA = S[:s] / math.sqrt(s)
    SJ = SA[:, Ja]
    AJ = A64[:, Ja]
    G = AJ.T @ AJ
    P4a = coeff_alg4(SJ, SA)
    kept = J[act] == Jp[act]
    P_prev_ext = np.zeros((na, n))
    P_prev_ext[:, :n_prev] = Pp[act, :]
    P_prev_ext[:, n_prev:] = P4a[:, n_prev:]
    P6 = coeff_alg6(SJ, SA, P_prev_ext, kept)
    kap = np.linalg.cond(SJ)
    assert np.linalg.norm(cand[2][:na] - P6) <= 1e-10 * max(1.0, kap) * max(np.linalg.norm(P6), 1e-300)
    pact = np.nonzero(Jp >= 0)[0]
    P7 = np.zeros((na, n))
    P7[:, :n_prev] = coeff_alg7(AJ, A64[:, Jp[pact]], Pp[pact, :])
    P7[:, n_prev:] = P4a[:, n_prev:]
    kapG = np.linalg.cond(G)
    assert np.linalg.norm(cand[3][:na] - P7) <= 1e-5 * max(1.0, kapG) * np.linalg.norm(P7)
    cfg = RIDConfig(m=A.shape[0], k=k, s=s, h=h, seed=3)
    split = cfg.probe_split()
    base = split[0][0]
    H = S[base: split[2][1]]
    rel = tuple((a - base, b - base) for a, b in split)
    n1, n2 = rel[0][1] - rel[0][0], rel[1][1] - rel[1][0]
    rcond = max(max(n1, n2) * np.finfo(np.float64).eps, 2e-5)
    for q in range(4):
        Pq = cand[q][:na]
        est_o = na_hutchpp_sq_error(H, H[:, Ja], Pq, G, fro, rel, rcond=rcond)
        ener = float(np.einsum("a,aj->", np.diag(G), Pq * Pq))
        assert abs(est_g[q] - est_o) <= 1e-9 * fro + 5e-5 * ener, (q, est_g[q], est_o, ener)
