"""GPU <-> oracle parity on the small configuration and its edge cases.

The CUDA path (through the C ABI) and the FP64 oracle run the same seeded
stream with the same counter-based random numbers.  FP64 mode bar: indices
bit-exact unless a sampling decision of the oracle lies within 1e-10 (relative
to the score) of its threshold; coefficients within 1e-10 relative Frobenius
error; error estimates within 1e-9 of ||A||_F^2.
"""
import numpy as np
import pytest

from oracle import offline
from oracle.rid import OnlineRID as Oracle, RIDConfig
from workloads import config1_matrix

pytestmark = pytest.mark.gpu

P_TOL = 1e-10
MARGIN = 1e-10


def _gpu():
    import torch
    from paper_2405_16076_gb300 import rid
    return torch, rid


def run_oracle(A, **kw):
    o = Oracle(RIDConfig(m=A.shape[0], **kw))
    o.ingest(A)
    J, P = o.finalize()
    return o, J, P


def run_gpu(A, block=1, host=False, dtype="f64", n_max=1024, **kw):
    """The CUDA path over A's columns in ingest calls of `block` columns.  g.jcs: the basis slot
    contents after each batch step (read through the C ABI as each step completes; the last is
    the final J), for re-synchronising the oracle when a near-tie decision went the other way."""
    torch, rid = _gpu()
    m, n = A.shape
    t = kw["k"]
    g = rid.OnlineRID(m=m, k=t, s=kw["s"], h=kw.get("h", 0), dtype=dtype,
                      omega=kw.get("omega_kind", "rademacher"), lambda_mode=kw.get("lambda_mode", "streaming"),
                      lambda_fixed=kw.get("lambda_fixed", 0.0), seed=kw.get("seed", 0), n_max=n_max,
                      c1=kw.get("c1", 1 / 6), c2=kw.get("c2", 1 / 3), refill=kw.get("refill", "first"),
                      lookahead=kw.get("lookahead", 0))
    npd = np.float64 if dtype == "f64" else np.float32
    rows = np.ascontiguousarray(A.T.astype(npd))          # row q = column q
    if host:
        src = rows
    else:
        src = torch.from_numpy(rows).cuda()
    jcs = []
    for j0 in range(0, n, block):
        g.ingest(src[j0:j0 + block])
        while len(jcs) < min(j0 + block, n) // t:        # a batch step ran inside this call
            jcs.append(g.state(rid.RID_STATE_JC).astype(np.int64).copy())
    J, P = g.finalize()
    if n % t:
        jcs.append(J.copy())
    g.jcs = jcs
    g.okw = {key: kw[key] for key in kw if key in RIDConfig.__dataclass_fields__}
    return g, J, P


def resynced_oracle(A, jcs, okw):
    """The oracle over the same stream with each batch step's selection re-synchronised to the
    GPU's (the decisions that differ are listed in o.flips with their margins)."""
    o = Oracle(RIDConfig(m=A.shape[0], **okw))
    o.resync = {b: jc for b, jc in enumerate(jcs)}
    o.ingest(A)
    J, P = o.finalize()
    return o, J, P


def assert_parity(o, Jo, Po, g, Jg, Pg, A):
    """Parity of the GPU run g with the oracle run o on the same stream.  When J differs, every
    decision that went the other way must be a near tie (its score within MARGIN of the value
    at which it flips): the oracle is re-run with its selection re-synchronised to the GPU's at
    each batch step, and the comparison of P and of the estimates continues against it.
    Returns False when a re-synchronisation was needed."""
    S_o = o.S
    S_g = g.state(0)
    assert S_g.shape == S_o.shape
    assert np.abs(S_g - S_o).max() <= 1e-12 * np.abs(S_o).max()
    fro = g.state(3)
    assert abs(fro[0] - o.fro2) <= 1e-13 * o.fro2
    synced = True
    if not np.array_equal(Jg, Jo):
        o, Jo, Po = resynced_oracle(A, g.jcs, g.okw)
        assert o.flips, "J differs, yet every decision agrees on the GPU's selections"
        for (b, i, kind, mg) in o.flips:
            assert mg <= MARGIN, ("decision far from its threshold went the other way", b, i, kind, mg)
        assert np.array_equal(Jg, Jo)
        synced = False
    # Algorithms 5 and 7 solve through the Gram matrix A_J^T A_J, so two correct FP64
    # implementations agree to ~kappa(A_J)^2 * eps; the bar is 1e-10 unless the basis is
    # ill-conditioned enough for that bound to exceed it.
    act = Jo >= 0
    kappa = np.linalg.cond(A[:, Jo[act]]) if act.any() else 1.0
    tol = max(P_TOL, 10.0 * kappa ** 2 * np.finfo(np.float64).eps)
    err = np.linalg.norm(Pg - Po) / max(np.linalg.norm(Po), 1e-300)
    assert err <= tol, (err, tol, kappa)
    sq, fro_est, q = g.error_estimate()
    est_o, q_o = o.error_estimates()
    etol = max(1e-9, 10.0 * kappa ** 2 * np.finfo(np.float64).eps) * o.fro2
    assert np.abs(sq[1:] - est_o).max() <= etol, (sq[1:], est_o)
    srt = np.sort(est_o)
    if srt[1] - srt[0] > 2 * etol:
        assert q == q_o
    return synced


@pytest.mark.parametrize("seed", list(range(10)))
@pytest.mark.parametrize("omega", ["rademacher", "gaussian"])
def test_config1_fixed_lambda(seed, omega):
    A = config1_matrix(seed)
    k = 20
    lam = offline.tail_energy(A, k) / k
    kw = dict(k=k, s=4 * k + 3, h=30, lambda_mode="fixed", lambda_fixed=lam, omega_kind=omega, seed=seed)
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, **kw)
    assert_parity(o, Jo, Po, g, Jg, Pg, A)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("omega", ["rademacher", "gaussian"])
def test_config1_streaming_lambda(seed, omega):
    A = config1_matrix(seed)
    k = 20
    kw = dict(k=k, s=4 * k + 3, h=30, omega_kind=omega, seed=seed)
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, **kw)
    assert_parity(o, Jo, Po, g, Jg, Pg, A)
    # lambda depends on the sketch and ||A_obs||^2 only, not on the selection
    lam_g = g.state(6)[0]
    assert abs(lam_g - o.history[-1].lam) <= 1e-9 * abs(o.history[-1].lam) + 1e-13 * o.fro2


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("lambda_mode", ["fixed", "streaming"])
def test_config1_proportional_refill(seed, lambda_mode):
    """The alternative refill reading (a refilled slot draws its column with probability
    proportional to the ridge score) on the GPU against the oracle's."""
    A = config1_matrix(seed)
    k = 20
    lam = offline.tail_energy(A, k) / k
    kw = dict(k=k, s=4 * k + 3, h=30, lambda_mode=lambda_mode, lambda_fixed=lam, seed=seed, refill="proportional")
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, **kw)
    assert_parity(o, Jo, Po, g, Jg, Pg, A)
    # the reading changes the selection: the first-success run of the same stream differs
    o1, J1, _ = run_oracle(A, **{**kw, "refill": "first"})
    assert not np.array_equal(J1, Jo)


@pytest.mark.parametrize("lookahead", [2, 3, 4])
def test_lookahead_does_not_change_results(lookahead):
    """How far the ingest runs ahead of the batch steps (and so the pool slots each batch lands
    in) changes the schedule only: J, P and the estimates are bit-identical to the default's."""
    A = config1_matrix(5)
    k = 20
    kw = dict(k=k, s=83, h=30, seed=5)
    g0, J0, P0 = run_gpu(A, block=7, **kw)
    e0 = g0.error_estimate()[0]
    g, J, P = run_gpu(A, block=7, lookahead=lookahead, **kw)
    assert np.array_equal(J, J0)
    assert np.array_equal(P, P0)
    assert np.array_equal(g.error_estimate()[0], e0)
    o, Jo, Po = run_oracle(A, **kw)
    assert_parity(o, Jo, Po, g, J, P, A)


def test_last_batch_candidates_match():
    A = config1_matrix(3)
    k = 20
    kw = dict(k=k, s=83, h=30, seed=3)
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, **kw)
    assert np.array_equal(Jo, Jg)
    na = len(o._last_active)
    cand = g.candidates(A.shape[1])
    for q in range(4):
        ref = o._last_candidates[q]
        got = cand[q][:na]
        assert np.linalg.norm(got - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300), q


@pytest.mark.parametrize("block", [1, 7, 16])
def test_block_size_and_host_input_invariance(block):
    A = config1_matrix(5)[:, :120]
    kw = dict(k=20, s=83, h=30, seed=5)
    _, J1, P1 = run_gpu(A, block=1, **kw)
    gb, Jb, Pb = run_gpu(A, block=block, host=(block == 7), **kw)
    assert np.array_equal(J1, Jb)
    assert np.array_equal(P1, Pb)


@pytest.mark.parametrize("m,n,k,s,h", [
    (1000, 53, 6, 27, 12),      # m not a multiple of the tile, tail batch of 5
    (50, 30, 4, 19, 9),         # m smaller than one tile
    (777, 40, 1, 5, 6),         # t = 1
    (513, 45, 5, 23, 0),        # shared-row NA-Hutch++ (h = 0)
    (2049, 64, 16, 67, 30),     # n a multiple of t: no tail batch
])
def test_edge_shapes(m, n, k, s, h):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, 12)) @ np.diag(0.7 ** np.arange(12)) @ rng.standard_normal((12, n))
    A += 1e-3 * rng.standard_normal((m, n))
    A = np.asfortranarray(A)
    kw = dict(k=k, s=s, h=h, seed=11)
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, block=3, **kw)
    assert Pg.shape == (k, n)
    assert_parity(o, Jo, Po, g, Jg, Pg, A)


def test_capacity_growth_and_reset():
    A = config1_matrix(7)[:, :100]
    kw = dict(k=20, s=83, h=30, seed=7)
    _, J1, P1 = run_gpu(A, n_max=1024, **kw)
    g, J2, P2 = run_gpu(A, n_max=8, **kw)
    assert np.array_equal(J1, J2) and np.array_equal(P1, P2)
    torch, _ = _gpu()
    g.reset()
    g.ingest(torch.from_numpy(np.ascontiguousarray(A.T)).cuda())
    J3, P3 = g.finalize()
    assert np.array_equal(J1, J3) and np.array_equal(P1, P3)


def test_nonfinite_snapshot_is_reported():
    torch, rid = _gpu()
    A = config1_matrix(1)[:, :30].copy()
    A[17, 12] = np.nan
    g = rid.OnlineRID(m=A.shape[0], k=5, s=23, h=12, dtype="f64")
    g.ingest(torch.from_numpy(np.ascontiguousarray(A.T)).cuda())
    with pytest.raises(rid.RIDError) as e:
        g.finalize()
    assert e.value.code == rid.RID_ENONFINITE


def test_fp32_data_matches_fp64_oracle_within_fp32_accuracy():
    A64 = config1_matrix(2)
    A = A64.astype(np.float32).astype(np.float64)
    kw = dict(k=20, s=83, h=30, seed=2)
    o, Jo, Po = run_oracle(A, **kw)
    g, Jg, Pg = run_gpu(A, dtype="f32", **kw)
    S_o, S_g = o.S, g.state(0)
    scale = np.linalg.norm(A, axis=0)[None, :]
    assert np.abs(S_g - S_o).max() <= 1e-5 * scale.max()
    eo = offline.id_error(A, Jo, Po) / np.linalg.norm(A)
    eg = offline.id_error(A, Jg, Pg) / np.linalg.norm(A)
    if np.array_equal(Jg, Jo):
        assert np.linalg.norm(Pg - Po) <= 1e-3 * np.linalg.norm(Po)
    assert np.isfinite(eg)
