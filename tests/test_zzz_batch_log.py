"""The per-batch log (rid_log_enable / rid_get_log) against the oracle's history of batch steps.

Configuration 1 with streaming lambda (m = 4096, n = 256, k = t = 20, s = 83, h = 30, FP64,
one column per call): 13 batch steps, the last one the tail step of finalize.  Each record must
match the oracle's step: its index and column count exactly, lambda within 1e-9 (the bar of the
streaming-lambda parity test), ||A_obs||^2 within 1e-13, the four estimates within the FP64
parity bar max(1e-9, 10 kappa(A_J)^2 eps) ||A_obs||^2, q* wherever the estimates are further
apart than twice that bar, and the slot counts (active, kept, new) exactly; FP64 sketches carry
no rounding uncertainty.  A log shorter than the stream keeps its newest records, and rid_reset
empties it.
"""
import numpy as np
import pytest

from oracle.rid import OnlineRID as Oracle, RIDConfig
from workloads import config1_matrix

pytestmark = pytest.mark.gpu

K, S, H, SEED = 20, 83, 30, 3


def _run(A, capacity):
    import torch
    from paper_2405_16076_gb300 import rid
    g = rid.OnlineRID(m=A.shape[0], k=K, s=S, h=H, dtype="f64", seed=SEED)
    g.log_enable(capacity)
    src = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j in range(A.shape[1]):
        g.ingest(src[j:j + 1])
    J, P = g.finalize()
    return g, J, P


def test_batch_log_matches_the_oracle_history():
    A = config1_matrix(SEED)
    o = Oracle(RIDConfig(m=A.shape[0], k=K, s=S, h=H, seed=SEED))
    o.ingest(A)
    Jo, _ = o.finalize()
    g, J, _ = _run(A, 64)
    assert np.array_equal(J, Jo)
    log = g.log()
    hist = o.history
    assert len(log) == len(hist) == 13
    csq = np.cumsum(np.sum(A * A, axis=0))
    eps = np.finfo(np.float64).eps
    for rec, hr in zip(log, hist):
        assert rec["batch"] == hr.batch and rec["n_obs"] == hr.n_obs
        fro2 = csq[hr.n_obs - 1]
        assert abs(rec["fro2"] - fro2) <= 1e-13 * fro2
        assert abs(rec["lambda"] - hr.lam) <= 1e-9 * abs(hr.lam) + 1e-13 * fro2
        act = hr.JC >= 0
        kappa = np.linalg.cond(A[:, hr.JC[act]])
        etol = max(1e-9, 10.0 * kappa ** 2 * eps) * fro2
        est = np.array(rec["est_sq"])
        assert np.abs(est - hr.est_sq).max() <= etol, (hr.batch, est, hr.est_sq)
        srt = np.sort(hr.est_sq)
        if srt[1] - srt[0] > 2 * etol:
            assert rec["q_star"] == hr.q_star
        assert rec["n_active"] == int(act.sum())
        assert rec["n_kept"] == int(np.sum(hr.kept))
        assert rec["n_new"] == rec["n_active"] - rec["n_kept"]
        assert rec["est_unc"] == [0.0] * 4 and rec["gram_shift"] >= 0.0
    g2, J2, _ = _run(A, 5)
    assert np.array_equal(J2, J)
    assert g2.log() == log[-5:]
    assert g2.log(max_records=2) == log[-2:]
    g2.reset()
    assert g2.log() == []
    g.close()
    g2.close()
