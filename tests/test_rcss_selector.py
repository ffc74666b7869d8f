"""Algorithm 1 as the selector of the online ID (the paper's online rows for the residual CSS,
Sec. 4.1): the coefficient updates (Algorithms 4-7) and Algorithm 8 on Algorithm 1's subset, on
the GPU against the oracle's ``selector="residual"``.

Algorithm 1's decisions are compared up to rounding as in ``test_rcss.py``: the streams here have
no decision within the GPU's rounding of a threshold (checked), so J must be identical; P and the
estimates meet the bars of the Algorithm 3 parity tests (1e-10, widened by kappa(A_J)^2 eps).
"""
import numpy as np
import pytest

from oracle.rid import OnlineRID as Oracle, RIDConfig
from test_rcss import first_near_tie
from workloads import config1_matrix

pytestmark = pytest.mark.gpu

P_TOL = 1e-10


def _run(A, k, s, h, xi, seed, rseed, block, dtype="f64"):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A.shape
    g = rid.OnlineRID(m=m, k=k, s=s, h=h, dtype=dtype, seed=seed, n_max=n)
    sel = rid.ResidualCSS(m, k, xi, seed=rseed, data_dtype=rid.RID_F64 if dtype == "f64" else rid.RID_F32,
                          cap=k, stop_at_cap=True)
    g.attach_rcss(sel)
    rows = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j0 in range(0, n, block):
        g.ingest(rows[j0:j0 + block])
    J, P = g.finalize()
    sq, _, q = g.error_estimate()
    chosen = sel.selection()[0]
    g.close()
    sel.close()
    return J, P, sq, q, chosen


@pytest.mark.parametrize("block", [1, 4])
def test_residual_selector_matches_oracle(block):
    """m = 3000, 400 snapshots of rank 40 plus noise, t = k = 10 (the subset fills over several
    batches), s = 43, h = 30, FP64."""
    A = config1_matrix(5, m=3000, n=400, r=40, noise_var=1e-7)
    m, n = A.shape
    k, s, h, seed, rseed = 10, 43, 30, 3, 7
    xi = 0.5 * k * float(np.median(np.einsum("ij,ij->j", A, A)))
    o = Oracle(RIDConfig(m=m, k=k, s=s, h=h, seed=seed, selector="residual", rcss_xi=xi, rcss_seed=rseed))
    o.ingest(A)
    Jo, Po = o.finalize()
    assert first_near_tie(o.rcss, A, k, xi, 1e-12) == n
    J, P, sq, q, chosen = _run(A, k, s, h, xi, seed, rseed, block)
    np.testing.assert_array_equal(chosen, o.rcss.selection())
    np.testing.assert_array_equal(J, Jo)
    act = Jo >= 0
    assert act.sum() == k                                  # the subset filled every slot
    assert sorted(J[act]) == sorted(o.rcss.selection())
    assert len({hh.JC.tobytes() for hh in o.history}) >= 3  # the basis grew over several steps
    kappa = np.linalg.cond(A[:, Jo[act]])
    tol = max(P_TOL, 10.0 * kappa ** 2 * np.finfo(np.float64).eps)
    assert np.linalg.norm(P - Po) <= tol * np.linalg.norm(Po)
    est_o, q_o = o.error_estimates()
    etol = max(1e-9, 10.0 * kappa ** 2 * np.finfo(np.float64).eps) * o.fro2
    assert np.abs(sq[1:] - est_o).max() <= etol
    srt = np.sort(est_o)
    if srt[1] - srt[0] > 2 * etol:
        assert q == q_o


def test_residual_selector_arguments():
    from paper_2405_16076_gb300 import rid
    g = rid.OnlineRID(m=500, k=8, s=35, h=12, dtype="f64", n_max=64)
    with pytest.raises(rid.RIDError):
        g.attach_rcss(rid.ResidualCSS(400, 8, 1.0, cap=8, stop_at_cap=True))     # m differs
    with pytest.raises(rid.RIDError):
        g.attach_rcss(rid.ResidualCSS(500, 8, 1.0, cap=9, stop_at_cap=True))     # cap > t
    with pytest.raises(rid.RIDError):
        g.attach_rcss(rid.ResidualCSS(500, 8, 1.0, cap=8, stop_at_cap=False))    # no cap
    with pytest.raises(rid.RIDError):
        g.attach_rcss(rid.ResidualCSS(500, 8, 1.0, data_dtype=rid.RID_F32, cap=8, stop_at_cap=True))
    sel = rid.ResidualCSS(500, 8, 1.0, cap=8, stop_at_cap=True)
    g.attach_rcss(sel)
    g.ingest(np.random.default_rng(0).standard_normal((500, 3)))
    with pytest.raises(rid.RIDError) as e:
        g.checkpoint()                                                           # not covered
    assert e.value.code == rid.RID_ESTATE
    with pytest.raises(rid.RIDError) as e:
        g.attach_rcss(None)                                                      # after an ingest
    assert e.value.code == rid.RID_ESTATE
    g.close()
    sel.close()
