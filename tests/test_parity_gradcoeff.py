"""GPU <-> oracle parity of Sec. 3.4's gradient-augmented coefficients (sketched GCV).

The streamed sketches Omega G^p a_j match the oracle's within 1e-12 of their largest entry
(FP64).  The golden-section search compares GCV values; near the minimum two probes can differ
by rounding only, so lambda* is checked by the oracle's own GCV: the GPU's lambda* is at least
as good as the oracle's (to 1e-9 relative) and the two lie within a few final brackets.  At the
GPU's lambda*, GCV and P(lambda*) match the oracle's within 1e-10 relative.
"""
import math

import numpy as np
import pytest

from oracle import gcv
from oracle.gradient import grid_gradient_operator
from oracle.rid import OnlineRID as Oracle, RIDConfig
from test_parity_grad import grid_stream

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("omega", ["rademacher", "gaussian"])
def test_gradient_coefficients_match_oracle(omega):
    import torch
    from paper_2405_16076_gb300 import rid
    nx, ny, nf, n = 24, 16, 2, 60
    A = grid_stream(nx, ny, nf, n, 3)
    m = A.shape[0]
    kw = dict(k=10, s=43, h=30, omega_kind=omega, seed=3)
    G = grid_gradient_operator((nx, ny), nfields=nf)
    o = Oracle(RIDConfig(m=m, grad_op=G, grad_coeff=True, **kw))
    o.ingest(A)
    Jo, _ = o.finalize()
    lam_o, P_o, g_o = o.gradient_coefficients()

    g = rid.OnlineRID(m=m, k=10, s=43, h=30, dtype="f64", omega=omega, seed=3, n_max=n, grad_dims=2, nx=nx, ny=ny,
                      nfields=nf, grad_coeff=True)
    X = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    for j0 in range(0, n, 5):
        g.ingest(X[j0:j0 + 5])
    Jg, _ = g.finalize()
    assert np.array_equal(Jg, Jo)
    SG = g.state(rid.RID_STATE_GRAD_SKETCH)
    assert SG.shape == o.SG.shape
    assert np.abs(SG - o.SG).max() <= 1e-12 * np.abs(o.SG).max()
    lam_g, P_g, g_g = g.gradient_coefficients()
    g.close()

    # the oracle's quantities at the GPU's lambda*
    s = 43
    act = Jo >= 0
    S = o.S[:s] / math.sqrt(s)
    Gs = [o.SG[p] / math.sqrt(s) for p in range(2)]
    Om = o.omega()[:s]
    K = [Om @ (Gp @ Om.T) / s for Gp in gcv.split_gradient(G, m)]
    SJ, GJ = S[:, Jo[act]], [x[:, Jo[act]] for x in Gs]
    g_at = gcv.gcv(SJ, S, GJ, K, lam_g)
    assert g_at <= g_o * (1 + 1e-9)
    assert abs(math.log10(lam_g) - math.log10(lam_o)) <= 5e-3
    assert abs(g_g - g_at) <= 1e-10 * g_at
    P_ref = np.zeros_like(P_g)
    P_ref[act] = gcv.p_of_lambda(SJ, S, GJ, Gs, lam_g)
    assert np.linalg.norm(P_g - P_ref) <= 1e-10 * np.linalg.norm(P_ref)
    assert np.all(P_g[~act] == 0.0)


def test_gradient_coefficients_need_the_sketches():
    from paper_2405_16076_gb300 import rid
    with pytest.raises(rid.RIDError):
        rid.OnlineRID(m=100, k=5, s=23, h=12, dtype="f64", grad_coeff=True)     # no gradient mode
    g = rid.OnlineRID(m=100, k=5, s=23, h=12, dtype="f64", grad_dims=2, nx=10, ny=10)
    with pytest.raises(rid.RIDError):
        g.gradient_coefficients()
    g.close()
