"""GPU <-> oracle parity in gradient mode (Sec. 3.4, Eqs. 38-43).

The ridge scores and lambda use the sketch of [a; G a] with an independent
Omega_g and the norm ||a||^2 + ||G a||^2 (reading R16); everything else uses the
plain sketch.  Same bars as the FP64 parity tests: leverage sketch within
1e-12 of its largest entry, norms within 1e-13, indices bit-exact unless an
oracle decision lies within 1e-10 of its threshold, coefficients within
max(1e-10, 10 kappa^2 eps).
"""
import numpy as np
import pytest

from oracle.gradient import grid_gradient_operator
from oracle.rid import OnlineRID as Oracle, RIDConfig
from test_parity_small import assert_parity

pytestmark = pytest.mark.gpu


def grid_stream(nx, ny, nfields, n, seed):
    """Smooth travelling modes on an nx x ny grid per field (x fastest), plus small noise."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    A = np.empty((nx * ny * nfields, n))
    modes = [(rng.integers(-3, 4), rng.integers(-3, 4), rng.uniform(0, 2 * np.pi), 1.0 / (1 + q))
             for q in range(12)]
    for j in range(n):
        cols = []
        for f in range(nfields):
            fld = np.zeros((ny, nx))
            for q, (a, b, c, amp) in enumerate(modes):
                w = rng.standard_normal() if f == 0 else np.cos(0.3 * j + q + f)
                fld += amp * w * np.cos(2 * np.pi * (a * x + b * y) + c + 0.05 * j * (q + 1))
            cols.append(fld.reshape(-1))              # row-major (y, x): x fastest
        A[:, j] = np.concatenate(cols)
    return A + 1e-3 * rng.standard_normal(A.shape)


def run_both(A, nx, ny, nfields, **kw):
    from paper_2405_16076_gb300 import rid
    import torch
    m, n = A.shape
    G = grid_gradient_operator((nx, ny), nfields=nfields)
    o = Oracle(RIDConfig(m=m, grad_op=G, **kw))
    o.ingest(A)
    Jo, Po = o.finalize()
    g = rid.OnlineRID(m=m, k=kw["k"], s=kw["s"], h=kw["h"], dtype="f64", omega=kw["omega_kind"],
                      seed=kw["seed"], n_max=n, grad_dims=2, nx=nx, ny=ny, nfields=nfields)
    src = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    jcs, t = [], kw["k"]
    for j0 in range(0, n, 5):
        g.ingest(src[j0:j0 + 5])
        while len(jcs) < min(j0 + 5, n) // t:              # selections per batch step, for re-syncs
            jcs.append(g.state(rid.RID_STATE_JC).copy())
    Jg, Pg = g.finalize()
    if n % t:
        jcs.append(Jg.copy())
    g.jcs, g.okw = jcs, dict(kw, grad_op=G)
    return o, Jo, Po, g, Jg, Pg


@pytest.mark.parametrize("omega", ["rademacher", "gaussian"])
@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_mode_matches_oracle(omega, seed):
    nx, ny, nfields = 24, 16, 3
    A = grid_stream(nx, ny, nfields, 60, seed)
    kw = dict(k=10, s=43, h=30, omega_kind=omega, seed=seed)
    o, Jo, Po, g, Jg, Pg = run_both(A, nx, ny, nfields, **kw)
    lev_g = g.state(1)                                   # leverage sketch, s x n
    assert lev_g.shape == o.S_lev.shape
    assert np.abs(lev_g - o.S_lev).max() <= 1e-12 * np.abs(o.S_lev).max()
    fro = g.state(3)
    assert abs(fro[1] - o.fro2_lev) <= 1e-13 * o.fro2_lev
    assert o.fro2_lev > o.fro2                          # the gradient term is present
    assert_parity(o, Jo, Po, g, Jg, Pg, A)
    g.close()


def test_gradient_mode_rejects_bad_grids():
    from paper_2405_16076_gb300 import rid
    with pytest.raises(rid.RIDError):
        rid.OnlineRID(m=100, k=5, s=23, h=0, dtype="f64", grad_dims=2, nx=10, ny=9, nfields=1)   # m != nx ny
    with pytest.raises(rid.RIDError):        # E4M3 sketches have no gradient form
        rid.OnlineRID(m=100, k=5, s=23, h=0, dtype="f32", sketch="fp8x2", grad_dims=2, nx=10, ny=10)
    with pytest.raises(rid.RIDError):        # the coefficient sketches run on the native path
        rid.OnlineRID(m=100, k=5, s=23, h=0, dtype="f32", sketch="bf16x2", grad_dims=2, nx=10, ny=10,
                      grad_coeff=True)
    with pytest.raises(rid.RIDError):
        rid.OnlineRID(m=100, k=5, s=23, h=0, dtype="f64", grad_dims=3, nx=10, ny=10)
