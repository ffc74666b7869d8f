"""rid_sketch_noalloc against the handle's own ingest sketch.

This file is named to be collected after every other test module, so that a run that stops at
its first failure has run everything else when it reaches these tests.

The allocation-free entry point must give the sketch and squared norms that
a handle (rid_init + rid_ingest + rid_get_state) records for the same
columns, within the bars the parity tests use for the sketch: 1e-12 of the
largest entry for FP64 data, 1e-5 of the largest column norm for FP32 data.
Two calls run back to back on one stream -- the first with the maximum 16
columns, the second with fewer columns and other data -- so that what the
first call leaves in the shared scratch cannot leak into the second.
"""
import ctypes

import numpy as np
import pytest


def _lib():
    from paper_2405_16076_gb300 import rid
    return rid


def _cfg(rid, m, s, h, seed, dtype, stream=0):
    cfg = rid.rid_config()
    assert rid.rid_config_default(ctypes.byref(cfg)) == rid.RID_OK
    cfg.m, cfg.k, cfg.s, cfg.h = m, 100, s, h
    cfg.seed = seed
    cfg.data_dtype = rid.RID_F64 if dtype == "f64" else rid.RID_F32
    cfg.omega_kind = rid.RID_OMEGA_RADEMACHER
    cfg.cuda_stream = ctypes.c_void_p(stream)
    return cfg


def test_noalloc_rejects_sizes_beyond_its_limits():
    """Host-side checks: nothing is launched, the error names the limit."""
    rid = _lib()
    cfg = _cfg(rid, 1000, 403, 50, 1, "f64")
    dummy = ctypes.c_void_p(16)
    rc = rid.rid_sketch_noalloc(ctypes.byref(cfg), dummy, 1000, 17, dummy, 453, dummy)
    assert rc == rid.RID_EINVAL
    assert b"16" in rid.rid_last_error(None)
    cfg.s, cfg.h = 480, 40
    rc = rid.rid_sketch_noalloc(ctypes.byref(cfg), dummy, 1000, 4, dummy, 520, dummy)
    assert rc == rid.RID_EINVAL
    assert b"512" in rid.rid_last_error(None)
    cfg.s, cfg.h = 403, 50
    cfg.omega_kind = rid.RID_OMEGA_GAUSSIAN
    assert rid.rid_sketch_noalloc(ctypes.byref(cfg), dummy, 1000, 4, dummy, 453, dummy) == rid.RID_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_sketch_matches_handle_on_two_calls(dtype):
    import torch
    rid = _lib()
    m, s, h, seed = 300_001, 403, 50, 11          # ragged m: many 256-coordinate chunks per block
    tdt = torch.float64 if dtype == "f64" else torch.float32
    gen = torch.Generator(device="cpu").manual_seed(5)
    X1 = torch.randn(16, m, generator=gen, dtype=torch.float64).to(tdt).cuda()    # row q = column q
    X2 = (3.0 * torch.rand(5, m, generator=gen, dtype=torch.float64) - 1.0).to(tdt).cuda()

    # existing entry point: one handle ingests both blocks (no batch step: 21 < t = 100)
    g = rid.OnlineRID(m=m, k=100, s=s, h=h, dtype=dtype, seed=seed)
    g.ingest(X1)
    g.ingest(X2)
    S_ref = g.state(rid.RID_STATE_SKETCH)                    # (s+h) x 21
    fro_ref = g.state(rid.RID_STATE_FRO2)[0]
    g.close()

    torch.cuda.synchronize()                                 # inputs complete before the side stream reads them
    stream = torch.cuda.Stream()
    cfg = _cfg(rid, m, s, h, seed, dtype, stream.cuda_stream)
    rows = s + h
    outs = []
    for X in (X1, X2):
        nb = X.shape[0]
        S = torch.full((nb, rows + 3), float("nan"), dtype=torch.float64, device="cuda")   # lds = rows + 3
        nrm = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
        rc = rid.rid_sketch_noalloc(ctypes.byref(cfg), ctypes.c_void_p(X.data_ptr()), m, nb,
                                    ctypes.c_void_p(S.data_ptr()), rows + 3, ctypes.c_void_p(nrm.data_ptr()))
        assert rc == rid.RID_OK, rid.rid_last_error(None)
        outs.append((S, nrm))
    stream.synchronize()

    S_na = np.concatenate([S[:, :rows].cpu().numpy().T for S, _ in outs], axis=1)
    norms = np.concatenate([n.cpu().numpy() for _, n in outs])
    assert np.isfinite(S_na).all() and np.isfinite(norms).all()
    # the padding rows past s + h are untouched
    assert all(torch.isnan(S[:, rows:]).all().item() for S, _ in outs)
    if dtype == "f64":
        bar = 1e-12 * np.abs(S_ref).max()
        assert np.abs(norms.sum() - fro_ref) <= 1e-13 * fro_ref
    else:
        bar = 1e-5 * np.sqrt(norms.max())
        assert np.abs(norms.sum() - fro_ref) <= 1e-6 * fro_ref
    assert np.abs(S_na[:, :16] - S_ref[:, :16]).max() <= bar
    assert np.abs(S_na[:, 16:] - S_ref[:, 16:]).max() <= bar
    Xd = np.concatenate([X1.double().cpu().numpy(), X2.double().cpu().numpy()])
    np.testing.assert_allclose(norms, (Xd * Xd).sum(axis=1), rtol=1e-12 if dtype == "f64" else 1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("m", [1, 255, 257, 40_000])
@pytest.mark.parametrize("ncols", [1, 16])
@pytest.mark.parametrize("rows", [256, 257, 512])
def test_noalloc_edge_sizes_against_exact_sketch(m, ncols, rows):
    """The short paths of the fixed-scratch sketch: fewer split-K blocks than the maximum (m below
    32768), a single partial chunk (m < 256), one column, and s + h on both sides of the 256-row
    boundary of the second row group.  Every output entry is compared with the exact FP64 sketch
    Omega a (the Rademacher entries of the counter-based generator); the outputs start as NaN, so
    an entry the kernels never wrote, or a partial sum read before it was written, fails."""
    import torch
    from oracle import philox
    rid = _lib()
    s = rows - 30
    h = 30
    seed = 7 + m + ncols
    gen = torch.Generator(device="cpu").manual_seed(m * 31 + ncols)
    X = (torch.rand(ncols, m, generator=gen, dtype=torch.float64) * 2.0 - 1.0).cuda()   # row q = column q
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    cfg = _cfg(rid, m, s, h, seed, "f64", stream.cuda_stream)
    for call in range(2):                                  # twice: the shared scratch keeps the first call's partials
        S = torch.full((ncols, rows + 1), float("nan"), dtype=torch.float64, device="cuda")
        nrm = torch.full((ncols,), float("nan"), dtype=torch.float64, device="cuda")
        rc = rid.rid_sketch_noalloc(ctypes.byref(cfg), ctypes.c_void_p(X.data_ptr()), m, ncols,
                                    ctypes.c_void_p(S.data_ptr()), rows + 1, ctypes.c_void_p(nrm.data_ptr()))
        assert rc == rid.RID_OK, rid.rid_last_error(None)
        stream.synchronize()
        A = X.cpu().numpy().T                              # m x ncols
        Om = philox.omega_block("rademacher", seed, np.arange(rows), 0, m)
        S_ref = Om @ A
        S_na = S[:, :rows].cpu().numpy().T
        assert np.isfinite(S_na).all() and np.isfinite(nrm.cpu().numpy()).all()
        assert torch.isnan(S[:, rows:]).all().item()
        assert np.abs(S_na - S_ref).max() <= 1e-12 * max(np.abs(S_ref).max(), 1e-300)
        np.testing.assert_allclose(nrm.cpu().numpy(), (A * A).sum(axis=0), rtol=1e-12)
        X = X.flip(1).contiguous() * 0.5                   # other data for the second call
        torch.cuda.synchronize()
