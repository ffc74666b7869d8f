"""The ingest launch-shape autotuner (rid_autotune) on the device.

A 1,048,576-coordinate FP32 stream with BF16x2 sketches (k = 20, s = 83, h = 30, 40 columns):
the tuner returns a group size that is a power of two in [1, 32] (32 is the first power of two
>= min(40, k)), a CTA count that is 0 (automatic) or one of the SM fractions it tries, and a
positive time per column, and writes one cache line; a second call returns the stored result
without measuring (the file keeps one line).  A handle with the tuned launch shape gives the
same results as one with the defaults: bit for bit when the CTA count stays automatic (the
sketch of a column does not depend on the group it was read with), and otherwise the sketch
within the BF16x2 bar of 2e-5 ||a_j||_2 (another CTA count sums the per-CTA partials of the
later batches in another order).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_autotune_launch_shape_cache_and_results(tmp_path, monkeypatch):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n, k, s, h = 1 << 20, 40, 20, 83, 30
    gen = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn((n, m), generator=gen, device="cuda", dtype=torch.float32)   # row j = column j
    cache = tmp_path / "rid_tune.txt"
    monkeypatch.setenv("RID_AUTOTUNE_CACHE", str(cache))
    kw = dict(dtype="f32", sketch="bf16x2", seed=5)
    G, C, us = rid.autotune_group(X, m, k, s, h, **kw)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert G in (1, 2, 4, 8, 16, 32) and us > 0.0
    assert C == 0 or C in [max(1, n_sm * q // 6) for q in range(1, 7)]
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    key, g_txt, c_txt, us_txt = lines[0].split()
    assert int(g_txt) == G and int(c_txt) == C and "|m1048576|k20|s83|h30|" in key
    G2, C2, us2 = rid.autotune_group(X, m, k, s, h, **kw)
    assert (G2, C2) == (G, C) and us2 == pytest.approx(float(us_txt), rel=1e-12)
    assert len(cache.read_text().splitlines()) == 1
    outs = []
    for gm, ct in ((G, C), (0, 0)):
        hd = rid.OnlineRID(m=m, k=k, s=s, h=h, n_max=n, defer=True, group_max=gm, ingest_ctas=ct, **kw)
        for j0 in range(0, n, 8):
            hd.ingest(X[j0:j0 + 8])
        J, P = hd.finalize()
        outs.append((hd.state(rid.RID_STATE_SKETCH), J, P))
        hd.close()
    if C == 0:
        assert np.array_equal(outs[0][0], outs[1][0])
        assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])
    else:
        norms = X.double().norm(dim=1).cpu().numpy()
        assert (np.abs(outs[0][0] - outs[1][0]) / norms[None, :]).max() <= 2e-5
