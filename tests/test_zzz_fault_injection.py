"""Allocation failures injected on the host (RID_FAULT_INJECT=alloc:<n>); no GPU fault is involved.

rid_init fails cleanly at each of its device allocations in turn: RID_ENOMEM, no handle, and no
device memory left behind (free memory after the sweep within 64 MiB of its value before it,
where a leaked buffer-slot pool alone would be 320 MiB per failure).  A failure in a later
capacity growth leaves the handle usable: after the failed rid_ingest the recorded columns are
sketched by the next rid_sync, and the stream ends with the same J and P, bit for bit, as a run
without injection (same group boundaries, same kernels).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M, K, S, H = 1 << 20, 20, 83, 30


def test_injected_allocation_failures_in_init_and_growth(monkeypatch):
    import torch
    from paper_2405_16076_gb300 import rid
    kw = dict(dtype="f32", sketch="bf16x2", seed=9)
    cfg = rid.make_config(M, K, S, H, n_max=64, **kw)
    monkeypatch.delenv("RID_FAULT_INJECT", raising=False)
    h = ctypes.c_void_p()
    assert rid.rid_init(ctypes.byref(h), ctypes.byref(cfg)) == rid.RID_OK     # context warm
    rid.rid_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_init = None
    for n in range(1, 200):
        monkeypatch.setenv("RID_FAULT_INJECT", f"alloc:{n}")
        h = ctypes.c_void_p()
        rc = rid.rid_init(ctypes.byref(h), ctypes.byref(cfg))
        if rc == rid.RID_OK:                     # n is past the last allocation of rid_init
            rid.rid_destroy(h)
            n_init = n - 1
            break
        assert rc == rid.RID_ENOMEM, (n, rc)
        assert not h.value
        assert b"allocation" in rid.rid_last_error(None)
    assert n_init is not None and n_init >= 20
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= 64 << 20, (free0, free1)

    gen = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn((60, M), generator=gen, device="cuda", dtype=torch.float32)   # row j = column j
    monkeypatch.delenv("RID_FAULT_INJECT")
    ref = rid.OnlineRID(m=M, k=K, s=S, h=H, n_max=8, **kw)
    for j0 in range(0, 60, 8):
        ref.ingest(X[j0:j0 + 8])
    Jr, Pr = ref.finalize()
    ref.close()

    monkeypatch.setenv("RID_FAULT_INJECT", f"alloc:{n_init + 1}")   # the first allocation after init
    g = rid.OnlineRID(m=M, k=K, s=S, h=H, n_max=8, **kw)
    monkeypatch.delenv("RID_FAULT_INJECT")
    g.ingest(X[0:8])                             # fits the capacity of 8 columns
    with pytest.raises(rid.RIDError) as e:
        g.ingest(X[8:16])                        # growth to 16 columns fails
    assert e.value.code == rid.RID_ENOMEM and "capacity growth" in str(e.value)
    g.sync()                                     # the recorded group goes through now
    for j0 in range(16, 60, 8):
        g.ingest(X[j0:j0 + 8])
    J, P = g.finalize()
    g.close()
    assert np.array_equal(J, Jr) and np.array_equal(P, Pr)


@pytest.mark.parametrize("sketch", ["bf16x2", "fp8x2"])
def test_bounded_pipeline_wait_gives_up_cleanly(monkeypatch, sketch):
    """RID_FAULT_INJECT=wait:1 gives the tensor-core kernels' pipeline waits a limit of one poll, so
    that the MMA issuer's first wait for a staged chunk runs out: the kernel raises the timeout bit
    of the device error word, every role stops at its next wait, the MMAs already issued are waited
    for with the full limit, TMEM is freed and the kernel returns.  The host sees RID_ETIMEOUT at
    the next synchronizing call; the context stays usable, and a handle created without the
    injection then gives the reference results."""
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = 300_000, 50
    kw = dict(dtype="f32", sketch=sketch, seed=11, n_max=n)
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((n, m), generator=gen, device="cuda", dtype=torch.float32)
    monkeypatch.delenv("RID_FAULT_INJECT", raising=False)
    ref = rid.OnlineRID(m=m, k=K, s=S, h=H, **kw)
    for j0 in range(0, n, 10):
        ref.ingest(X[j0:j0 + 10])
    Jr, Pr = ref.finalize()
    ref.close()

    monkeypatch.setenv("RID_FAULT_INJECT", "wait:1")
    g = rid.OnlineRID(m=m, k=K, s=S, h=H, **kw)
    monkeypatch.delenv("RID_FAULT_INJECT")
    for j0 in range(0, n, 10):
        g.ingest(X[j0:j0 + 10])
    with pytest.raises(rid.RIDError) as e:
        g.sync()
    assert e.value.code == rid.RID_ETIMEOUT, e.value
    g.close()
    torch.cuda.synchronize()                     # no sticky CUDA error: the kernels returned

    h2 = rid.OnlineRID(m=m, k=K, s=S, h=H, **kw)
    for j0 in range(0, n, 10):
        h2.ingest(X[j0:j0 + 10])
    J, P = h2.finalize()
    h2.close()
    assert np.array_equal(J, Jr) and np.array_equal(P, Pr)
