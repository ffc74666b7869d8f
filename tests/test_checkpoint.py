"""Checkpoint / resume: a stream checkpointed part-way, restored into a fresh handle and
continued gives exactly the results of the uninterrupted stream (same kernels, same order)."""
import numpy as np
import pytest

from workloads import config1_matrix

pytestmark = pytest.mark.gpu


def _run(rid, torch, A, split, dtype, sketch, **kw):
    m, n = A.shape
    npd = np.float64 if dtype == "f64" else np.float32
    src = torch.from_numpy(np.ascontiguousarray(A.T.astype(npd))).cuda()

    def mk():
        return rid.OnlineRID(m=m, dtype=dtype, sketch=sketch, n_max=n, **kw)

    ref = mk()
    for j0 in range(0, n, 7):
        ref.ingest(src[j0:j0 + 7])
    J0, P0 = ref.finalize()
    e0 = ref.error_estimate()[0]
    ref.close()

    first = mk()
    for j0 in range(0, split, 7):
        first.ingest(src[j0:min(split, j0 + 7)])
    state = first.checkpoint()
    first.close()
    second = mk()
    second.restore(state)
    assert second.n_obs() == split
    for j0 in range(split, n, 7):
        second.ingest(src[j0:min(n, j0 + 7)])
    J1, P1 = second.finalize()
    e1 = second.error_estimate()[0]
    second.close()
    return (J0, P0, e0), (J1, P1, e1)


@pytest.mark.parametrize("split", [25, 60, 131])
def test_checkpoint_resume_fp64(split):
    import torch
    from paper_2405_16076_gb300 import rid
    A = config1_matrix(4)
    (J0, P0, e0), (J1, P1, e1) = _run(rid, torch, A, split, "f64", "native", k=20, s=83, h=30, seed=4)
    assert np.array_equal(J0, J1)
    assert np.array_equal(P0, P1)
    assert np.array_equal(e0, e1)


def test_checkpoint_resume_tensor_cores():
    import torch
    from paper_2405_16076_gb300 import rid
    A = config1_matrix(5)
    (J0, P0, e0), (J1, P1, e1) = _run(rid, torch, A, 90, "f32", "bf16x2", k=20, s=83, h=30, seed=5)
    assert np.array_equal(J0, J1)
    assert np.array_equal(P0, P1)


def test_restore_rejects_other_configuration():
    import torch
    from paper_2405_16076_gb300 import rid
    A = config1_matrix(6)
    src = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    a = rid.OnlineRID(m=A.shape[0], k=20, s=83, h=30, dtype="f64", seed=6)
    a.ingest(src[:10])
    state = a.checkpoint()
    b = rid.OnlineRID(m=A.shape[0], k=20, s=83, h=30, dtype="f64", seed=7)
    with pytest.raises(rid.RIDError):
        b.restore(state)
    with pytest.raises(rid.RIDError):
        a.restore(state[:100])
    a.close()
    b.close()


@pytest.mark.parametrize("field,value", [("nslots", -1), ("count", 21), ("count", -3), ("n_prev", 10 ** 6),
                                         ("finalized", 2), ("batch", -1), ("nslots", 10 ** 6)])
def test_restore_rejects_inconsistent_counters(field, value):
    """A checkpoint whose counters were corrupted is rejected with RID_EINVAL before the handle
    changes: the live stream it was offered to continues exactly as an untouched one."""
    import ctypes
    import torch
    from paper_2405_16076_gb300 import rid
    A = config1_matrix(7)
    m, n = A.shape
    src = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    ref = rid.OnlineRID(m=m, k=20, s=83, h=30, dtype="f64", seed=8, n_max=n)
    ref.ingest(src[:n])
    J0, P0 = ref.finalize()
    ref.close()
    a = rid.OnlineRID(m=m, k=20, s=83, h=30, dtype="f64", seed=8, n_max=n)
    a.ingest(src[:45])
    state = bytearray(a.checkpoint())
    # counters follow the magic number and the configuration: int64 n_obs, n_prev, then int32
    # count, batch, finalized, nslots
    off = 8 + ctypes.sizeof(rid.rid_config)
    fields = {"n_obs": (0, "<q"), "n_prev": (8, "<q"), "count": (16, "<i"), "batch": (20, "<i"),
              "finalized": (24, "<i"), "nslots": (28, "<i")}
    import struct
    o, fmt = fields[field]
    struct.pack_into(fmt, state, off + o, value)
    with pytest.raises(rid.RIDError) as ei:
        a.restore(bytes(state))
    assert ei.value.code == rid.RID_EINVAL
    assert a.n_obs() == 45
    a.ingest(src[45:n])
    J1, P1 = a.finalize()
    a.close()
    assert np.array_equal(J0, J1)
    assert np.array_equal(P0, P1)
