"""SM partition (green contexts): the batch steps in one SM partition and the ingest in the
other change only where kernels run, so J, P and the estimates are bit-identical to the
unpartitioned handle's; a partition that cannot exist is refused at init."""
import numpy as np
import pytest

from workloads import config1_matrix

pytestmark = pytest.mark.gpu


def _run(A, dtype, sketch, batch_sms, block=7, lookahead=0):
    import torch
    from paper_2405_16076_gb300 import rid
    m, n = A.shape
    g = rid.OnlineRID(m=m, k=20, s=83, h=30, dtype=dtype, sketch=sketch, seed=4, batch_sms=batch_sms,
                      lookahead=lookahead)
    npd = np.float64 if dtype == "f64" else np.float32
    X = torch.from_numpy(np.ascontiguousarray(A.T.astype(npd))).cuda()
    for j0 in range(0, n, block):
        g.ingest(X[j0:j0 + block])
    J, P = g.finalize()
    est = g.error_estimate()[0]
    g.close()
    return J, P, est


@pytest.mark.parametrize("dtype,sketch", [("f32", "bf16x2"), ("f64", "native")])
@pytest.mark.parametrize("batch_sms", [32, 48])
def test_partition_does_not_change_results(dtype, sketch, batch_sms):
    A = config1_matrix(4)
    J0, P0, e0 = _run(A, dtype, sketch, 0)
    J1, P1, e1 = _run(A, dtype, sketch, batch_sms)
    assert np.array_equal(J0, J1)
    assert np.array_equal(P0, P1)
    assert np.array_equal(e0, e1)


def test_partition_with_lookahead_and_host_input():
    import torch
    from paper_2405_16076_gb300 import rid
    A = config1_matrix(6)
    J0, P0, _ = _run(A, "f32", "bf16x2", 0, lookahead=4)
    m, n = A.shape
    g = rid.OnlineRID(m=m, k=20, s=83, h=30, dtype="f32", sketch="bf16x2", seed=4, batch_sms=40, lookahead=4)
    rows = np.ascontiguousarray(A.T.astype(np.float32))
    for j0 in range(0, n, 5):
        g.ingest(rows[j0:j0 + 5])                       # host columns: copy stream, then the ingest stream
    J1, P1 = g.finalize()
    g.close()
    assert np.array_equal(J0, J1) and np.array_equal(P0, P1)


def test_partition_refused_when_impossible():
    import torch
    from paper_2405_16076_gb300 import rid
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    with pytest.raises(rid.RIDError) as e:
        rid.OnlineRID(m=1000, k=5, s=23, h=0, dtype="f32", sketch="bf16x2", batch_sms=n_sm)
    assert e.value.code == rid.RID_EINVAL
