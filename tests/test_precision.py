"""Reduced-precision forms against the FP64 oracle (configuration C4).

The small low-rank stream (m = 4096, n = 256, k = 20, s = 83, h = 30, columns one at a time,
fixed lambda = ||A - A_k||_F^2 / k) runs through the FP64 oracle and, with the data in FP32,
through the plain FP32 sketch, the BF16x2 and BF16 tensor-core sketches and the block-scaled
E4M3 sketches (FP8x2, FP8).  Every form reports
its relative Frobenius reconstruction error; the target is at most 1.05 times the oracle's, taken
as the mean over seeds 0..9 (a sampling decision that flips under a rounding change moves one
seed's error either way).  The FP64 GPU path equals the oracle.
"""
import numpy as np
import pytest

from oracle.offline import id_error, tail_energy
from oracle.rid import OnlineRID as Oracle, RIDConfig
from workloads import config1_matrix

pytestmark = pytest.mark.gpu

K, S, H, M, N = 20, 83, 30, 4096, 256


def _gpu_error(A, lam, seed, dtype, sketch):
    import torch
    from paper_2405_16076_gb300 import rid
    g = rid.OnlineRID(m=M, k=K, s=S, h=H, dtype=dtype, sketch=sketch, lambda_mode="fixed", lambda_fixed=lam,
                      seed=seed, n_max=N)
    X = torch.from_numpy(np.ascontiguousarray(A.T, dtype=np.float64 if dtype == "f64" else np.float32)).cuda()
    for j in range(N):
        g.ingest(X[j:j + 1])
    J, P = g.finalize()
    g.close()
    return J, id_error(A, J, P) / np.linalg.norm(A)


def test_precision_forms_against_oracle():
    res = {"oracle": [], "f64": [], "f32": [], "bf16x2": [], "bf16": [], "fp8x2": [], "fp8": []}
    same_J = {"f32": 0, "bf16x2": 0, "bf16": 0, "fp8x2": 0, "fp8": 0}
    for seed in range(10):
        A = config1_matrix(seed)
        lam = tail_energy(A, K) / K
        o = Oracle(RIDConfig(m=M, k=K, s=S, h=H, lambda_mode="fixed", lambda_fixed=lam, seed=seed))
        o.ingest(A)
        Jo, Po = o.finalize()
        res["oracle"].append(id_error(A, Jo, Po) / np.linalg.norm(A))
        for name, dtype, sketch in (("f64", "f64", "native"), ("f32", "f32", "native"),
                                    ("bf16x2", "f32", "bf16x2"), ("bf16", "f32", "bf16"),
                                    ("fp8x2", "f32", "fp8x2"), ("fp8", "f32", "fp8")):
            J, e = _gpu_error(A, lam, seed, dtype, sketch)
            res[name].append(e)
            if name in same_J:
                same_J[name] += int(np.array_equal(J, Jo))
    mean = {key: float(np.mean(v)) for key, v in res.items()}
    print("mean relative errors", mean, "seeds with the oracle's J", same_J)
    assert np.allclose(res["f64"], res["oracle"], rtol=1e-8, atol=0)
    assert mean["f32"] <= 1.05 * mean["oracle"]
    assert mean["bf16x2"] <= 1.05 * mean["oracle"]
    assert same_J["bf16x2"] >= 8                     # BF16x2 keeps the oracle's decisions on most seeds
    # the two-term block-scaled E4M3 form (8 significant bits, like BF16) within the same bar; the
    # one-term form (4 bits) is reported, not bounded
    assert mean["fp8x2"] <= 1.05 * mean["oracle"]
