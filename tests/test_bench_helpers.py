"""The benchmark's accuracy evaluation, on the CPU, against independent routes.

id_error_device (chunked FP64 residual norm on torch tensors) against numpy's norm of the
explicit residual; grad_field_error (x / y differences of the stacked fields by slicing)
against the gradient operator of Sec. 3.4 built from the grid graph (oracle.gradient)."""
import numpy as np
import torch

import bench
from oracle.gradient import grid_gradient_operator


def _case(seed, n, m, t):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)).astype(np.float32).astype(np.float64)
    J = np.array(list(rng.choice(n, size=t - 1, replace=False)) + [-1])     # one empty slot
    P = rng.standard_normal((t, n))
    P[-1] = 0.0
    return A, J, P


def test_id_error_matches_explicit_residual():
    A, J, P = _case(0, n=23, m=1000, t=6)
    X = torch.from_numpy(np.ascontiguousarray(A.T)).float()
    err, fro2 = bench.id_error_device(X, torch.from_numpy(J), torch.from_numpy(np.ascontiguousarray(P.T)), chunk=97)
    act = J >= 0
    ref = np.linalg.norm(A - A[:, J[act]] @ P[act]) / np.linalg.norm(A)
    assert abs(err - ref) <= 1e-12 * ref
    assert abs(fro2 - np.sum(A * A)) <= 1e-12 * np.sum(A * A)


def test_gradient_field_error_matches_grid_operator():
    N, nf, n, t = 7, 3, 9, 4
    A, J, P = _case(1, n=n, m=nf * N * N, t=t)
    X = torch.from_numpy(np.ascontiguousarray(A.T)).float()
    got = bench.grad_field_error(X, torch.from_numpy(J), torch.from_numpy(np.ascontiguousarray(P.T)),
                                 {"N": N, "nfields": nf}, chunk=4)
    G = grid_gradient_operator((N, N), nfields=nf)
    act = J >= 0
    R = A - A[:, J[act]] @ P[act]
    ref = np.linalg.norm(G @ R) / np.linalg.norm(G @ A)
    assert abs(got - ref) <= 1e-10 * ref


def test_reference_arm_prints_its_contract_line():
    """bench.py --impl reference (the oracle on the host cores, a bounded sample of the workload)
    prints one JSON line with the keys the benchmark contract asks of the reference arm."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--config",
                        "channel_small", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == "snapshots/s" and line["unit"] == "snapshots/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_single_thread_cpu_baseline_runs_on_one_core():
    r = bench.cpu_baseline_single_thread("channel_small")
    assert "error" not in r, r
    assert r["cores"] == 1 and r["value"] > 0 and r["unit"] == "snapshots/s"


def test_least_squares_error_closed_forms():
    """The tables' least-squares error: 0 when the chosen columns span the matrix, 1 for an empty
    choice, and the distance of the last column from the line of the first otherwise."""
    from paper_2405_16076_gb300 import tables
    A = np.array([[1.0, 2.0, 0.0], [0.0, 0.0, 1.0]])
    assert tables.least_squares_error(A, [0, 2]) <= 1e-15
    assert tables.least_squares_error(A, []) == 1.0
    assert abs(tables.least_squares_error(A, [0]) - 1.0 / np.linalg.norm(A)) <= 1e-15
