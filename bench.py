"""Benchmark of the single-pass online randomized ID ingest path on GB300.

Workload (default): the channel-flow-shaped stream -- three velocity
components on a 192 x 129 x 192 grid (m = 14,266,368 FP32 values per
snapshot), n = 1000 snapshots streamed in blocks of 8, k = t = 100,
s = 403 left-sketch rows, h = 50 NA-Hutch++ probe rows, Rademacher test
matrix, streaming lambda.  One step = one whole stream through the C ABI
(reset, 125 ingest calls with the batch step every 100 snapshots, finalize).

Prints one JSON line.  ``value`` is snapshots/s over all ranks with the
inputs resident in HBM; ``e2e`` is the same metric through rid_ingest with
pinned host buffers (host->device copies inside the timed region) and the
coefficients read back to the host.  ``roofline`` reports the fused
ingest/sketch kernel (the dominant kernel), timed live with CUDA events on
its stream.  ``--impl reference`` times the CPU oracle on a bounded sample of
the same workload.  Under torchrun every rank runs its own independent stream
(weak scaling, no collective on the data path).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {
    "channel": dict(workload="channel-flow-shaped stream, 3 x 192 x 129 x 192 FP32, n=1000, blocks of 8",
                    nx=192, ny=129, nz=192, n=1000, b=8, k=100, s=403, h=50),
    # the same stream with the optional m x l right sketch (l = 2k + 1; not part of the paper)
    "channel_right": dict(workload="channel-flow-shaped stream, 3 x 192 x 129 x 192 FP32, n=1000, blocks of 8, "
                                   "with the m x 201 right sketch", nx=192, ny=129, nz=192, n=1000, b=8, k=100,
                          s=403, h=50, right_l=201),
    "channel_mid": dict(workload="channel-flow-shaped stream, 3 x 96 x 65 x 96 FP32, n=200, blocks of 8",
                        nx=96, ny=65, nz=96, n=200, b=8, k=100, s=403, h=50),
    "channel_small": dict(workload="channel-flow-shaped stream, 3 x 48 x 33 x 48 FP32, n=200, blocks of 8",
                          nx=48, ny=33, nz=48, n=200, b=8, k=20, s=83, h=30),
    # configuration C5: 64 independent streams through rid_batch_ingest (m log-uniform in
    # [2^16, 2^21], n in [100, 1000], k in {10, 30, 60}, h = 30, blocks of 8, BF16x2 sketches)
    "streams64": dict(workload="64 independent streams (half imaging-, half low-rank-shaped), FP32, blocks of 8",
                      kind="streams", nstreams=64, b=8, h=30),
    # gradient mode (Sec. 3.4) on 11 fields of 1024 x 1024: the native-precision FP32 path
    # configuration C4: the small FP64 stream (m = 4096, n = 256, k = 20, s = 83, h = 30, columns one
    # at a time, fixed lambda) in FP32 with BF16x2 / BF16 tensor-core sketches, beside FP32 and FP64
    "precision": dict(workload="precision forms of the 4096 x 256 low-rank stream (k=20, s=83, h=30, "
                               "columns one at a time, fixed lambda), seeds 0..9",
                      kind="precision", m=4096, n=256, k=20, s=83, h=30, seeds=10),
    "ignition": dict(workload="ignition-shaped stream, 11 fields x 1024 x 1024 FP32, gradient mode, n=2000, "
                              "blocks of 8", kind="ignition", N=1024, nfields=11, n=2000, b=8, k=150, s=603, h=50),
}


def ingest_kernel_hash(src_path):
    """SHA-256 of the source the ingest kernel's DRAM counters depend on: tc_ingest.cu from its
    start through the end of tc_ingest_kernel (the helpers it calls come before it) and the
    counter-based generator it includes.  Later code in the file does not change that kernel."""
    text = open(src_path, "rb").read()
    start = text.index(b"tc_ingest_kernel(Dev d,")
    end = text.index(b"\n}\n", start) + 3
    gen = open(os.path.join(os.path.dirname(src_path), "philox.cuh"), "rb").read()
    return hashlib.sha256(text[:end] + gen).hexdigest()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def low_rank_inputs(cfg):
    """The small stream for seeds 0.. with its fixed lambda = ||A - A_k||_F^2 / k (from the SVD)."""
    from workloads import config1_matrix
    out = []
    for seed in range(cfg["seeds"]):
        A = config1_matrix(seed, m=cfg["m"], n=cfg["n"])
        sv = np.linalg.svd(A, compute_uv=False)
        out.append((seed, A, float((sv[cfg["k"]:] ** 2).sum() / cfg["k"])))
    return out


def rel_id_error(A, J, P):
    """||A - A_J P||_F / ||A||_F on the host (P is t x n; empty slots have J < 0)."""
    act = J >= 0
    return float(np.linalg.norm(A - A[:, J[act]] @ P[act]) / np.linalg.norm(A))


def cpu_baseline(cfg, seconds_target=15.0, m_sample=1 << 17):
    """The oracle as it stands on a bounded sample: the first m_sample coordinates of one block of
    b snapshots of the same stream; throughput extrapolated linearly in m (ingest is linear in m)."""
    import torch
    from oracle.rid import OnlineRID as Oracle, RIDConfig
    from workloads import ChannelFlowStream, IgnitionStream
    if cfg.get("kind") == "precision":
        # the whole workload: every seed's stream, one column at a time, in FP64
        errs, dt = [], 0.0
        for seed, A, lam in low_rank_inputs(cfg):
            o = Oracle(RIDConfig(m=cfg["m"], k=cfg["k"], s=cfg["s"], h=cfg["h"], lambda_mode="fixed",
                                 lambda_fixed=lam, seed=seed))
            t0 = time.perf_counter()
            for j in range(cfg["n"]):
                o.ingest(A[:, j:j + 1])
            J, P = o.finalize()
            dt += time.perf_counter() - t0
            errs.append(rel_id_error(A, J, P))
        return {"value": cfg["seeds"] * cfg["n"] / dt, "unit": "snapshots/s", "cores": torch.get_num_threads(),
                "kind": "oracle", "rel_fro_err": errs,
                "sample": f"the whole workload: {cfg['seeds']} streams of {cfg['n']} columns ({dt:.1f} s)"}
    if cfg.get("kind") == "streams":
        # the first 4 of the 64 streams, their first m_sample coordinates, one block of b snapshots
        from workloads import ImagingStream, LowRankStream, batched_streams_spec
        spec = batched_streams_spec(seed=0, nstreams=cfg["nstreams"])[:4]
        dt_full, nsnap = 0.0, 0
        for sp in spec:
            gen = (ImagingStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device="cpu") if sp["kind"] == "imaging"
                   else LowRankStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device="cpu"))
            ms = min(m_sample, sp["m"])
            blk = gen.block(0, cfg["b"]).double().numpy()[:, :ms]
            o = Oracle(RIDConfig(m=ms, k=sp["k"], s=4 * sp["k"] + 3, h=cfg["h"], seed=sp["seed"]))
            t0 = time.perf_counter()
            o.ingest(blk.T)
            dt_full += (time.perf_counter() - t0) * sp["m"] / ms
            nsnap += cfg["b"]
        return {"value": nsnap / dt_full, "unit": "snapshots/s", "cores": torch.get_num_threads(), "kind": "oracle",
                "sample": f"oracle ingest of {cfg['b']} snapshots of each of the first 4 streams, restricted to "
                          f"their first {m_sample} coordinates, extrapolated linearly in m; batch steps not included"}
    if cfg.get("kind") == "ignition":
        # gradient mode: the sample is the first rows of field 0, a 1024-wide grid of its own
        # (s = 603 rows of Omega and Omega_g make the oracle slow: 32 rows keep it to ~30 s)
        m_sample = min(m_sample, 1 << 15)
        from oracle.gradient import grid_gradient_operator
        st = IgnitionStream(seed=0, N=cfg["N"], nfields=cfg["nfields"], n=cfg["n"], device="cpu")
        m = st.m
        rows_s = max(2, min(m_sample, m) // cfg["N"])
        ms = rows_s * cfg["N"]
        blk = st.block(0, cfg["b"]).double().numpy()[:, :ms]
        o = Oracle(RIDConfig(m=ms, k=cfg["k"], s=cfg["s"], h=cfg["h"], seed=0,
                             grad_op=grid_gradient_operator((cfg["N"], rows_s))))
    else:
        st = ChannelFlowStream(seed=0, nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], n=cfg["n"], device="cpu")
        m = st.m
        ms = min(m_sample, m)
        blk = st.block(0, cfg["b"]).double().numpy()[:, :ms]
        o = Oracle(RIDConfig(m=ms, k=cfg["k"], s=cfg["s"], h=cfg["h"], seed=0))
    t0 = time.perf_counter()
    o.ingest(blk.T)
    dt = time.perf_counter() - t0
    cores = torch.get_num_threads()
    per_snap_full = dt / cfg["b"] * (m / ms)
    return {"value": 1.0 / per_snap_full, "unit": "snapshots/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle ingest of {cfg['b']} snapshots restricted to the first {ms} of m={m} coordinates "
                      f"({dt:.1f} s), extrapolated linearly in m; batch steps not included",
            "note": "cores = the BLAS threads of the matrix products; numpy's elementwise work (the Philox "
                    "draws of Omega, most of the time) runs on one core"}


def cpu_baseline_single_thread(config, timeout=300):
    """The oracle's rate on one host core: the reference arm of this script in a child process with
    every thread pool limited to one thread (its own bounded sample of the workload).  A failure is
    reported in the result, never raised."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--config", config, "--steps", "1",
           "--warmup", "0"]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"error": f"exit {r.returncode}: {r.stderr.strip()[-200:]}"}
        ref = json.loads(lines[-1])
        cb = ref.get("cpu_baseline", {})
        return {"value": ref["value"], "unit": ref["unit"], "cores": cb.get("cores"), "sample": cb.get("sample")}
    except Exception as exc:                            # the baseline is a report, not the product
        return {"error": f"{type(exc).__name__}: {exc}"}


def id_error_device(X, J, P, chunk=1 << 17):
    """Relative Frobenius error ||A - A_J P||_F / ||A||_F of a finished stream, for the report only.

    X (n, m) FP32 on the device, row j = snapshot j; J (t,) int64 (-1 = empty slot); P (n, t)
    FP64, row j = coefficients of snapshot j.  Coordinates are taken in chunks and everything
    runs in FP64: coefficients of ill-conditioned bases reach 1e6 and more, and their
    cancellation must not be lost to the evaluation's own rounding."""
    import torch
    act = (J >= 0).nonzero().flatten()
    Jv = J[act]
    Pv = P[:, act]
    num = torch.zeros((), dtype=torch.float64, device=X.device)
    den = torch.zeros((), dtype=torch.float64, device=X.device)
    for c0 in range(0, X.shape[1], chunk):
        Xc = X[:, c0:c0 + chunk].double()
        R = torch.addmm(Xc, Pv, X[Jv, c0:c0 + chunk].double(), alpha=-1.0)
        num += R.square().sum()
        den += Xc.square().sum()
    return float((num / den).sqrt().item()), float(den.item())


def grad_field_error(X, J, P, cfg, chunk=64):
    """||G (A - A_J P)||_F / ||G A||_F for the stacked fields of the ignition stream (central
    differences along x and y inside, one-sided at the boundary), in FP64 on the device."""
    import torch
    N, nf = cfg["N"], cfg["nfields"]
    act = (J >= 0).nonzero().flatten()
    Jv = J[act]
    Pv = P[:, act]
    B = X[Jv].double()                                   # t x m basis
    num = torch.zeros((), dtype=torch.float64, device=X.device)
    den = torch.zeros((), dtype=torch.float64, device=X.device)

    def grad2(F):                                        # F: (c, nf, N, N) -> list of (c, nf, N, N)
        gx = torch.empty_like(F)
        gx[..., 1:-1] = 0.5 * (F[..., 2:] - F[..., :-2])
        gx[..., 0] = F[..., 1] - F[..., 0]
        gx[..., -1] = F[..., -1] - F[..., -2]
        gy = torch.empty_like(F)
        gy[..., 1:-1, :] = 0.5 * (F[..., 2:, :] - F[..., :-2, :])
        gy[..., 0, :] = F[..., 1, :] - F[..., 0, :]
        gy[..., -1, :] = F[..., -1, :] - F[..., -2, :]
        return gx, gy
    for j0 in range(0, X.shape[0], chunk):
        Xc = X[j0:j0 + chunk].double()
        R = Xc - Pv[j0:j0 + chunk] @ B
        for F, acc in ((R, "num"), (Xc, "den")):
            gx, gy = grad2(F.view(-1, nf, N, N))
            v = gx.square().sum() + gy.square().sum()
            if acc == "num":
                num += v
            else:
                den += v
    return float((num / den).sqrt().item())


def accuracy_report(h, X, Jd, Pd):
    """Exact relative error of the result and the NA-Hutch++ estimate of it (Algorithm 8)."""
    err, fro2 = id_error_device(X, Jd, Pd)
    est_sq, est_fro, q = h.error_estimate()
    return {"rel_fro_err": err, "est_rel_fro_err": float(est_fro[0] / np.sqrt(fro2)), "q_star": q}


def residual_css_comparison(rid, X, k, b, st, seed):
    """Algorithm 1 (online CSS by residual-based sampling, Sec. 2.2.1) on the same resident stream,
    as the experiments run it (Sec. 4.1: the subset stops growing at k columns): its throughput,
    blocks of b snapshots through rid_rcss_ingest, and the relative error of projecting the stream
    onto its selected columns (the least-squares coefficients P = A_J^+ A of Sec. 3).  xi is the smallest
    value the algorithm's guarantee allows, ||A - A_k||_F^2, from the eigenvalues of A^T A; the
    Gram matrices of the set-up and the evaluation take FP32 products over chunks of 2^16
    coordinates with FP64 sums (cuBLAS, outside the timed region)."""
    import torch
    n, m = X.shape
    dev = X.device
    G = torch.zeros((n, n), dtype=torch.float64, device=dev)
    for c0 in range(0, m, 1 << 16):
        Xc = X[:, c0:c0 + (1 << 16)]
        G += (Xc @ Xc.T).double()
    ev = torch.linalg.eigvalsh(G.cpu()).flip(0)
    total = float(ev.sum())
    xi = float(ev[k:].sum())
    # one warm-up pass over the first 64 snapshots, on a handle of its own
    g = rid.ResidualCSS(m, k, xi, seed=seed, data_dtype=rid.RID_F32, cap=k, stop_at_cap=True,
                        cuda_stream=st.cuda_stream)
    g.ingest(X[:min(n, 64)])
    g.close()
    torch.cuda.synchronize()
    g = rid.ResidualCSS(m, k, xi, seed=seed, data_dtype=rid.RID_F32, cap=k, stop_at_cap=True,
                        cuda_stream=st.cuda_stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for j0 in range(0, n, b):
        g.ingest(X[j0:j0 + b])
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sel, sigma, nbasis = g.selection()
    p = g.probabilities()
    g.close()
    # ||A - S S^+ A||_F^2 = ||A||_F^2 - tr(B^T Gs^+ B), Gs = S^T S, B = S^T A
    idx = torch.from_numpy(sel).to(dev)
    Gs = torch.zeros((len(sel), len(sel)), dtype=torch.float64, device=dev)
    B = torch.zeros((len(sel), n), dtype=torch.float64, device=dev)
    for c0 in range(0, m, 1 << 16):
        Xc = X[:, c0:c0 + (1 << 16)]
        Sc = Xc[idx]
        Gs += (Sc @ Sc.T).double()
        B += (Sc @ Xc.T).double()
    w, U = torch.linalg.eigh(Gs.cpu())
    keep = w > w.max() * 1e-12
    C = (U[:, keep].T @ B.cpu()) / w[keep].sqrt()[:, None]
    captured = float(C.square().sum())
    err = max(total - captured, 0.0) / total
    return {"value": n / (ms / 1e3), "unit": "snapshots/s", "ms": ms, "k": k, "xi": xi,
            "n_selected": int(len(sel)), "basis_size": int(nbasis), "steps_forced": int((p >= 1).sum()),
            "rel_fro_err": err ** 0.5, "kernel": "rcss_thin_stage_kernel (basis x block dots)",
            "note": "Algorithm 1 with the subset capped at k columns (Sec. 4.1); xi = ||A - A_k||_F^2; "
                    "rel_fro_err = ||A - S S^+ A||_F / ||A||_F, S the selected columns (least-squares "
                    "coefficients); blocks of the bench's size from the resident stream, decisions in "
                    "FP64 on the device"}


def rank_seeds(rank):
    """Seeds of rank r's independent stream (data generator, sketch): every rank has its own."""
    return 1000 + rank, 7 + rank


def max_over_ranks(ms, world, device):
    """The slowest rank's time (all ranks take part; a no-op for one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world, units_per_rank, t_max_ms):
    """Units all ranks processed divided by the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (t_max_ms / 1e3)


def write_timeline(path, tl, names, steps):
    """The per-batch phase records of the timed steps, and per phase the mean duration and the
    mean gap between consecutive batches' starts (the phase's period)."""
    recs = [{"batch": int(b), "phase": names[int(p)], "start_ms": float(a), "end_ms": float(e)}
            for b, p, a, e in tl]
    summ = {}
    for pi, name in enumerate(names):
        rows = tl[tl[:, 1] == pi]
        if len(rows) == 0:
            continue
        dur = rows[:, 3] - rows[:, 2]
        summ[name] = {"count": int(len(rows)), "mean_ms": float(dur.mean()), "max_ms": float(dur.max()),
                      "total_ms_per_step": float(dur.sum() / max(steps, 1))}
    with open(path, "w") as f:
        json.dump({"summary": summ, "records": recs}, f)


def run_streams(args, cfg):
    """Configuration C5: all streams stepped together through rid_batch_ingest (each handle on its
    own CUDA stream), against the same streams run one after another."""
    import torch
    from paper_2405_16076_gb300 import rid
    from workloads import ImagingStream, LowRankStream, batched_streams_spec
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    spec = batched_streams_spec(seed=0, nstreams=cfg["nstreams"])
    data = []
    for sp in spec:
        gen = (ImagingStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device=dev) if sp["kind"] == "imaging"
               else LowRankStream(seed=sp["seed"], m=sp["m"], n=sp["n"], device=dev))
        X = torch.empty((sp["n"], sp["m"]), dtype=torch.float32, device=dev)
        for j0 in range(0, sp["n"], 100):
            gen.block(j0, min(100, sp["n"] - j0), out=X[j0:j0 + 100])
        data.append(X)
    torch.cuda.synchronize()
    b = cfg["b"]
    streams = [torch.cuda.Stream(device=dev) for _ in spec]
    hs = [rid.OnlineRID(m=sp["m"], k=sp["k"], s=4 * sp["k"] + 3, h=cfg["h"], dtype="f32", sketch="bf16x2",
                        n_max=sp["n"], seed=sp["seed"], stream=st, defer=True, group_max=64)
          for sp, st in zip(spec, streams)]
    outs = [(torch.empty(sp["k"], dtype=torch.int64, device=dev),
             torch.empty((sp["n"], sp["k"]), dtype=torch.float64, device=dev)) for sp in spec]
    nmax = max(sp["n"] for sp in spec)
    total = sum(sp["n"] for sp in spec)

    def batched(sync=True):
        for hd in hs:
            hd.reset()
        for j0 in range(0, nmax, b):
            sel = [(hd, X[j0:j0 + b]) for hd, X, sp in zip(hs, data, spec) if j0 < sp["n"]]
            rid.batch_ingest([x[0] for x in sel], [x[1] for x in sel])
        for hd, (J, P) in zip(hs, outs):
            hd.finalize_device(J, P, sync=sync)

    def sequential():
        for hd, X, sp, (J, P) in zip(hs, data, spec, outs):
            hd.reset()
            for j0 in range(0, sp["n"], b):
                hd.ingest(X[j0:j0 + b])
            hd.finalize_device(J, P)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    tb = timed(batched, args.steps)
    ts = timed(sequential, 1)
    # kernels of one batched step, counted by the library (the graph replays the same launches)
    for hd in hs:
        hd.profile(True)
    batched()
    launches = 0
    for hd in hs:
        launches += int(hd.profile_read()[1].sum())
        hd.profile(False)

    # The whole batched run (resets, every stream's ingest and batch steps, the device
    # finalize) captured once into a CUDA graph and replayed: one launch per step from the host
    graph_note = None
    try:
        for hd in hs:
            hd.reset()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        with torch.cuda.graph(graph, stream=cap, capture_error_mode="relaxed"):
            fork = torch.cuda.Event()
            fork.record(cap)
            for st in streams:
                st.wait_event(fork)
            batched(sync=False)
            for st in streams:
                ev = torch.cuda.Event()
                ev.record(st)
                cap.wait_event(ev)
        with torch.cuda.stream(cap):                # replays run on the current stream
            for _ in range(args.warmup):
                graph.replay()
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            with ClockSampler(0) as clk:
                g0.record(cap)
                for _ in range(args.steps):
                    graph.replay()
                g1.record(cap)
                torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) / 1e3 / args.steps
        for hd in hs:
            hd.sync()                               # device errors behind the replays
    except Exception as exc:                        # capture unsupported here: eager timing only
        graph_note = f"graph capture failed ({type(exc).__name__}: {exc}); eager batched timing reported"
        with ClockSampler(0) as clk:
            tb = timed(batched, args.steps)
        tg = None
    errs = [id_error_device(X, J, P, chunk=1 << 20)[0] for X, (J, P) in zip(data, outs)]
    accuracy = {"rel_fro_err_mean": float(np.mean(errs)), "rel_fro_err_max": float(np.max(errs)),
                "rel_fro_err": [float(e) for e in errs],
                "sketch": "bf16x2",
                "note": "||A - A_J P||_F / ||A||_F per stream after the timed region (the batched and the "
                        "one-after-another runs give identical J and P)"}
    pk = peaks()
    algo = sum(8.0 * sp["m"] * sp["n"] for sp in spec)     # read + slot write of every snapshot
    t_head = tg if tg is not None else tb
    line = {
        "metric": "snapshots/s", "value": total / t_head, "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_head * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 data, bf16x2 sketch", "data": "synthetic",
        "config": {"workload": cfg["workload"], "streams": len(spec), "snapshots": total,
                   "m_range": [min(sp["m"] for sp in spec), max(sp["m"] for sp in spec)],
                   "k": sorted({sp["k"] for sp in spec}), "h": cfg["h"], "block": b,
                   "timing": ("CUDA events around graph replays of the whole batched run" if tg is not None
                              else "host clock around whole steps, synchronized on both sides"),
                   "form": "graph-captured" if tg is not None else "eager batched"},
        "eager_batched": {"value": total / tb, "unit": "snapshots/s", "ms_per_step": tb * 1e3,
                          "note": "rid_batch_ingest called from the host, every handle on its own CUDA stream"},
        "sequential": {"value": total / ts, "unit": "snapshots/s", "ms_per_step": ts * 1e3,
                       "note": "the same 64 streams run one after another"},
        "e2e": None,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": algo / t_head / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": algo / t_head / 1e9 / pk.get("hbm_gbs"), "traffic": None, "kernel": "whole step",
                     "note": "algorithmic bytes of every ingest (8 m per snapshot) over the whole batched step"},
        "clocks": clk.summary(),
        "accuracy": accuracy,
    }
    if graph_note:
        line["graph_note"] = graph_note
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, m_sample=1 << 15)
    print(json.dumps(line), flush=True)
    for hd in hs:
        hd.close()


def run_precision(args, cfg):
    """Configuration C4: the same seeded streams through FP64, plain FP32, BF16x2, BF16 and the
    block-scaled E4M3 (FP8x2, FP8) sketches.

    Every form runs every seed (columns one at a time, fixed lambda); the line reports the relative
    Frobenius error of each form's result and of the oracle's (its cpu_baseline leg), and the
    throughput of each form on seed 0 (W warm-up and K timed passes, CUDA events).  The headline
    value is the BF16x2 form."""
    import torch
    from paper_2405_16076_gb300 import rid
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    k, n, m = cfg["k"], cfg["n"], cfg["m"]
    inputs = low_rank_inputs(cfg)
    st = torch.cuda.Stream(device=dev)
    Jd = torch.empty(k, dtype=torch.int64, device=dev)
    Pd = torch.empty((n, k), dtype=torch.float64, device=dev)
    forms = {"f64": ("f64", "native"), "f32": ("f32", "native"), "bf16x2": ("f32", "bf16x2"), "bf16": ("f32", "bf16"),
             "fp8x2": ("f32", "fp8x2"), "fp8": ("f32", "fp8")}
    res, clk_summary, launches = {}, None, 0
    for name, (dtype, sk) in forms.items():
        errs, ests = [], []
        for seed, A, lam in inputs:
            hd = rid.OnlineRID(m=m, k=k, s=cfg["s"], h=cfg["h"], dtype=dtype, sketch=sk, lambda_mode="fixed",
                               lambda_fixed=lam, seed=seed, n_max=n, stream=st, defer=True)
            X = torch.from_numpy(np.ascontiguousarray(A.T, dtype=np.float64 if dtype == "f64" else np.float32)).to(dev)

            def step():
                hd.reset()
                for j in range(n):
                    hd.ingest(X[j:j + 1])
                hd.finalize_device(Jd, Pd)
            step()
            torch.cuda.synchronize()
            if seed == 0:
                for _ in range(args.warmup):
                    step()
                torch.cuda.synchronize()
                hd.profile(True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with ClockSampler(0) as clk:
                    e0.record(st)
                    for _ in range(args.steps):
                        step()
                    e1.record(st)
                    torch.cuda.synchronize()
                prof_ms, prof_kern, prof_grp = hd.profile_read()
                hd.profile(False)
                ms = e0.elapsed_time(e1) / args.steps
                res[name] = {"value": n / (ms / 1e3), "unit": "snapshots/s", "ms_per_step": ms,
                             "ingest_ms_per_launch": prof_ms[0] / max(int(prof_grp[0]), 1)}
                if name == "bf16x2":
                    clk_summary = clk.summary()
                    launches = int(prof_kern.sum())
            J = Jd.cpu().numpy()
            P = Pd.cpu().numpy().T
            errs.append(rel_id_error(A, J, P))
            ests.append(float(hd.error_estimate()[1][0] / np.linalg.norm(A)))
            hd.close()
        res[name].update({"rel_fro_err": errs, "rel_fro_err_mean": float(np.mean(errs)),
                          "est_rel_fro_err_mean": float(np.mean(ests))})
    accuracy = {"forms": res, "err_ratio_bf16x2_vs_f64": res["bf16x2"]["rel_fro_err_mean"] / res["f64"]["rel_fro_err_mean"],
                "err_ratio_bf16_vs_f64": res["bf16"]["rel_fro_err_mean"] / res["f64"]["rel_fro_err_mean"],
                "err_ratio_fp8x2_vs_f64": res["fp8x2"]["rel_fro_err_mean"] / res["f64"]["rel_fro_err_mean"],
                "err_ratio_fp8_vs_f64": res["fp8"]["rel_fro_err_mean"] / res["f64"]["rel_fro_err_mean"],
                "note": "||A - A_J P||_F / ||A||_F per seed (0..9) for each form; est = the NA-Hutch++ estimate"}
    pk = peaks()
    per_launch = res["bf16x2"]["ingest_ms_per_launch"]
    ach = 2.0 * m * 4 / (per_launch / 1e3) / 1e9
    line = {
        "metric": "snapshots/s", "value": res["bf16x2"]["value"], "unit": "snapshots/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["bf16x2"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 data, bf16x2 sketch",
        "data": "synthetic",
        "config": {"workload": cfg["workload"], "m": m, "n": n, "block": 1, "k": k, "s": cfg["s"], "h": cfg["h"],
                   "omega": "rademacher", "lambda": "fixed, ||A - A_k||_F^2 / k",
                   "l2": "small inputs (the stream is 4 MB): latency-bound, L2-resident"},
        "e2e": None,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": ach, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": ach / pk.get("hbm_gbs"), "traffic": None, "kernel": "tc_ingest_kernel",
                     "avg_launch_ms": per_launch, "cols_per_launch": 1,
                     "note": "one 4096-coordinate column per launch: launch- and latency-bound, far from HBM",
                     "peak_source": "measured (MEASURED_PEAKS.json)" if "fallback" not in pk else "fallback"},
        "clocks": clk_summary,
        "accuracy": accuracy,
    }
    if not args.no_cpu_baseline:
        cb = cpu_baseline(cfg)
        line["cpu_baseline"] = {key: v for key, v in cb.items() if key != "rel_fro_err"}
        oe = float(np.mean(cb["rel_fro_err"]))
        accuracy["oracle_f64"] = {"rel_fro_err": cb["rel_fro_err"], "rel_fro_err_mean": oe}
        accuracy["err_ratio_bf16x2_vs_oracle"] = res["bf16x2"]["rel_fro_err_mean"] / oe
    print(json.dumps(line), flush=True)


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(cfg, m_sample=1 << 15)
        if i >= args.warmup:
            steps.append(cb)
    v = float(np.mean([c["value"] for c in steps]))
    line = {"metric": "snapshots/s", "value": v, "unit": "snapshots/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "impl": "reference", "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["workload"]},
            "cpu_baseline": {"kind": "oracle", "cores": steps[0]["cores"], "sample": steps[0]["sample"], "value": v},
            "e2e": {"value": v, "unit": "snapshots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="channel", choices=sorted(CONFIGS))
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sketch", default="bf16x2", choices=["bf16x2", "bf16", "fp8x2", "fp8", "native"])
    ap.add_argument("--group", type=int, default=0,
                    help="columns per sketch launch (1..64); 0 = measure it and the CTAs per launch "
                         "with rid_autotune on the first 8k snapshots before the timed region")
    ap.add_argument("--grad-coeff", action="store_true",
                    help="gradient mode: keep Omega G^p a and report Sec. 3.4's gradient-augmented coefficients")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the accuracy comparison with the other sketch precisions")
    ap.add_argument("--no-rcss", dest="rcss", action="store_false",
                    help="skip the comparison with Algorithm 1 (online CSS by residual-based sampling)")
    ap.add_argument("--timeline", default=None,
                    help="write the per-batch phase timeline of the timed steps (JSON) to this file")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    if cfg.get("kind") == "streams":
        return run_streams(args, cfg)
    if cfg.get("kind") == "precision":
        return run_precision(args, cfg)

    import torch
    import torch.distributed as dist
    from paper_2405_16076_gb300 import rid
    from workloads import ChannelFlowStream, IgnitionStream

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    n, b = cfg["n"], cfg["b"]
    grad = cfg.get("kind") == "ignition"
    if grad:
        gen = IgnitionStream(seed=rank_seeds(rank)[0], N=cfg["N"], nfields=cfg["nfields"], n=n, device=dev)
        if args.grad_coeff:
            args.sketch = "native"                  # the coefficient sketches run on the native path
    else:
        gen = ChannelFlowStream(seed=rank_seeds(rank)[0], nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], n=n, device=dev)
    m = gen.m
    X = torch.empty((n, m), dtype=torch.float32, device=dev)     # row j = snapshot j, resident in HBM
    for j0 in range(0, n, 50):
        gen.block(j0, min(50, n - j0), out=X[j0:j0 + 50])
    torch.cuda.synchronize()

    st = torch.cuda.Stream(device=dev)
    gkw = dict(grad_dims=2, nx=cfg["N"], ny=cfg["N"], nfields=cfg["nfields"]) if grad else {}
    if grad and args.grad_coeff:
        gkw["grad_coeff"] = True
    tune = None
    if args.group == 0:
        # the launch shape measured on this stream's first eight batches, outside the timed region:
        # enough for the batch steps that run beside the ingest in the steady state to weigh in (on
        # two batches the ingest runs almost alone and every SM looks best)
        ntune = min(n, 8 * cfg["k"])
        gbest, cbest, us = rid.autotune_group(X[:ntune], m, cfg["k"], cfg["s"], cfg["h"], dtype="f32",
                                              sketch=args.sketch, seed=rank_seeds(rank)[1], stream=st,
                                              right_l=cfg.get("right_l", 0), **gkw)
        args.group = gbest
        tune = {"group_max": gbest, "ingest_ctas": cbest, "us_per_column": us, "columns": ntune}
    h = rid.OnlineRID(m=m, k=cfg["k"], s=cfg["s"], h=cfg["h"], dtype="f32", sketch=args.sketch, n_max=n,
                      seed=rank_seeds(rank)[1], stream=st, defer=True, group_max=args.group,
                      right_l=cfg.get("right_l", 0), ingest_ctas=tune["ingest_ctas"] if tune else 0, **gkw)
    Jd = torch.empty(cfg["k"], dtype=torch.int64, device=dev)
    Pd = torch.empty((n, cfg["k"]), dtype=torch.float64, device=dev)

    def step():
        h.reset()
        for j0 in range(0, n, b):
            h.ingest(X[j0:j0 + b])
        h.finalize_device(Jd, Pd)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    h.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        barrier()
    ms_total = e0.elapsed_time(e1)
    prof_ms, prof_kern, prof_grp = h.profile_read()
    if args.timeline:
        write_timeline(args.timeline, h.profile_timeline(), h.TIMELINE_PHASES, args.steps)
    h.profile(False)
    accuracy = accuracy_report(h, X, Jd, Pd)
    gradc = None
    if grad and args.grad_coeff:
        # Sec. 3.4's gradient-augmented coefficients for the final basis (lambda by sketched GCV),
        # timed once after the stream; errors of the data and of its gradient field
        Pg = torch.empty((n, cfg["k"]), dtype=torch.float64, device=dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(st)
        lam, _, gval = h.gradient_coefficients(out=Pg)
        c1.record(st)
        torch.cuda.synchronize()
        e_g = id_error_device(X, Jd, Pg)[0]
        gradc = {"lambda": lam, "gcv": gval, "ms": c0.elapsed_time(c1), "rel_fro_err": e_g,
                 "grad_rel_fro_err": grad_field_error(X, Jd, Pg, cfg), "streaming_grad_rel_fro_err":
                 grad_field_error(X, Jd, Pd, cfg),
                 "note": "P(lambda*) of the augmented sketched least squares (Sec. 3.4) after the stream, "
                         "the first call including Omega G^p Omega^T / s; errors of A and of its x/y "
                         "differences, against the streaming P of Algorithms 4-8"}
    t_max = max_over_ranks(ms_total, world, dev)
    value = whole_job_rate(world, n * args.steps, t_max)

    # e2e: same metric through rid_ingest with pinned host buffers and a host read of P
    ring = max(1, min(32, n // b))
    Xh = torch.empty((ring * b, m), dtype=torch.float32, pin_memory=True)
    Xh.copy_(X[: ring * b].cpu())
    J_h = np.empty(cfg["k"], dtype=np.int64)
    P_h = np.empty((n, cfg["k"]))

    def step_e2e():
        h.reset()
        for q, j0 in enumerate(range(0, n, b)):
            r0 = (q % ring) * b
            h.ingest(Xh[r0:r0 + b])
        J, P = h.finalize()
        return P

    e2e_val = None
    if args.e2e_steps > 0:
        step_e2e()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_e2e()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e_val = world * n / e2e_s

    # The ingest kernel alone (no batch step running beside it): one group of G columns per
    # launch, G < t so that no batch step is triggered.  Reported beside the in-step figure.
    G = max(1, min(args.group, cfg["k"] - 1, n))
    if args.sketch == "native":
        G = min(G, 16)                              # one SIMT sketch launch takes up to 16 columns
    h.reset()
    h.ingest(X[:G])
    h.sync()
    h.reset()
    h.profile(True)
    for _ in range(5):
        h.ingest(X[:G])
        h.sync()
        h.reset()
    iso_ms_tot, _, iso_grp = h.profile_read()
    h.profile(False)
    iso_ms = iso_ms_tot[0] / max(int(iso_grp[0]), 1)

    h.close()

    # The optional right sketch: its kernels timed alone, as the difference between ingesting one
    # group of G columns with and without it (CUDA events on the handle's stream, 5 repetitions)
    right = None
    if cfg.get("right_l", 0) > 0:
        rl = cfg["right_l"]

        def group_ms(l):
            hr = rid.OnlineRID(m=m, k=cfg["k"], s=cfg["s"], h=cfg["h"], dtype="f32", sketch=args.sketch, n_max=n,
                               seed=rank_seeds(rank)[1], stream=st, defer=True, group_max=args.group, right_l=l)
            hr.ingest(X[:G])
            hr.sync()
            tot = 0.0
            for _ in range(5):
                hr.reset()
                torch.cuda.synchronize()
                r0 = torch.cuda.Event(enable_timing=True)
                r1 = torch.cuda.Event(enable_timing=True)
                r0.record(st)
                hr.ingest(X[:G])
                hr.sync()
                r1.record(st)
                torch.cuda.synchronize()
                tot += r0.elapsed_time(r1)
            hr.close()
            return tot / 5
        r_ms = group_ms(rl) - group_ms(0)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        pk0 = peaks()
        fma_peak = nsm * 128 * float(pk0.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12     # FP32 TFMA/s
        r_bytes = 2.0 * 4 * m * rl + 4.0 * m * G                                       # Y read + write, A read
        r_fma = float(m) * rl * G
        if args.sketch != "native":
            # tensor-core handles (a +-1 W) take the BF16x2 tcgen05 form: bound by Y's traffic
            right = {"bound": "hbm", "kernel": "tc_right_kernel", "cols_per_launch": G, "l": rl,
                     "avg_launch_ms": r_ms, "achieved": r_bytes / (r_ms / 1e3) / 1e9, "peak": pk0.get("hbm_gbs"),
                     "unit": "GB/s", "frac": r_bytes / (r_ms / 1e3) / 1e9 / pk0.get("hbm_gbs"),
                     "fma": {"achieved": r_fma / (r_ms / 1e3) / 1e12, "unit": "TFMA/s"},
                     "peak_source": "measured (MEASURED_PEAKS.json)",
                     "note": "Y += A_group W over m x l on tensor cores (BF16x2 split of the data, +-1 W): "
                             "2 x 4 m l bytes of Y and 4 m G of data per group; timed alone as the difference "
                             "between one group ingested with and without the right sketch"}
        else:
            right = {"bound": "alu", "kernel": "right_sketch_kernel", "cols_per_launch": G, "l": rl,
                     "avg_launch_ms": r_ms, "achieved": r_fma / (r_ms / 1e3) / 1e12, "peak": fma_peak,
                     "unit": "TFMA/s", "frac": r_fma / (r_ms / 1e3) / 1e12 / fma_peak,
                     "hbm": {"achieved": r_bytes / (r_ms / 1e3) / 1e9, "peak": pk0.get("hbm_gbs"), "unit": "GB/s",
                             "frac": r_bytes / (r_ms / 1e3) / 1e9 / pk0.get("hbm_gbs")},
                     "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x {pk0.get('sm_max_mhz', 2070.0)} MHz "
                                    "(FP32 FMA); HBM: measured (MEASURED_PEAKS.json)",
                     "note": "Y += A_group W over m x l: l FMAs per coordinate and column (FP32 pipe) against "
                             "2 x 4 m l bytes of Y per group; timed alone as the difference between one group "
                             "ingested with and without the right sketch"}

    # The same stream through the other sketch precisions, for the accuracy-throughput comparison
    # (one warm-up and one timed pass each; the plain FP32 form runs on the FP32 pipe)
    forms = {}
    if not grad and args.forms:
        for form in ("bf16x2", "bf16", "fp8x2", "native"):
            if form == args.sketch:
                continue
            hf = rid.OnlineRID(m=m, k=cfg["k"], s=cfg["s"], h=cfg["h"], dtype="f32", sketch=form, n_max=n,
                               seed=rank_seeds(rank)[1], stream=st, defer=True, group_max=args.group)

            def step_f():
                hf.reset()
                for j0 in range(0, n, b):
                    hf.ingest(X[j0:j0 + b])
                hf.finalize_device(Jd, Pd)
            step_f()
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(st)
            step_f()
            f1.record(st)
            torch.cuda.synchronize()
            forms[form] = {"value": n / (f0.elapsed_time(f1) / 1e3), "unit": "snapshots/s",
                           **accuracy_report(hf, X, Jd, Pd)}
            hf.close()
    comparison = None
    if not grad and args.rcss:
        comparison = {"residual_css": residual_css_comparison(rid, X, cfg["k"], b, st, rank_seeds(rank)[1])}
    accuracy["sketch"] = args.sketch
    if forms:
        accuracy["forms"] = forms
        if "native" in forms:
            accuracy["err_ratio_vs_plain_f32"] = accuracy["rel_fro_err"] / forms["native"]["rel_fro_err"]
    accuracy["note"] = ("rel_fro_err = ||A - A_J P||_F / ||A||_F over the whole stream (evaluated in FP64 after the "
                        "timed region); est_rel_fro_err = the NA-Hutch++ estimate of the "
                        "chosen candidate; forms = the same stream with the other sketch precisions "
                        "('native' = plain FP32 on the FP32 pipe)")

    pk = peaks()
    groups = max(int(prof_grp[0]), 1)
    avg_ms = prof_ms[0] / groups
    cols_per_launch = int(prof_kern[0] and (n * args.steps) / max(int(prof_grp[0]), 1))
    if args.sketch == "native":
        cols_per_launch = min(cols_per_launch, 16)  # the timed launch is the group's first (16 columns)
    bytes_per_launch = 2.0 * cols_per_launch * m * 4    # read each column once + write it to its slot
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    # DRAM bytes per launch from the committed ncu counters, scaled by the columns and coordinates
    # of a launch; null unless the counters were taken on this very kernel source
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "ingest_traffic.json")
    src_path = os.path.join(ROOT, "paper_2405_16076_gb300", "csrc", "tc_ingest.cu")
    if args.sketch != "native" and os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            if tr.get("ingest_kernel_sha256") == ingest_kernel_hash(src_path):
                traffic = tr["dram_bytes_per_column_coordinate"] * cols_per_launch * m
        except Exception:
            traffic = None
    line = {
        "metric": "snapshots/s", "value": value, "unit": "snapshots/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x2": "f32 data, bf16x2 sketch", "bf16": "f32 data, bf16 sketch",
                  "fp8x2": "f32 data, block-scaled e4m3x2 sketch", "fp8": "f32 data, block-scaled e4m3 sketch",
                  "native": "f32"}[args.sketch],
        "data": "synthetic",
        "config": {"workload": cfg["workload"], "m": m, "n": n, "block": b, "k": cfg["k"], "s": cfg["s"],
                   "h": cfg["h"], "omega": "rademacher", "lambda": "streaming", "sketch": args.sketch,
                   "group": args.group, "autotune": tune,
                   "l2": f"inputs larger than L2 ({m * 4 / 1e6:.0f} MB per snapshot, whole stream resident in HBM)",
                   "parallelism": f"{world} independent streams"},
        "e2e": {"value": e2e_val, "unit": "snapshots/s", "h2d_bytes_per_step": int(n * m * 4),
                "d2h_bytes_per_step": int(cfg["k"] * n * 8 + cfg["k"] * 8)},
        "gpu_launches": int(prof_kern.sum()),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                     "frac": achieved / pk.get("hbm_gbs"), "traffic": traffic,
                     "kernel": {"native": "ingest_sketch_kernel", "fp8x2": "tc_ingest_fp8_kernel",
                                "fp8": "tc_ingest_fp8_kernel"}.get(args.sketch, "tc_ingest_kernel"),
                     "avg_launch_ms": avg_ms, "cols_per_launch": cols_per_launch,
                     "isolated": {"cols_per_launch": G, "avg_launch_ms": iso_ms,
                                  "achieved": 2.0 * G * m * 4 / (iso_ms / 1e3) / 1e9,
                                  "frac": 2.0 * G * m * 4 / (iso_ms / 1e3) / 1e9 / pk.get("hbm_gbs"),
                                  "note": "same kernel timed alone (no batch step beside it)"},
                     "phase_ms_per_step": {"ingest_sketch": prof_ms[0] / args.steps,
                                           "ingest_reduce": prof_ms[1] / args.steps,
                                           "batch_step": prof_ms[2] / args.steps},
                     "peak_source": "measured (MEASURED_PEAKS.json)" if "fallback" not in pk else "fallback"},
        "clocks": clk.summary(),
        "accuracy": accuracy,
    }
    if gradc is not None:
        line["gradient_coefficients"] = gradc
    if comparison is not None:
        line["comparison"] = comparison
    if right is not None:
        line["ingest_roofline"] = line["roofline"]
        line["roofline"] = right
        line["config"]["right_l"] = cfg["right_l"]
    if grad and args.sketch != "native":
        # Gradient mode on tensor cores: the leverage sketch of [a; G a] needs 2 m (s + h) + 2 (2 m) s
        # multiply-adds per snapshot (the plain sketch, and Omega_g over the 2 m gradient entries),
        # taken in row slices of at most 512 rows per pass; tensor-bound.  Achieved: those
        # algorithmic flops of a group over the group's whole sketch time (every pass, the stencil
        # and the reductions); BF16x2 issues twice these flops (hi and lo rows).
        flop_col = 2.0 * m * (cfg["s"] + cfg["h"]) + 2.0 * (2 * m) * cfg["s"]
        ach = cols_per_launch * flop_col / (avg_ms / 1e3) / 1e12
        iso = G * flop_col / (iso_ms / 1e3) / 1e12
        peak_t = float(pk.get("bf16_tflops", 1900.0))
        line["roofline"].update({"bound": "tensor", "achieved": ach, "peak": peak_t, "unit": "TFLOP/s",
                                 "frac": ach / peak_t, "traffic": None, "kernel": "tc_ingest_kernel (all passes)",
                                 "flop_per_snapshot": flop_col,
                                 "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" if "fallback" not in pk
                                 else "fallback"})
        line["roofline"]["isolated"].update({"achieved": iso, "frac": iso / peak_t})
    if args.sketch == "native":
        # The native-precision sketch runs on the FP32 pipe: one signed add per (row, coordinate,
        # column) of the s + h sketch rows.  Peak: SMs x 128 FP32 lanes x the maximum SM clock.
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_t = nsm * 128 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        rows = cfg["s"] + cfg["h"]
        ach = cols_per_launch * m * rows / (avg_ms / 1e3) / 1e12
        iso = G * m * rows / (iso_ms / 1e3) / 1e12
        line["roofline"].update({"bound": "alu", "achieved": ach, "peak": peak_t, "unit": "Tadd/s",
                                 "frac": ach / peak_t, "traffic": None,
                                 "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x {pk.get('sm_max_mhz', 2070.0)} MHz"})
        line["roofline"]["isolated"].update({"achieved": iso, "frac": iso / peak_t})
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
        line["cpu_baseline"]["single_thread"] = cpu_baseline_single_thread(args.config)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
