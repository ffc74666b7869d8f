"""Synthetic snapshot generators (inputs only; no decomposition arithmetic).

* ``config1_matrix``: A = U diag(sigma) V^T + noise, m=4096, n=256, U from the
  QR of a Gaussian m x 64 matrix, V the thin-QR orthonormalization (diag(R) > 0)
  of the temporally smooth columns cos(pi j t / n), j = 0..63, t = 0..n-1,
  sigma_j = 10^(-j/8), i.i.d. noise of variance 1e-8.
* ``ChannelFlowStream``: three velocity components on an nx x ny x nz grid over
  the 8 pi x 2 x 3 pi channel (Sec. 4.1), x fastest, then z, then y, then
  component.  200 travelling Fourier modes (n_x, n_z) in [-16, 16]^2 \\ {0},
  wavenumber kappa = (2 pi n_x / L_x, 2 pi n_z / L_z), amplitude
  (1 + |kappa|)^(-5/3), per-component N(0,1) weights, phase U[0, 2 pi), phase
  speed U(0.5, 1.5) along x, time step 0.05 per snapshot; the wall-normal
  profile y (2 - y) multiplies every mode; i.i.d. noise of variance 1e-4.
* ``IgnitionStream``: nfields fields on an N x N grid (10 species mass
  fractions and a temperature by default).  Species i is a tanh front of width
  8 cells, 0.5 (1 + tanh((R_i + v_i t - |x - x_i|)/8)), centred at a seeded
  point, radius R_i, speed v_i ~ U(0.2, 1) cells per step; the last field is the
  mean of the species.  Values lie in [0, 1].
* ``ImagingStream``: 64 x 80-pixel frames tiled to length m; log-normal
  intensity exp(0.5 z) of a smooth N(0,1) field z plus 5 advected Gaussian blobs.

The streams build each block of snapshots on the requested torch device.
"""
import math

import numpy as np
import torch


def config1_matrix(seed, m=4096, n=256, r=64, noise_var=1e-8):
    rng = np.random.default_rng(seed)
    U, Ru = np.linalg.qr(rng.standard_normal((m, r)))
    U = U * np.sign(np.diag(Ru))
    tt = np.arange(n)[:, None]
    jj = np.arange(r)[None, :]
    V, Rv = np.linalg.qr(np.cos(np.pi * jj * tt / n))
    V = V * np.sign(np.diag(Rv))
    sigma = 10.0 ** (-np.arange(r) / 8.0)
    A = (U * sigma) @ V.T + math.sqrt(noise_var) * rng.standard_normal((m, n))
    return np.asfortranarray(A)


class ChannelFlowStream:
    """Channel-flow-shaped stream; ``block(j0, b)`` returns an m x b column-major tensor."""

    def __init__(self, seed=0, nx=192, ny=129, nz=192, n=1000, nmodes=200,
                 dtype=torch.float32, device="cpu", noise_var=1e-4, dt=0.05):
        self.seed, self.nx, self.ny, self.nz, self.n = seed, nx, ny, nz, n
        self.m = 3 * nx * ny * nz
        self.dtype, self.device, self.noise_std, self.dt = dtype, torch.device(device), math.sqrt(noise_var), dt
        rng = np.random.default_rng(seed)
        cand = [(a, b) for a in range(-16, 17) for b in range(-16, 17) if (a, b) != (0, 0)]
        pick = rng.choice(len(cand), size=nmodes, replace=False)
        nxz = np.array([cand[i] for i in pick])
        Lx, Lz = 8 * math.pi, 3 * math.pi
        kx = 2 * math.pi * nxz[:, 0] / Lx
        kz = 2 * math.pi * nxz[:, 1] / Lz
        amp = (1.0 + np.hypot(kx, kz)) ** (-5.0 / 3.0)
        w = rng.standard_normal((3, nmodes))
        phi = rng.uniform(0, 2 * math.pi, nmodes)
        c = rng.uniform(0.5, 1.5, nmodes)
        self.ix = nxz[:, 0] + 16
        self.iz = nxz[:, 1] + 16
        self.kx, self.amp, self.w, self.phi, self.c = kx, amp, w, phi, c
        x = np.arange(nx) * Lx / nx
        z = np.arange(nz) * Lz / nz
        y = np.linspace(0.0, 2.0, ny)
        kxs = 2 * math.pi * np.arange(-16, 17) / Lx
        kzs = 2 * math.pi * np.arange(-16, 17) / Lz
        dev = self.device
        self.Ex = torch.tensor(np.exp(1j * np.outer(x, kxs)), dtype=torch.complex128, device=dev)   # nx x 33
        self.Ez = torch.tensor(np.exp(1j * np.outer(z, kzs)), dtype=torch.complex128, device=dev)   # nz x 33
        self.prof = torch.tensor(y * (2.0 - y), dtype=torch.float64, device=dev)

    def _snapshot(self, j, out):
        t = j * self.dt
        psi = self.phi - self.kx * self.c * t
        coef = self.amp * np.exp(1j * psi)
        for comp in range(3):
            C = np.zeros((33, 33), dtype=np.complex128)
            np.add.at(C, (self.ix, self.iz), self.w[comp] * coef)
            Ct = torch.tensor(C, device=self.device)
            F = torch.imag(self.Ex @ Ct @ self.Ez.T)                     # nx x nz, F[x, z]
            field = self.prof[:, None, None] * F.T[None, :, :]            # y, z, x
            blk = out[comp * self.ny * self.nz * self.nx:(comp + 1) * self.ny * self.nz * self.nx]
            blk.copy_(field.reshape(-1).to(self.dtype))
        g = torch.Generator(device=self.device)
        g.manual_seed(int(self.seed) * 1000003 + int(j) + 1)
        out.add_(torch.randn(out.shape, generator=g, device=self.device, dtype=torch.float32)
                 .to(self.dtype) * self.noise_std)

    def block(self, j0, b, out=None):
        if out is None:
            out = torch.empty((b, self.m), dtype=self.dtype, device=self.device)
        for q in range(b):
            self._snapshot(j0 + q, out[q])
        return out        # row q = snapshot j0 + q, i.e. an m x b column-major matrix


class IgnitionStream:
    """Ignition-shaped stream of tanh fronts; ``block(j0, b)`` returns b x m (column-major m x b)."""

    def __init__(self, seed=0, N=1024, nfields=11, n=2000, width=8.0,
                 dtype=torch.float32, device="cpu"):
        self.seed, self.N, self.nfields, self.n, self.width = seed, N, nfields, n, width
        self.m = nfields * N * N
        self.dtype, self.device = dtype, torch.device(device)
        rng = np.random.default_rng(seed)
        ns = nfields - 1
        self.cx = rng.uniform(0.2 * N, 0.8 * N, ns)
        self.cy = rng.uniform(0.2 * N, 0.8 * N, ns)
        self.R0 = rng.uniform(0.02 * N, 0.1 * N, ns)
        self.v = rng.uniform(0.2, 1.0, ns) * (N / 1024.0)
        ax = torch.arange(N, dtype=torch.float64, device=self.device)
        self.X = ax[None, :].expand(N, N)     # x fastest
        self.Y = ax[:, None].expand(N, N)

    def block(self, j0, b, out=None):
        if out is None:
            out = torch.empty((b, self.m), dtype=self.dtype, device=self.device)
        NN = self.N * self.N
        for q in range(b):
            t = float(j0 + q)
            acc = torch.zeros((self.N, self.N), dtype=torch.float64, device=self.device)
            for i in range(self.nfields - 1):
                dist = torch.sqrt((self.X - self.cx[i]) ** 2 + (self.Y - self.cy[i]) ** 2)
                f = 0.5 * (1.0 + torch.tanh((self.R0[i] + self.v[i] * t - dist) / self.width))
                out[q, i * NN:(i + 1) * NN] = f.reshape(-1).to(self.dtype)
                acc += f
            out[q, (self.nfields - 1) * NN:] = (acc / (self.nfields - 1)).reshape(-1).to(self.dtype)
        return out


class ImagingStream:
    """Imaging-shaped stream: 64 x 80 frames tiled to length m (log-normal intensities, advected blobs)."""

    def __init__(self, seed=0, m=65536, n=200, dtype=torch.float32, device="cpu", H=64, W=80):
        self.seed, self.m, self.n, self.H, self.W = seed, m, n, H, W
        self.dtype, self.device = dtype, torch.device(device)
        rng = np.random.default_rng(seed)
        z = rng.standard_normal((H, W))
        # smooth the N(0,1) field with a separable 5-tap binomial filter, renormalize to unit variance
        k = np.array([1, 4, 6, 4, 1], dtype=np.float64) / 16.0
        for ax in (0, 1):
            z = np.apply_along_axis(lambda v: np.convolve(np.pad(v, 2, mode="wrap"), k, "valid"), ax, z)
        z = (z - z.mean()) / z.std()
        self.base = np.exp(0.5 * z)
        self.bx = rng.uniform(0, W, 5)
        self.by = rng.uniform(0, H, 5)
        self.br = rng.uniform(4, 8, 5)
        self.vx = rng.uniform(-1, 1, 5)
        self.vy = rng.uniform(-1, 1, 5)
        self.ba = rng.uniform(0.5, 2.0, 5)

    def frame(self, j):
        yy, xx = np.mgrid[0:self.H, 0:self.W]
        f = self.base.copy()
        for i in range(5):
            cx = (self.bx[i] + self.vx[i] * j) % self.W
            cy = (self.by[i] + self.vy[i] * j) % self.H
            f += self.ba[i] * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * self.br[i] ** 2))
        return f

    def block(self, j0, b, out=None):
        if out is None:
            out = torch.empty((b, self.m), dtype=self.dtype, device=self.device)
        fs = self.H * self.W
        reps = -(-self.m // fs)
        for q in range(b):
            f = np.tile(self.frame(j0 + q).reshape(-1), reps)[: self.m]
            out[q] = torch.tensor(f, dtype=self.dtype, device=self.device)
        return out


class LowRankStream:
    """Configuration-1-style stream with m rows: U diag(sigma) V^T + noise, built on ``device``.

    U: m x r Gaussian columns scaled to unit norm; sigma_j = 10^(-j/8); V(t, j) = cos(pi j t / n);
    noise variance 1e-8.  ``block(j0, b)`` returns b x m (row q = snapshot j0 + q)."""

    def __init__(self, seed=0, m=65536, n=200, r=64, dtype=torch.float32, device="cpu"):
        self.m, self.n, self.r = m, n, r
        self.dtype, self.device = dtype, torch.device(device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        U = torch.randn(m, r, generator=g, dtype=torch.float32)
        self.U = (U / U.norm(dim=0, keepdim=True)).to(self.device)
        self.sigma = (10.0 ** (-torch.arange(r, dtype=torch.float32) / 8.0)).to(self.device)
        self.g = torch.Generator(device=self.device).manual_seed(seed + 1)

    def block(self, j0, b, out=None):
        t = torch.arange(j0, j0 + b, dtype=torch.float32)[:, None]
        V = torch.cos(math.pi * t * torch.arange(self.r, dtype=torch.float32)[None, :] / self.n).to(self.device)
        X = (V * self.sigma[None, :]) @ self.U.T
        X += 1e-4 * torch.randn(b, self.m, generator=self.g, dtype=torch.float32, device=self.device)
        if out is None:
            return X.to(self.dtype)
        out.copy_(X)
        return out


def batched_streams_spec(seed=0, nstreams=64):
    """Per-stream (kind, m, n, k) for the batched form: m log-uniform in [2^16, 2^21],
    n uniform in [100, 1000], k in {10, 30, 60}, half imaging- and half flow-shaped."""
    rng = np.random.default_rng(seed)
    spec = []
    for i in range(nstreams):
        m = int(round(2.0 ** rng.uniform(16, 21)))
        n = int(rng.integers(100, 1001))
        k = int(rng.choice([10, 30, 60]))
        kind = "imaging" if i % 2 == 0 else "flow"
        spec.append(dict(kind=kind, m=m, n=n, k=k, seed=seed * 1000 + i))
    return spec
