// Gradient-augmented coefficients with the sketched GCV choice of lambda (Sec. 3.4).
//
// For the final basis J (na active columns) and the scaled sketches S~ = Omega A / sqrt(s),
// G~^p = Omega G^p A / sqrt(s) (kept during the ingest), K^p = Omega G^p Omega^T / s:
//   P(lam) = M(lam)^{-1} (S~_J^T S~ + lam sum_p G~_J^p^T G~^p),
//   M(lam) = S~_J^T S~_J + lam sum_p G~_J^p^T G~_J^p,
//   GCV(lam) = ||S~ - S~_J X(lam)||_F^2 / (s - tr(M(lam)^{-1} (S~_J^T S~_J + lam Z1)))^2,
//   X(lam) = M(lam)^{-1} (S~_J^T S~ + lam V^T S~),  V = sum_p K^p^T G~_J^p,  Z1 = V^T S~_J,
// which is the paper's C(lam) S~ = S~_J M^{-1} W^T S~ with W = S~_J + lam V and
// tr C = tr(M^{-1} W^T S~_J).  lam* minimises GCV by golden-section search over log10(lam) in
// [lo, hi] (bracket narrower than tol; the midpoint of the last bracket), the same steps as
// the host loop below takes.  The small products are FP64 GEMMs over the s sketch rows; M is
// factored by Cholesky; the residual is formed explicitly, column by column.
// K^p is formed once per handle: Omega's s left rows are materialised (Rademacher entries
// exact in FP32, Gaussian in FP64) and multiplied by their stencil over all m coordinates.
#include <cmath>
#include <vector>

#include "linalg.cuh"
#include "philox.cuh"
#include "rid_internal.cuh"

namespace rid {
namespace {

template <typename T>
__global__ void omega_rows_kernel(Dev d, T* __restrict__ Om) {
  const int64_t total = (int64_t)d.s * d.m_pad;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / d.m_pad);
    const int64_t i = idx - (int64_t)r * d.m_pad;
    double v = 0.0;
    if (i < d.m)
      v = d.omega_kind == 1 ? rademacher_entry(d.seed, kTagRademacher, (uint32_t)r, (uint64_t)i)
                            : gauss_entry(d.seed, kTagGauss, (uint32_t)r, (uint64_t)i);
    Om[idx] = (T)v;
  }
}

// Partial K^p over coordinate slice z of gridDim.z: Kp[z][r + c s] = sum_{i in slice} Om[r][i]
// (G^p Om[c])[i] in 64 x 64 tiles, chunks of 32 coordinates; 256 threads, 4 x 4 outputs each;
// working-precision sums flushed to FP64 every 64 chunks.
template <typename T>
__global__ void __launch_bounds__(256) kgram_kernel(Dev d, const T* __restrict__ Om, int p, double* __restrict__ Kp) {
  __shared__ T As[32][65];
  __shared__ T Bs[32][65];
  const int s = d.s;
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc[u][v] = T(0); acc64[u][v] = 0.0; }
  int pending = 0;
  const int64_t nch = (d.m + 31) / 32;
  const int64_t per = (nch + gridDim.z - 1) / gridDim.z;
  const int64_t ib = (int64_t)blockIdx.z * per * 32;
  const int64_t ie = ib + per * 32 < d.m ? ib + per * 32 : d.m;
  for (int64_t i0 = ib; i0 < ie; i0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
      const int kk = idx & 31, rr = idx >> 5;
      const int64_t i = i0 + kk;
      const int r = r0 + rr, c = c0 + rr;
      As[kk][rr] = (r < s && i < d.m) ? Om[(int64_t)r * d.m_pad + i] : T(0);
      T b = T(0);
      if (c < s && i < d.m) {
        const GradStencil g = grad_stencil((int64_t)p * d.m + i, d.m, d.nx, d.ny);
        const T* row = Om + (int64_t)c * d.m_pad;
        b = (T)g.wc * row[g.i];
        if (g.wm != 0.0) b += (T)g.wm * row[g.i - g.st];
        if (g.wp != 0.0) b += (T)g.wp * row[g.i + g.st];
      }
      Bs[kk][rr] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
    if (++pending == 64) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { acc64[u][v] += (double)acc[u][v]; acc[u][v] = T(0); }
      pending = 0;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (r < s && c < s) Kp[(size_t)blockIdx.z * s * s + r + (size_t)c * s] = acc64[u][v] + (double)acc[u][v];
    }
}

// K^p = (sum of the slices in order) / s.
__global__ void kgram_reduce_kernel(const double* Kp, int nz, int s, int p, double* K) {
  const int64_t ss = (int64_t)s * s;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < ss; idx += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < nz; ++z) v += Kp[z * ss + idx];
    K[p * ss + idx] = v / (double)s;
  }
}

// C (M x N, ldc) = alpha A^T B (+ C when acc), A: K x M (lda), B: K x N (ldb), column-major.
__global__ void __launch_bounds__(256) dgemm_tn_kernel(const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb, double* C,
                                                       int64_t ldc, int M, int64_t N, int K, double alpha, int acc) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int m0 = blockIdx.x * 32;
  const int64_t n0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double sum[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
      const int kk = idx & 31, cc = idx >> 5;
      const int k = k0 + kk;
      As[cc][kk] = (k < K && m0 + cc < M) ? A[k + (int64_t)(m0 + cc) * lda] : 0.0;
      Bs[cc][kk] = (k < K && n0 + cc < N) ? B[k + (n0 + cc) * ldb] : 0.0;
    }
    __syncthreads();
    const int kmax = (K - k0) < 32 ? (K - k0) : 32;
    for (int kk = 0; kk < kmax; ++kk) {
      const double bv = Bs[tx][kk];
#pragma unroll
      for (int u = 0; u < 4; ++u) sum[u] = fma(As[ty + 8 * u][kk], bv, sum[u]);
    }
    __syncthreads();
  }
  const int64_t nb = n0 + tx;
  if (nb >= N) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int mq = m0 + ty + 8 * u;
    if (mq < M) C[mq + nb * ldc] = alpha * sum[u] + (acc ? C[mq + nb * ldc] : 0.0);
  }
}

// Copy selected sketch columns: out[:, a] = scale * src[:, col[a]] (rows of length s, ld lds).
__global__ void gather_cols_kernel(const double* __restrict__ src, int64_t lds, int64_t off, const int64_t* col,
                                   int na, int s, double scale, double* out) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)na * s;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / s), i = (int)(idx % s);
    out[idx] = scale * src[col[a] * lds + off + i];
  }
}

// C = A + lam B (count entries).
__global__ void comb_kernel(const double* A, const double* B, double lam, double* C, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    C[i] = A[i] + lam * B[i];
}

// In-place Cholesky of the n x n SPD matrix (one CTA) and its reciprocal diagonal.
__global__ void __launch_bounds__(1024) gcv_chol_kernel(double* Mx, int n, double* linv) {
  __shared__ int fail;
  __shared__ double gm;
  if (threadIdx.x == 0) {
    fail = 0;
    double m = 0.0;
    for (int a = 0; a < n; ++a) m = fmax(m, Mx[a + (size_t)a * n]);
    gm = m;
  }
  __syncthreads();
  cta_cholesky(Mx, n, n, 1e-13 * gm, &fail);
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const double l = Mx[a + (size_t)a * n];
    linv[a] = (l != 0.0) ? 1.0 / l : 0.0;
  }
}

// X(:, j) <- M^{-1} X(:, j) for ncol columns, one warp per column (L L^T from gcv_chol_kernel).
__global__ void gcv_solve_kernel(const double* L, const double* linv, int n, double* X, int64_t ldx, int64_t ncol) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= ncol) return;
  double* x = X + gw * ldx;
  warp_trsv_lower_r(L, linv, n, n, x);
  warp_trsv_lower_t_r(L, linv, n, n, x);
}

// part[j] = ||scale S(:, j) - SJ X(:, j)||^2 over the s rows, one warp per column.
__global__ void resid_kernel(const double* __restrict__ S, int64_t lds, double scale, const double* __restrict__ SJ,
                             int na, int s, const double* __restrict__ X, int64_t ldx, int64_t n, double* part) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  const double* xj = X + j * ldx;
  double acc = 0.0;
  for (int i = lane; i < s; i += 32) {
    double r = scale * S[j * lds + i];
    for (int a = 0; a < na; ++a) r -= SJ[i + (size_t)a * s] * xj[a];
    acc += r * r;
  }
  acc = warp_sum(acc);
  if (lane == 0) part[j] = acc;
}

// out[0] = GCV = sum_j part[j] / (s - tr T)^2 (fixed summation order), one thread.
__global__ void gcv_value_kernel(const double* part, int64_t n, const double* T, int na, int s, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double num = 0.0;
  for (int64_t j = 0; j < n; ++j) num += part[j];
  double tr = 0.0;
  for (int a = 0; a < na; ++a) tr += T[a + (size_t)a * na];
  const double den = (double)s - tr;
  out[0] = num / (den * den);
}

// P_out rows of the active slots <- X (na x n), other rows 0.
__global__ void scatter_p_kernel(const double* X, int na, const int* slot, int t, int64_t n, double* P, int64_t ldp) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)t * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % t);
    const int64_t j = idx / t;
    P[i + j * ldp] = 0.0;
  }
}
__global__ void scatter_p2_kernel(const double* X, int na, const int* slot, int64_t n, double* P, int64_t ldp) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)na * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % na);
    const int64_t j = idx / na;
    P[slot[a] + j * ldp] = X[a + j * na];
  }
}

void gemm_tn(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int M, int64_t N,
             int K, double alpha, int acc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 g((unsigned)((M + 31) / 32), (unsigned)((N + 31) / 32));
  dgemm_tn_kernel<<<g, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, alpha, acc);
}

}  // namespace

int gradient_coefficients(const Dev& d, cudaStream_t st, int64_t n, const int64_t* jact, const int* slot, int na,
                          double lo, double hi, double tol, double* P_out, int64_t ldp, int on_device,
                          bool* kg_ready, double* lambda_out, double* gcv_out) {
  const int s = d.s, t = d.t;
  const double rs = 1.0 / std::sqrt((double)s);
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes > 0 ? bytes : 8) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  auto release = [&]() { for (void* p : bufs) cudaFree(p); bufs.clear(); };
#define GA(ptr, type, count) type* ptr = (type*)alloc(sizeof(type) * (size_t)(count)); if (!ptr) { release(); return -1; }
  if (!*kg_ready) {
    // K^p = Omega G^p Omega^T / s from the materialised left rows of Omega
    // enough coordinate slices that the tiles fill the GPU a few times over
    const int tiles = ((s + 63) / 64) * ((s + 63) / 64);
    int nz = (4 * d.n_sm + tiles - 1) / tiles;
    const int64_t nch = (d.m + 31) / 32;
    if (nz > nch) nz = (int)nch;
    if (nz < 1) nz = 1;
    const dim3 gk((unsigned)((s + 63) / 64), (unsigned)((s + 63) / 64), (unsigned)nz);
    GA(Kp, double, (size_t)nz * s * s);
    if (d.omega_kind == 1) {                 // +-1 entries: FP32 products and sums are exact
      GA(Om, float, (size_t)s * d.m_pad);
      omega_rows_kernel<float><<<4 * d.n_sm, 256, 0, st>>>(d, Om);
      for (int p = 0; p < 2; ++p) {
        kgram_kernel<float><<<gk, 256, 0, st>>>(d, Om, p, Kp);
        kgram_reduce_kernel<<<2 * d.n_sm, 256, 0, st>>>(Kp, nz, s, p, d.Kg);
      }
    } else {
      GA(Om, double, (size_t)s * d.m_pad);
      omega_rows_kernel<double><<<4 * d.n_sm, 256, 0, st>>>(d, Om);
      for (int p = 0; p < 2; ++p) {
        kgram_kernel<double><<<gk, 256, 0, st>>>(d, Om, p, Kp);
        kgram_reduce_kernel<<<2 * d.n_sm, 256, 0, st>>>(Kp, nz, s, p, d.Kg);
      }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) { release(); return -1; }
    release();
    *kg_ready = true;
  }
  GA(jd, int64_t, na);
  GA(sd, int, na);
  GA(SJ, double, (size_t)s * na);
  GA(GJ, double, (size_t)2 * s * na);
  GA(V, double, (size_t)s * na);
  GA(A0, double, (size_t)na * na);
  GA(B0, double, (size_t)na * na);
  GA(Z1, double, (size_t)na * na);
  GA(Mx, double, (size_t)na * na);
  GA(Tm, double, (size_t)na * na);
  GA(linv, double, na);
  GA(Y0, double, (size_t)na * n);
  GA(Y1, double, (size_t)na * n);
  GA(YG, double, (size_t)na * n);
  GA(X, double, (size_t)na * n);
  GA(part, double, n);
  GA(val, double, 1);
#undef GA
  cudaMemcpyAsync(jd, jact, sizeof(int64_t) * na, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(sd, slot, sizeof(int) * na, cudaMemcpyHostToDevice, st);
  const int gb = 2 * d.n_sm;
  // S~_J, G~_J^p (scaled columns of the kept sketches)
  gather_cols_kernel<<<gb, 256, 0, st>>>(d.S, d.rows, 0, jd, na, s, rs, SJ);
  for (int p = 0; p < 2; ++p) gather_cols_kernel<<<gb, 256, 0, st>>>(d.Sg, 2 * (int64_t)s, (int64_t)p * s, jd, na, s, rs,
                                                                      GJ + (size_t)p * s * na);
  // V = sum_p K^p^T G~_J^p
  for (int p = 0; p < 2; ++p)
    gemm_tn(d.Kg + (size_t)p * s * s, s, GJ + (size_t)p * s * na, s, V, s, s, na, s, 1.0, p, st);
  // small products (S~ and G~^p read in place with their scale)
  gemm_tn(SJ, s, SJ, s, A0, na, na, na, s, 1.0, 0, st);
  gemm_tn(GJ, s, GJ, s, B0, na, na, na, s, 1.0, 0, st);
  gemm_tn(GJ + (size_t)s * na, s, GJ + (size_t)s * na, s, B0, na, na, na, s, 1.0, 1, st);
  gemm_tn(V, s, SJ, s, Z1, na, na, na, s, 1.0, 0, st);
  gemm_tn(SJ, s, d.S, d.rows, Y0, na, na, n, s, rs, 0, st);
  gemm_tn(V, s, d.S, d.rows, Y1, na, na, n, s, rs, 0, st);
  gemm_tn(GJ, s, d.Sg, 2 * (int64_t)s, YG, na, na, n, s, rs, 0, st);
  gemm_tn(GJ + (size_t)s * na, s, d.Sg + s, 2 * (int64_t)s, YG, na, na, n, s, rs, 1, st);
  const int64_t nn = (int64_t)na * na, nx = (int64_t)na * n;
  auto factor = [&](double lam) {
    comb_kernel<<<gb, 256, 0, st>>>(A0, B0, lam, Mx, nn);
    gcv_chol_kernel<<<1, 1024, 0, st>>>(Mx, na, linv);
  };
  auto solve = [&](double* Bm, int64_t ncol) {
    gcv_solve_kernel<<<(unsigned)((ncol * 32 + 255) / 256), 256, 0, st>>>(Mx, linv, na, Bm, na, ncol);
  };
  auto gcv_at = [&](double x) -> double {
    const double lam = std::pow(10.0, x);
    factor(lam);
    comb_kernel<<<gb, 256, 0, st>>>(Y0, Y1, lam, X, nx);
    solve(X, n);
    comb_kernel<<<gb, 256, 0, st>>>(A0, Z1, lam, Tm, nn);
    solve(Tm, na);
    resid_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(d.S, d.rows, rs, SJ, na, s, X, na, n, part);
    gcv_value_kernel<<<1, 32, 0, st>>>(part, n, Tm, na, s, val);
    double h = NAN;
    if (cudaMemcpyAsync(&h, val, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NAN;
    return h;
  };
  // golden-section search over log10(lambda)
  const double inv_phi = (std::sqrt(5.0) - 1.0) / 2.0;
  double a = lo, b = hi;
  double x1 = b - inv_phi * (b - a), x2 = a + inv_phi * (b - a);
  double f1 = gcv_at(x1), f2 = gcv_at(x2);
  while (b - a > tol) {
    if (f1 < f2) {
      b = x2; x2 = x1; f2 = f1;
      x1 = b - inv_phi * (b - a);
      f1 = gcv_at(x1);
    } else {
      a = x1; x1 = x2; f1 = f2;
      x2 = a + inv_phi * (b - a);
      f2 = gcv_at(x2);
    }
  }
  const double xs = 0.5 * (a + b);
  const double g_star = gcv_at(xs);
  const double lam = std::pow(10.0, xs);
  // P(lam*) = M(lam*)^{-1} (Y0 + lam* YG), into the slot rows of P_out
  factor(lam);
  comb_kernel<<<gb, 256, 0, st>>>(Y0, YG, lam, X, nx);
  solve(X, n);
  double* Pd = P_out;
  double* Ptmp = nullptr;
  if (!on_device) {
    Ptmp = (double*)alloc(sizeof(double) * (size_t)ldp * n);
    if (!Ptmp) { release(); return -1; }
    Pd = Ptmp;
  }
  scatter_p_kernel<<<gb, 256, 0, st>>>(X, na, sd, t, n, Pd, ldp);
  scatter_p2_kernel<<<gb, 256, 0, st>>>(X, na, sd, n, Pd, ldp);
  if (!on_device) cudaMemcpyAsync(P_out, Ptmp, sizeof(double) * (size_t)ldp * n, cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  release();
  if (lambda_out) *lambda_out = lam;
  if (gcv_out) *gcv_out = g_star;
  return (e == cudaSuccess && std::isfinite(g_star)) ? 0 : -1;
}

}  // namespace rid
