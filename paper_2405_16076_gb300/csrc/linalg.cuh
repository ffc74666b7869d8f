// Small dense FP64 routines for the batch step, cooperative over one CTA or
// one warp.  Matrices are column-major in global memory (L1/L2 resident at
// these sizes).  Rank deficiency is handled by skipping non-positive (or
// negligible) pivots, which yields a basic rather than a minimum-norm
// solution.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rid {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block-wide sum; sh must hold 33 doubles; all threads get the result.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double x = (lane < nw) ? sh[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) sh[32] = x;
  }
  __syncthreads();
  return sh[32];
}

// In-place lower Cholesky of the n x n SPD matrix A (lower triangle used).
// A non-positive pivot (relative to tol) zeroes its column; returns via *fail.
// pmin (shared, may be null) receives the smallest pivot, before its square root.
static __device__ void cta_cholesky(double* A, int n, int lda, double tol, int* fail, double* pmin = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    double djj = A[j + (size_t)j * lda];
    const bool ok = djj > tol;
    if (!ok && tid == 0) *fail = 1;
    if (pmin && tid == 0) *pmin = (j == 0 || djj < *pmin) ? djj : *pmin;
    djj = ok ? sqrt(djj) : 0.0;
    __syncthreads();
    if (tid == 0) A[j + (size_t)j * lda] = djj;
    const double inv = ok ? 1.0 / djj : 0.0;
    for (int i = j + 1 + tid; i < n; i += nt) A[i + (size_t)j * lda] *= inv;
    __syncthreads();
    // trailing lower triangle, one warp per column
    const int lane = tid & 31, nw = nt >> 5;
    for (int l = j + 1 + (tid >> 5); l < n; l += nw) {
      const double alj = A[l + (size_t)j * lda];
      for (int i = l + lane; i < n; i += 32) A[i + (size_t)l * lda] -= A[i + (size_t)j * lda] * alj;
    }
  }
  __syncthreads();
}

// Solve L y = b in place (L lower from cta_cholesky); warp cooperative.
static __device__ void warp_trsv_lower(const double* L, int n, int lda, double* b) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const double ljj = L[j + (size_t)j * lda];
    const double yj = (ljj != 0.0) ? b[j] / ljj : 0.0;
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) b[i] -= L[i + (size_t)j * lda] * yj;
    if (lane == 0) b[j] = yj;
    __syncwarp();
  }
}

// Solve L^T x = y in place; warp cooperative.
static __device__ void warp_trsv_lower_t(const double* L, int n, int lda, double* b) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    const double ljj = L[j + (size_t)j * lda];
    const double xj = (ljj != 0.0) ? b[j] / ljj : 0.0;
    __syncwarp();
    for (int i = lane; i < j; i += 32) b[i] -= L[j + (size_t)i * lda] * xj;
    if (lane == 0) b[j] = xj;
    __syncwarp();
  }
}

// Householder QR of the m x n matrix A (m >= n) in place.  R is the upper
// triangle of A; reflector j is v = [vhead[j]; A(j+1:m, j)], H_j = I - beta[j] v v^T.
static __device__ void cta_householder_qr(double* A, int m, int n, int lda, double* beta, double* vhead,
                                   double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int j = 0; j < n; ++j) {
    double* col = A + (size_t)j * lda;
    double part = 0.0;
    for (int i = j + tid; i < m; i += nt) part += col[i] * col[i];
    const double nrm2 = block_sum(part, sh);
    const double x0 = col[j];
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    const double b = (nrm2 > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
    __syncthreads();
    if (tid == 0) { col[j] = (b > 0.0) ? alpha : x0; vhead[j] = v0; beta[j] = b; }
    if (b > 0.0) {
      for (int l = j + 1 + wid; l < n; l += nw) {
        double* a = A + (size_t)l * lda;
        double dot = (lane == 0) ? v0 * a[j] : 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) dot += col[i] * a[i];
        dot = warp_sum(dot);
        const double f = b * dot;
        if (lane == 0) a[j] -= f * v0;
        for (int i = j + 1 + lane; i < m; i += 32) a[i] -= f * col[i];
      }
    }
    __syncthreads();
  }
}

// b <- Q^T b for the reflectors of cta_householder_qr; warp cooperative.
static __device__ void warp_apply_qt(const double* QR, int m, int n, int lda, const double* beta,
                              const double* vhead, double* b) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const double bj = beta[j];
    if (bj == 0.0) continue;
    const double* v = QR + (size_t)j * lda;
    const double vh = vhead[j];
    double dot = (lane == 0) ? vh * b[j] : 0.0;
    for (int i = j + 1 + lane; i < m; i += 32) dot += v[i] * b[i];
    dot = warp_sum(dot);
    const double f = bj * dot;
    __syncwarp();
    if (lane == 0) b[j] -= f * vh;
    for (int i = j + 1 + lane; i < m; i += 32) b[i] -= f * v[i];
    __syncwarp();
  }
}

// Solve R x = c in place (R = upper triangle of QR, n x n); |r_jj| <= tol gives x_j = 0.
static __device__ void warp_trsv_upper(const double* R, int n, int lda, double* c, double tol) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    const double rjj = R[j + (size_t)j * lda];
    const double xj = (fabs(rjj) > tol) ? c[j] / rjj : 0.0;
    __syncwarp();
    for (int i = lane; i < j; i += 32) c[i] -= R[i + (size_t)j * lda] * xj;
    if (lane == 0) c[j] = xj;
    __syncwarp();
  }
}

// Solve R x = c in place with R's diagonal held apart in rdiag (the QR of qr_coop).
static __device__ void warp_trsv_upper_d(const double* R, const double* rdiag, int n, int lda, double* c,
                                         double tol) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    const double rjj = rdiag[j];
    const double xj = (fabs(rjj) > tol) ? c[j] / rjj : 0.0;
    __syncwarp();
    for (int i = lane; i < j; i += 32) c[i] -= R[i + (size_t)j * lda] * xj;
    if (lane == 0) c[j] = xj;
    __syncwarp();
  }
}

// The same three triangular solves with precomputed reciprocal diagonals (0 where the
// division is skipped): this GPU's FP64 division is a long multi-instruction sequence.
static __device__ void warp_trsv_lower_r(const double* L, const double* linv, int n, int lda, double* b) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    const double yj = b[j] * linv[j];
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) b[i] -= L[i + (size_t)j * lda] * yj;
    if (lane == 0) b[j] = yj;
    __syncwarp();
  }
}
static __device__ void warp_trsv_lower_t_r(const double* L, const double* linv, int n, int lda, double* b) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    const double xj = b[j] * linv[j];
    __syncwarp();
    for (int i = lane; i < j; i += 32) b[i] -= L[j + (size_t)i * lda] * xj;
    if (lane == 0) b[j] = xj;
    __syncwarp();
  }
}
static __device__ void warp_trsv_upper_r(const double* R, const double* rinv, int n, int lda, double* c) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    const double xj = c[j] * rinv[j];
    __syncwarp();
    for (int i = lane; i < j; i += 32) c[i] -= R[i + (size_t)j * lda] * xj;
    if (lane == 0) c[j] = xj;
    __syncwarp();
  }
}

// Householder tridiagonalization of the symmetric n x n matrix A (full
// storage, destroyed); diagonal to dvec, off-diagonal to evec.  v, p: n doubles each.
static __device__ void cta_tridiagonalize(double* A, int n, int lda, double* dvec, double* evec,
                                   double* v, double* p, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k + 2 < n; ++k) {
    const int nn = n - k - 1;
    double* Ab = A + (k + 1) + (size_t)(k + 1) * lda;   // trailing block
    const double* x = A + (k + 1) + (size_t)k * lda;
    double part = 0.0;
    for (int i = tid; i < nn; i += nt) { const double xi = x[i]; v[i] = xi; part += xi * xi; }
    const double nrm2 = block_sum(part, sh);
    const double x0 = v[0];
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    const double beta = (nrm2 - x0 * x0 > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
    __syncthreads();
    if (tid == 0) {
      v[0] = v0;
      dvec[k] = A[k + (size_t)k * lda];
      evec[k] = (beta > 0.0) ? alpha : x0;
    }
    __syncthreads();
    if (beta == 0.0) continue;
    for (int i = tid; i < nn; i += nt) {
      double acc = 0.0;
      for (int j = 0; j < nn; ++j) acc += Ab[i + (size_t)j * lda] * v[j];
      p[i] = beta * acc;
    }
    __syncthreads();
    part = 0.0;
    for (int i = tid; i < nn; i += nt) part += p[i] * v[i];
    const double ptv = block_sum(part, sh);
    const double kc = 0.5 * beta * ptv;
    for (int i = tid; i < nn; i += nt) p[i] -= kc * v[i];
    __syncthreads();
    for (long long q = tid; q < (long long)nn * nn; q += nt) {
      const int i = (int)(q % nn), j = (int)(q / nn);
      Ab[i + (size_t)j * lda] -= v[i] * p[j] + p[i] * v[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dvec[n - 2] = A[(n - 2) + (size_t)(n - 2) * lda];
      evec[n - 2] = A[(n - 1) + (size_t)(n - 2) * lda];
    }
    dvec[n - 1] = A[(n - 1) + (size_t)(n - 1) * lda];
  }
  __syncthreads();
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) smaller than x (Sturm count).
static __device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// j-th smallest eigenvalue (0-based) of the tridiagonal (d, e) by bisection.
static __device__ double tridiag_eig_bisect(const double* d, const double* e, int n, int j) {
  double lo = d[0], hi = d[0], emax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = ((i > 0) ? fabs(e[i - 1]) : 0.0) + ((i + 1 < n) ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < n) emax = fmax(emax, fabs(e[i]));
  }
  const double scale = fmax(fabs(lo), fabs(hi));
  const double pivmin = fmax(2.2250738585072014e-308, 2.2250738585072014e-308 * emax * emax) + 1e-300;
  lo -= 2.220446049250313e-16 * scale + pivmin;
  hi += 2.220446049250313e-16 * scale + pivmin;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(d, e, n, mid, pivmin) > j) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace rid
