// Small dense FP64 routines for the batch step, cooperative over one CTA or
// one warp.  Matrices are column-major (shared memory or L1/L2-resident global
// memory at these sizes).  Rank deficiency is handled by skipping non-positive
// (or negligible) pivots, which yields a basic rather than a minimum-norm
// solution.  GB300's FP64 pipe is narrow and its square root and division are
// long instruction sequences: scalar steps run on one thread, and the solves
// take precomputed reciprocal diagonals.
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
// Thread 0 takes the square root and the reciprocal of each pivot.
static __device__ void cta_cholesky(double* A, int n, int lda, double tol, int* fail, double* pmin = nullptr) {
  __shared__ double s_inv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < n; ++j) {
    __syncthreads();
    if (tid == 0) {
      const double djj = A[j + (size_t)j * lda];
      const bool ok = djj > tol;
      if (!ok) *fail = 1;
      if (pmin) *pmin = (j == 0 || djj < *pmin) ? djj : *pmin;
      const double r = ok ? sqrt(djj) : 0.0;
      A[j + (size_t)j * lda] = r;
      s_inv = ok ? 1.0 / r : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
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

// Triangular solves with precomputed reciprocal diagonals (0 where the component is
// dropped), warp cooperative: L y = b, L^T x = y (L lower from cta_cholesky), R x = c (R upper).
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

}  // namespace rid
