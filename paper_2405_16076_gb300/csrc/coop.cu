// Multi-SM FP64 kernels for the sketch Gram M = S_lev S_lev^T / s of the batch step.
//
// GB300's FP64 rate is ~2 FMA/clk per SM, so the O(s^3) reduction is spread
// over every SM with a grid barrier between the dependent phases:
//   * tridiag_coop_kernel: Householder reduction M = Q T Q^T (T tridiagonal),
//     reflectors kept in place for later use;
//   * topk_eig_kernel: the k largest eigenvalues of T by 32-way multisection of
//     Sturm counts (one warp per eigenvalue), then
//     lambda = (||A_obs||^2 - sum of the k largest) / k  (Eq. 23, floored);
//   * tri_scores_kernel: sketched ridge scores (Eq. 23)
//     tau = v^T (M + lambda I)^{-1} v = y^T (T + lambda I)^{-1} y with y = Q^T v,
//     using the stored reflectors and one LDL^T of the SPD tridiagonal T + lambda I.
// The grid barrier is a counter/generation pair with a bounded spin; on timeout
// the kernel raises ERR_TIMEOUT and every block stops at its next barrier.
#include <cuda_runtime.h>
#include <stdlib.h>

#include <array>
#include <stdint.h>

#include <cooperative_groups.h>

#include "linalg.cuh"
#include "rid_internal.cuh"

namespace rid {

namespace {

constexpr int kCoopThreads = 256;
constexpr int kTriThreads = 512;
constexpr int kRedWarps = 4;             // warps that take part in the vector reductions
namespace cg = cooperative_groups;
constexpr uint32_t kBarrierSpin = 1u << 24;

struct GridBar {
  unsigned int* count;   // monotonic ticket counter: barrier i completes at (i + 1) * gridDim.x
  unsigned int* unused;
  int* err;
  int* stop;             // set when any barrier timed out
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns false if the barrier timed out (or another block's did).
__device__ bool grid_barrier(const GridBar& b) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();                                   // release this block's writes
    const unsigned int ticket = atomicAdd(b.count, 1u);
    const unsigned int target = (ticket / gridDim.x + 1u) * gridDim.x;
    uint32_t it = 0;
    while ((int)(ld_acquire(b.count) - target) < 0) {
      if (++it > kBarrierSpin) { ok = 0; break; }
      if ((it & 1023u) == 0u && *(volatile int*)b.stop) { ok = 0; break; }
      if (it > 4096) __nanosleep(32);
    }
    if (!ok) {
      atomicExch(b.stop, 1);
      atomicOr(b.err, ERR_TIMEOUT);
    }
    __threadfence();
    ok_s = ok && !*(volatile int*)b.stop;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace

// Householder reduction M = Q T Q^T on every SM with one grid barrier per step.
// Block b owns the trailing columns j with j % gridDim.x == b.  At step k every
// block holds the (updated) column k locally, forms reflector k from it, computes
// p = beta A' v on its own columns, and after the barrier forms w, updates its
// own columns except column k+1, and recomputes the updated column k+1 -- the
// next reflector column -- itself from A, v and w.  Column k+1 is therefore never
// written back, and p is double-buffered by step parity.
// On exit: d[0..n), e[0..n-1), reflector k = [vhead[k]; R(k+2:n, k)] acting on
// rows k+1..n-1 with coefficient beta[k].
__global__ void __launch_bounds__(kCoopThreads)
tridiag_coop_kernel(Dev d, double* A, double* R, double* dvec, double* evec, double* beta,
                    double* vhead, double* pbuf, GridBar bar) {
  extern __shared__ double sm[];
  const int n = d.s;
  double* v = sm;            // reflector of the current step, trailing-relative index
  double* w = sm + n;
  double* x = sm + 2 * n;    // current column below the diagonal, trailing-relative index
  __shared__ double sh[33];
  __shared__ double diag_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const double inv_s = 1.0 / (double)n;
  for (int64_t i = (int64_t)b * blockDim.x + tid; i < (int64_t)n * n; i += (int64_t)G * blockDim.x)
    A[i] = d.SSt[i] * inv_s;
  if (!grid_barrier(bar)) return;
  for (int i = tid; i + 1 < n; i += blockDim.x) x[i] = A[(i + 1)];
  if (tid == 0) diag_s = A[0];
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int nn = n - k - 1;                   // trailing rows/columns k+1 .. n-1
    double part = 0.0;
    for (int i = tid; i < nn; i += blockDim.x) part += x[i] * x[i];
    const double nrm2 = block_sum(part, sh);
    const double x0 = x[0];
    const double tail = nrm2 - x0 * x0;
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = tail + v0 * v0;
    const double bt = (tail > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
    for (int i = tid; i < nn; i += blockDim.x) v[i] = (i == 0) ? v0 : x[i];
    if (b == 0) {
      if (tid == 0) {
        dvec[k] = diag_s;
        evec[k] = (bt > 0.0) ? alpha : x0;
        beta[k] = bt;
        vhead[k] = v0;
      }
      for (int i = 1 + tid; i < nn; i += blockDim.x) R[(k + 1 + i) + (size_t)k * n] = x[i];
    }
    __syncthreads();
    // p_j = beta * (A' v)_j on the owned trailing columns (A' symmetric: row j read as column j)
    double* pk = pbuf + (size_t)(k & 1) * n;
    const int j0 = ((b - (k + 1)) % G + G) % G;   // first owned trailing column
    for (int jl = j0 + wid * G; jl < nn; jl += nw * G) {
      const double* col = A + (k + 1) + (size_t)(k + 1 + jl) * n;
      double acc = 0.0;
      for (int i = lane; i < nn; i += 32) acc += col[i] * v[i];
      acc = warp_sum(acc);
      if (lane == 0) pk[jl] = bt * acc;
    }
    if (!grid_barrier(bar)) return;
    part = 0.0;
    for (int i = tid; i < nn; i += blockDim.x) { const double pi = pk[i]; w[i] = pi; part += pi * v[i]; }
    const double ptv = block_sum(part, sh);
    const double kc = 0.5 * bt * ptv;
    for (int i = tid; i < nn; i += blockDim.x) w[i] -= kc * v[i];
    __syncthreads();
    // owned columns except the next one: A' -= v w^T + w v^T
    for (int jl = j0 + wid * G; jl < nn; jl += nw * G) {
      if (jl == 0) continue;
      double* col = A + (k + 1) + (size_t)(k + 1 + jl) * n;
      const double wj = w[jl], vj = v[jl];
      for (int i = lane; i < nn; i += 32) col[i] -= v[i] * wj + w[i] * vj;
    }
    // the updated next column (trailing column 0), recomputed by every block
    const double* c0 = A + (k + 1) + (size_t)(k + 1) * n;
    for (int i = 1 + tid; i < nn; i += blockDim.x) x[i - 1] = c0[i] - v[i] * w[0] - w[i] * v[0];
    if (tid == 0) diag_s = c0[0] - 2.0 * v[0] * w[0];
    __syncthreads();
  }
  if (!grid_barrier(bar)) return;
  if (b == 0 && tid == 0) {
    if (n >= 2) {
      dvec[n - 2] = diag_s;
      evec[n - 2] = x[0];
      beta[n - 2] = 0.0;
      dvec[n - 1] = A[(n - 1) + (size_t)(n - 1) * n];
    } else {
      dvec[0] = A[0];
    }
  }
}

// The same reduction M = Q T Q^T with the same outputs, on one thread-block cluster: the
// trailing columns live in the shared memory of the cluster's CTAs (CTA r owns the columns
// j with j % C == r), and one cluster barrier per step replaces the grid barrier.  At step
// k every CTA holds column k below the diagonal, forms the reflector, computes p on its
// own columns and stores each p_j into every CTA's p buffer (distributed shared memory,
// double-buffered by step parity); after the barrier it forms w, reads the next column
// k+1 from its owner, updates its own columns except column k+1 (never written again, so
// the owner's copy is stable while others read it), and forms the updated column k+1.
// Control flow is uniform over the cluster, so every CTA meets every barrier.
__global__ void __launch_bounds__(kTriThreads, 1)
tridiag_cluster_kernel(Dev d, double* R, double* dvec, double* evec, double* beta, double* vhead, int ncl) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int n = d.s;
  extern __shared__ double tsm2[];
  double* cols = tsm2;                     // ncl x n: local column lc is global column lc * C + rank
  double* x = cols + (size_t)ncl * n;      // column k below the diagonal (trailing-relative)
  double* y = x + n;                       // column k+1 rows k+1.. as read from its owner
  double* v = y + n;
  double* w = v + n;
  double* pb = w + n;                      // 2 x n, p of the step, by step parity
  __shared__ double sh[33];
  __shared__ double diag_s;
  __shared__ double scal[4];               // beta, v0 of the step; kc
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const double inv_s = 1.0 / (double)n;
  for (int lc = wid; lc * C + rank < n; lc += nw) {
    const double* src = d.SSt + (size_t)(lc * C + rank) * n;
    for (int i = lane; i < n; i += 32) cols[(size_t)lc * n + i] = src[i] * inv_s;
  }
  for (int i = tid; i + 1 < n; i += blockDim.x) x[i] = d.SSt[i + 1] * inv_s;
  if (tid == 0) diag_s = d.SSt[0] * inv_s;
  cl.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int nn = n - k - 1;
    // GB300's FP64 pipe is narrow: reductions run on kRedWarps warps and the scalar
    // arithmetic (square root, division) on one thread
    if (wid < kRedWarps) {
      double part = 0.0;
      for (int i = tid; i < nn; i += 32 * kRedWarps) part += x[i] * x[i];
      part = warp_sum(part);
      if (lane == 0) sh[wid] = part;
    }
    __syncthreads();
    if (tid == 0) {
      double nrm2 = 0.0;
      for (int i = 0; i < kRedWarps; ++i) nrm2 += sh[i];
      const double x0 = x[0];
      const double tail = nrm2 - x0 * x0;
      const double nrm = sqrt(nrm2);
      const double alpha = (x0 >= 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = tail + v0 * v0;
      const double bt = (tail > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
      scal[0] = bt;
      scal[1] = v0;
      if (rank == 0) {
        dvec[k] = diag_s;
        evec[k] = (bt > 0.0) ? alpha : x0;
        beta[k] = bt;
        vhead[k] = v0;
      }
    }
    __syncthreads();
    const double bt = scal[0];
    for (int i = tid; i < nn; i += blockDim.x) v[i] = (i == 0) ? scal[1] : x[i];
    if (rank == 0)
      for (int i = 1 + tid; i < nn; i += blockDim.x) R[(k + 1 + i) + (size_t)k * n] = x[i];
    __syncthreads();
    // p_j = beta (A' v)_j on the owned trailing columns, stored into every CTA's buffer
    const int par = k & 1;
    const int lc0 = (k + 1 - rank + C - 1) / C;   // first owned column >= k+1
    for (int lc = lc0 + wid; lc * C + rank < n; lc += nw) {
      const int jl = lc * C + rank - (k + 1);
      const double* col = cols + (size_t)lc * n + (k + 1);
      double acc = 0.0;
      for (int i = lane; i < nn; i += 32) acc += col[i] * v[i];
      acc = warp_sum(acc);
      if (lane < C) {
        double* rp = cl.map_shared_rank(pb, lane);
        rp[(size_t)par * n + jl] = bt * acc;
      }
    }
    cl.sync();
    const double* pk = pb + (size_t)par * n;
    if (wid < kRedWarps) {
      double part = 0.0;
      for (int i = tid; i < nn; i += 32 * kRedWarps) part += pk[i] * v[i];
      part = warp_sum(part);
      if (lane == 0) sh[wid] = part;
    }
    __syncthreads();
    if (tid == 0) {
      double ptv = 0.0;
      for (int i = 0; i < kRedWarps; ++i) ptv += sh[i];
      scal[2] = 0.5 * bt * ptv;
    }
    __syncthreads();
    const double kc = scal[2];
    for (int i = tid; i < nn; i += blockDim.x) w[i] = pk[i] - kc * v[i];
    // column k+1 (rows k+1 ..) from its owner; it is not modified at this step
    {
      const int o = (k + 1) % C, lco = (k + 1) / C;
      const double* yc = cl.map_shared_rank(cols, o) + (size_t)lco * n + (k + 1);
      for (int i = tid; i < nn; i += blockDim.x) y[i] = yc[i];
    }
    __syncthreads();
    // owned columns except the next one: A' -= v w^T + w v^T
    for (int lc = lc0 + wid; lc * C + rank < n; lc += nw) {
      const int jl = lc * C + rank - (k + 1);
      if (jl == 0) continue;
      double* col = cols + (size_t)lc * n + (k + 1);
      const double wj = w[jl], vj = v[jl];
      for (int i = lane; i < nn; i += 32) col[i] -= v[i] * wj + w[i] * vj;
    }
    // the updated next column (trailing column 0)
    for (int i = 1 + tid; i < nn; i += blockDim.x) x[i - 1] = y[i] - v[i] * w[0] - w[i] * v[0];
    if (tid == 0) diag_s = y[0] - 2.0 * v[0] * w[0];
    __syncthreads();
  }
  cl.sync();
  if (rank == 0 && tid == 0) {
    if (n >= 2) {
      dvec[n - 2] = diag_s;
      evec[n - 2] = x[0];
      beta[n - 2] = 0.0;
      const double* last = cl.map_shared_rank(cols, (n - 1) % C) + (size_t)((n - 1) / C) * n;
      dvec[n - 1] = last[n - 1];
    } else {
      dvec[0] = diag_s;
    }
  }
  cl.sync();                               // no CTA leaves while its shared memory may be read
}

// Number of eigenvalues of the tridiagonal T below x, from the signs of the
// leading principal minors p_i = det(T_i - x I): p_0 = 1, p_1 = d_0 - x,
// p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1}; the count is the number of sign
// changes along p_0 .. p_n (Sturm's theorem).  Division-free (GB300's FP64 pipe
// is the bottleneck, and a divide costs several FMA-equivalents).  T is scaled
// so that ||T|| <= 1 (ds = d / sc, e2s = (e / sc)^2); every 4 steps both carried
// minors are multiplied by the same power of two (exact), which keeps them in
// range.  An exactly zero minor takes the sign opposite to its predecessor,
// like a zero pivot -pivmin in the LDL^T form of the count.
__device__ __forceinline__ int sign_flip(double a, double b) {
  return (int)(((uint32_t)__double2hiint(a) ^ (uint32_t)__double2hiint(b)) >> 31);
}
__device__ __forceinline__ bool is_zero(double a) {
  return ((__double2hiint(a) & 0x7FFFFFFF) | __double2loint(a)) == 0;
}
__device__ __forceinline__ void rescale_pair(double& p, double& pm) {
  const int ea = (__double2hiint(p) >> 20) & 0x7FF, eb = (__double2hiint(pm) >> 20) & 0x7FF;
  const int em = ea > eb ? ea : eb;
  const double f = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em)
  p *= f;
  pm *= f;
}
__device__ int sturm_count_minors(const double* ds, const double* e2s, int n, double x) {
  double pm = 1.0, p = ds[0] - x;
  if (is_zero(p)) p = -0x1p-600;
  int cnt = sign_flip(p, pm);
  for (int i = 1; i < n; ++i) {
    double pn = fma(ds[i] - x, p, -e2s[i - 1] * pm);
    if (is_zero(pn)) pn = -p * 0x1p-600;
    cnt += sign_flip(pn, p);
    pm = p;
    p = pn;
    if ((i & 3) == 0) rescale_pair(p, pm);
  }
  return cnt;
}

// One warp per requested eigenvalue index j (ascending order): 32-point multisection of the
// Sturm count until the bracket reaches the count's resolution eps * ||T||.  (A warp issues
// about one FP64 instruction per 64 cycles on this GPU, dependent or not, so more shifts per
// lane only add time.)  A CTA holds kTopkWarps warps -- one per SM sub-partition, each with its
// own FP64 pipe -- that share one staged copy of the scaled tridiagonal, so that the kernel
// occupies few SMs beside the ingest running on the others.
constexpr int kTopkWarps = 4;

__global__ void __launch_bounds__(32 * kTopkWarps) topk_eig_kernel(Dev d, const double* dvec, const double* evec,
                                                                   int k, double* mu) {
  extern __shared__ double tsm[];
  __shared__ double red[2][kTopkWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = blockIdx.x * kTopkWarps + wid;
  const int n = d.s;
  double* ds = tsm;
  double* e2s = tsm + n;
  // Gershgorin interval, CTA-parallel
  double lo = 1e300, hi = -1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = dvec[i];
    const double r = ((i > 0) ? fabs(evec[i - 1]) : 0.0) + ((i + 1 < n) ? fabs(evec[i]) : 0.0);
    lo = fmin(lo, di - r);
    hi = fmax(hi, di + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) { red[0][wid] = lo; red[1][wid] = hi; }
  __syncthreads();
  lo = red[0][0];
  hi = red[1][0];
  for (int w = 1; w < kTopkWarps; ++w) { lo = fmin(lo, red[0][w]); hi = fmax(hi, red[1][w]); }
  const double sc = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
  const double inv = 1.0 / sc;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ds[i] = dvec[i] * inv;
    if (i + 1 < n) { const double e = evec[i] * inv; e2s[i] = e * e; }
  }
  __syncthreads();
  if (gw >= k || gw >= n) return;             // after the last CTA-wide barrier
  const int j = n - 1 - gw;                    // the gw-th largest
  const double tol = 4.440892098500626e-16;    // in units of sc
  lo = lo * inv - 2.0 * tol;
  hi = hi * inv + 2.0 * tol;
  const double step = 1.0 / 33.0;
  for (int it = 0; it < 64; ++it) {
    const double x = lo + (hi - lo) * ((double)(lane + 1) * step);
    const unsigned msk = __ballot_sync(0xffffffffu, sturm_count_minors(ds, e2s, n, x) > j);  // eig j < x
    // first lane whose point lies above eigenvalue j
    const int a = msk ? __ffs(msk) - 1 : 32;
    const double nlo = (a == 0) ? lo : lo + (hi - lo) * ((double)a * step);
    const double nhi = (a == 32) ? hi : lo + (hi - lo) * ((double)(a + 1) * step);
    if (!(nhi - nlo < hi - lo)) break;
    lo = nlo;
    hi = nhi;
    // the Sturm count's backward error is ~eps * ||T||: narrower brackets carry no information
    if (hi - lo <= tol) break;
  }
  if (lane == 0) mu[gw] = 0.5 * (lo + hi) * sc;
}

// lambda from the k largest eigenvalues (summed largest first), the LDL^T of T + lambda I.
// One warp stages the tridiagonal and the eigenvalues in shared memory; lane 0 then runs
// the two sequential recurrences.
__global__ void __launch_bounds__(32) lambda_ldl_kernel(Dev d, const double* mu, int k, const double* dvec,
                                                        const double* evec, double* ldl_d, double* ldl_l,
                                                        int fro_slot, int lam_slot) {
  extern __shared__ double lsm[];
  const int n = d.s, lane = threadIdx.x;
  const int kk = k < n ? k : n;
  double* sd = lsm;            // n
  double* se = sd + n;         // n - 1
  double* smu = se + n;        // kk
  for (int i = lane; i < n; i += 32) { sd[i] = dvec[i]; if (i + 1 < n) se[i] = evec[i]; }
  if (d.lambda_mode != 1)
    for (int i = lane; i < kk; i += 32) smu[i] = mu[i];
  __syncwarp();
  if (lane != 0) return;
  double lam;
  if (d.lambda_mode == 1) {
    lam = d.lambda_fixed;
  } else {
    double top = 0.0;
    for (int i = 0; i < kk; ++i) top += smu[i];
    const double fro = d.fro2[1];
    lam = (fro - top) / (double)k;
    lam = fmax(lam, 1e-12 * fro / (double)k);
  }
  d.scal[lam_slot] = lam;
  d.scal[fro_slot] = d.fro2[0];         // the step's ||A_obs||^2: later ingest may add to fro2
  // T + lambda I = L D L^T; ldl_d holds the inverse pivots 1/D_i (0 for a non-positive pivot)
  double del = sd[0] + lam;
  for (int i = 1; i < n; ++i) {
    const double inv = (del != 0.0) ? 1.0 / del : 0.0;
    ldl_d[i - 1] = (del > 0.0) ? inv : 0.0;
    const double l = se[i - 1] * inv;
    ldl_l[i - 1] = l;
    del = sd[i] + lam - l * se[i - 1];
  }
  ldl_d[n - 1] = (del > 0.0) ? 1.0 / del : 0.0;
}

// One warp per vector: occupied C slots (v < t) and buffered D columns (t <= v < t + count).
__global__ void __launch_bounds__(32)
tri_scores_kernel(Dev d, const double* R, const double* beta, const double* vhead,
                  const double* ldl_d, const double* ldl_l, double* vecbuf, int vstride, int count,
                  int64_t jd0) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = d.s;
  const double rs = 1.0 / sqrt((double)n);
  double* y = vecbuf + (size_t)gw * vstride;
  for (int vi = gw; vi < d.t + count; vi += nwarps) {
    int64_t col;
    if (vi < d.t) { col = d.JC[vi]; if (col < 0) { if (lane == 0) d.tauC[vi] = 1.0; continue; } }
    else col = jd0 + (vi - d.t);            // buffered column q of the batch is jd0 + q
    const double* l = d.Slev + (size_t)col * d.lev_ld;
    for (int i = lane; i < n; i += 32) y[i] = l[i] * rs;
    __syncwarp();
    for (int k = 0; k + 2 < n; ++k) {          // y <- H_{n-3} ... H_0 y
      const double bt = beta[k];
      if (bt == 0.0) continue;
      const double* u = R + (size_t)k * n;       // u[k+1] = vhead[k], u[i] = R(i, k) for i >= k+2
      const double vh = vhead[k];
      double dot = (lane == 0) ? vh * y[k + 1] : 0.0;
      for (int i = k + 2 + lane; i < n; i += 32) dot += u[i] * y[i];
      dot = warp_sum(dot);
      const double f = bt * dot;
      __syncwarp();
      if (lane == 0) y[k + 1] -= f * vh;
      for (int i = k + 2 + lane; i < n; i += 32) y[i] -= f * u[i];
      __syncwarp();
    }
    if (lane == 0) {
      // tau = y^T (L D L^T)^{-1} y = sum_i z_i^2 / D_i with L z = y
      double z = y[0];
      double tau = z * z * ldl_d[0];            // ldl_d: inverse pivots, 0 where D_i <= 0
      for (int i = 1; i < n; ++i) {
        z = y[i] - ldl_l[i - 1] * z;
        tau += z * z * ldl_d[i];
      }
      if (vi < d.t) d.tauC[vi] = tau; else d.tauD[vi - d.t] = tau;
    }
    __syncwarp();
  }
}

// Cluster sizes to try in order (the first the device co-schedules is taken), or only the size
// named by the environment variable (8 or 16).  A smaller cluster leaves SMs to the ingest that
// runs beside the batch step and makes the step's own kernel slower: on the channel-flow
// benchmark (GB300) a QR cluster of 8 measured 1.7 % faster than 16 over three alternating runs,
// a tridiagonalization cluster of 8 5.5 % slower.
std::array<int, 2> cluster_candidates(const char* var, std::array<int, 2> order) {
  const char* e = getenv(var);
  if (e && (atoi(e) == 8 || atoi(e) == 16)) return {atoi(e), 0};
  return order;
}

size_t tri_cluster_smem(int n, int C) {
  const int ncl = (n + C - 1) / C;
  return ((size_t)ncl * n + 6 * (size_t)n) * sizeof(double);
}

// Cluster size for the shared-memory tridiagonalization of an n x n matrix: 16 (non-portable)
// or else 8 CTAs when the columns fit and the device can co-schedule the cluster, else 0.
int tri_cluster_size(int n) {
  static int cached_n = -1, cached_c = 0;
  if (n == cached_n) return cached_c;
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int best = 0;
  cudaFuncAttributes fa;
  const bool have_fa = cudaFuncGetAttributes(&fa, tridiag_cluster_kernel) == cudaSuccess;
  max_smem -= have_fa ? (int)fa.sharedSizeBytes : 0;          // static shared memory comes first
  if (have_fa &&
      cudaFuncSetAttribute(tridiag_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(tridiag_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) ==
          cudaSuccess) {
    for (int C : cluster_candidates("RID_TRI_CLUSTER", {16, 8})) {
      if (C == 0) continue;
      if (tri_cluster_smem(n, C) + 2048 > (size_t)max_smem || n < 2 * C) continue;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)C);
      cfg.blockDim = dim3(kTriThreads);
      cfg.dynamicSmemBytes = tri_cluster_smem(n, C);
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, tridiag_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0) {
        best = C;
        break;
      }
    }
  }
  cudaGetLastError();
  cached_n = n;
  cached_c = best;
  return best;
}

// The same scores with one 128-thread CTA per vector (n <= 512): thread t holds rows t + 128 q
// (q < 4) of y in registers; each reflector costs one CTA reduction (warp sums added in a fixed
// order) and the next reflector's entries are loaded while the current one is applied.  Then
// z = L^{-1} y is a first-order linear recurrence, solved as a scan of affine maps over
// contiguous 4-row segments, and tau = sum_i z_i^2 / D_i.
constexpr int kScThreads = 128, kScRows = 4;

__global__ void __launch_bounds__(kScThreads)
tri_scores_cta_kernel(Dev d, const double* __restrict__ R, const double* __restrict__ beta,
                      const double* __restrict__ vhead, const double* __restrict__ inv_d,
                      const double* __restrict__ ldl_l, int count, int64_t jd0) {
  __shared__ double red[kScThreads / 32];
  __shared__ double fsh;
  __shared__ double ys[kScThreads * kScRows];
  __shared__ double wa[kScThreads / 32], wb[kScThreads / 32], wz[kScThreads / 32];
  const int vi = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = d.s;
  int64_t col;
  if (vi < d.t) {
    col = d.JC[vi];
    if (col < 0) { if (tid == 0) d.tauC[vi] = 1.0; return; }   // uniform over the CTA
  } else {
    col = jd0 + (vi - d.t);                 // buffered column q of the batch is jd0 + q
  }
  const double rs = 1.0 / sqrt((double)n);
  const double* l = d.Slev + (size_t)col * d.lev_ld;
  double y[kScRows], un[kScRows];
#pragma unroll
  for (int q = 0; q < kScRows; ++q) {
    const int r = tid + kScThreads * q;
    y[q] = (r < n) ? l[r] * rs : 0.0;
  }
  auto load_u = [&](int k) {
#pragma unroll
    for (int q = 0; q < kScRows; ++q) {
      const int r = tid + kScThreads * q;
      un[q] = (r >= k + 2 && r < n) ? R[(size_t)r + (size_t)k * n] : 0.0;
    }
  };
  double bn = 0.0, vn = 0.0;
  if (n > 2) { load_u(0); bn = beta[0]; vn = vhead[0]; }
  for (int k = 0; k + 2 < n; ++k) {          // y <- H_{n-3} ... H_0 y
    double u[kScRows];
#pragma unroll
    for (int q = 0; q < kScRows; ++q) u[q] = un[q];
    const double bt = bn, vh = vn;
    if (k + 3 < n) { load_u(k + 1); bn = beta[k + 1]; vn = vhead[k + 1]; }
    if (bt == 0.0) continue;                 // uniform
    double dot = 0.0;
#pragma unroll
    for (int q = 0; q < kScRows; ++q) {
      const int r = tid + kScThreads * q;
      dot = fma(u[q], y[q], dot);
      if (r == k + 1) dot = fma(vh, y[q], dot);
    }
    dot = warp_sum(dot);
    if (lane == 0) red[wid] = dot;
    __syncthreads();
    if (tid == 0) fsh = bt * ((red[0] + red[1]) + (red[2] + red[3]));
    __syncthreads();
    const double f = fsh;
#pragma unroll
    for (int q = 0; q < kScRows; ++q) {
      const int r = tid + kScThreads * q;
      y[q] = fma(-f, u[q], y[q]);
      if (r == k + 1) y[q] = fma(-f, vh, y[q]);
    }
  }
  // L z = y: z_0 = y_0, z_i = y_i - l_{i-1} z_{i-1}; thread t takes rows 4t .. 4t+3
#pragma unroll
  for (int q = 0; q < kScRows; ++q) ys[tid + kScThreads * q] = y[q];
  __syncthreads();
  const int r0 = kScRows * tid;
  double A = 1.0, B = 0.0;                   // z_out = A z_in + B over this segment
#pragma unroll
  for (int q = 0; q < kScRows; ++q) {
    const int r = r0 + q;
    if (r < n) {
      const double a = (r == 0) ? 0.0 : -ldl_l[r - 1];
      B = fma(a, B, ys[r]);
      A = a * A;
    }
  }
  // inclusive scan of the maps over the lanes (earlier lanes applied first)
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
    if (lane >= o) { B = fma(A, Bp, B); A = A * Ap; }
  }
  if (lane == 31) { wa[wid] = A; wb[wid] = B; }
  __syncthreads();
  if (tid == 0) {
    double z = 0.0;                           // z entering warp 0 (none before row 0)
    for (int w = 0; w < kScThreads / 32; ++w) { wz[w] = z; z = fma(wa[w], z, wb[w]); }
  }
  __syncthreads();
  // exclusive prefix of this lane = inclusive prefix of the previous lane
  double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) { Ae = 1.0; Be = 0.0; }
  double z = fma(Ae, wz[wid], Be);          // z_{r0 - 1}
  double tau = 0.0;
#pragma unroll
  for (int q = 0; q < kScRows; ++q) {
    const int r = r0 + q;
    if (r < n) {
      const double a = (r == 0) ? 0.0 : -ldl_l[r - 1];
      z = fma(a, z, ys[r]);
      tau = fma(z * z, inv_d[r], tau);
    }
  }
  tau = warp_sum(tau);
  __syncthreads();
  if (lane == 0) red[wid] = tau;
  __syncthreads();
  if (tid == 0) {
    const double tt = (red[0] + red[1]) + (red[2] + red[3]);
    if (vi < d.t) d.tauC[vi] = tt; else d.tauD[vi - d.t] = tt;
  }
}

// Tridiagonalization, top-k eigenvalues and lambda / LDL^T; returns the number of kernels
// launched (0 on failure).
int launch_lambda(const Dev& d, int batch, double* work_base, int64_t off_A, int64_t off_R, int64_t off_d,
                  int64_t off_e, int64_t off_beta, int64_t off_vhead, int64_t off_p, int64_t off_mu,
                  int64_t off_ldld, int64_t off_ldll, unsigned int* bar_mem, int n_sm, cudaStream_t st) {
  double* A = work_base + off_A;
  double* R = work_base + off_R;
  double* dv = work_base + off_d;
  double* ev = work_base + off_e;
  double* bt = work_base + off_beta;
  double* vh = work_base + off_vhead;
  double* pg = work_base + off_p;
  double* mu = work_base + off_mu;
  double* ld = work_base + off_ldld;
  double* ll = work_base + off_ldll;
  const size_t shm = (size_t)3 * d.s * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tridiag_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 4096 * 8);
    cudaFuncSetAttribute(topk_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8);
    cudaFuncSetAttribute(lambda_ldl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 4096 * 8);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_coop_kernel, kCoopThreads, shm);
  int grid = n_sm * (per_sm > 0 ? 1 : 0);
  const int want = d.s - 1;                     // at least one trailing column per block
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  const int C = tri_cluster_size(d.s);
  if (C > 0) {
    const int ncl = (d.s + C - 1) / C;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kTriThreads);
    cfg.dynamicSmemBytes = tri_cluster_smem(d.s, C);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel, d, R, dv, ev, bt, vh, ncl) != cudaSuccess) return 0;
  } else {
    cudaMemsetAsync(bar_mem, 0, 4 * sizeof(unsigned int), st);
    GridBar gb{bar_mem, bar_mem + 1, d.err, (int*)(bar_mem + 2)};
    Dev dd = d;
    void* args[] = {&dd, &A, &R, &dv, &ev, &bt, &vh, &pg, &gb};
    if (cudaLaunchCooperativeKernel((void*)tridiag_coop_kernel, grid, kCoopThreads, args, shm, st) != cudaSuccess)
      return 0;
  }
  int nk = 2;
  const int k = d.t;
  if (d.lambda_mode == 0) {
    topk_eig_kernel<<<(k + kTopkWarps - 1) / kTopkWarps, 32 * kTopkWarps, (size_t)2 * d.s * sizeof(double), st>>>(
        d, dv, ev, k, mu);                                                           // FP64-bound
    ++nk;
  }
  lambda_ldl_kernel<<<1, 32, (size_t)(2 * d.s + (k < d.s ? k : d.s)) * sizeof(double), st>>>(
      d, mu, k, dv, ev, ld, ll, SCAL_FRO0 + (batch & 7), SCAL_LAMBDA + (batch & 1));
  return nk + 1;
}

// Sketched ridge scores of the occupied C slots and the count buffered columns.
int launch_scores(const Dev& d, int count, int64_t jd0, double* work_base, int64_t off_R, int64_t off_beta,
                  int64_t off_vhead, int64_t off_ldld, int64_t off_ldll, int64_t off_vec, int vstride,
                  cudaStream_t st) {
  const int nvec = d.t + count;
  if (d.s <= kScThreads * kScRows) {
    tri_scores_cta_kernel<<<nvec, kScThreads, 0, st>>>(d, work_base + off_R, work_base + off_beta,
                                                      work_base + off_vhead, work_base + off_ldld,
                                                      work_base + off_ldll, count, jd0);
    return 1;
  }
  tri_scores_kernel<<<nvec, 32, 0, st>>>(d, work_base + off_R, work_base + off_beta, work_base + off_vhead,
                                         work_base + off_ldld, work_base + off_ldll, work_base + off_vec,
                                         vstride, count, jd0);
  return 1;
}

}  // namespace rid

namespace rid {

// Householder QR of the m x n matrix A (column-major, lda = m) on every SM, one grid
// barrier per column: all blocks form reflector j from column j, each block applies it
// to the columns it owns (l % gridDim.x == blockIdx.x, l > j).  Column j is never
// rewritten: reflector j = [vhead[j]; A(j+1:m, j)], R(j, j) = rdiag[j], R(i, j) = A(i, j)
// for i < j.
__device__ bool qr_coop(double* A, int m, int n, double* beta, double* vhead, double* rdiag,
                        const GridBar& bar, double* sh) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  for (int j = 0; j < n; ++j) {
    const double* col = A + (size_t)j * m;
    double part = 0.0;
    for (int i = j + tid; i < m; i += blockDim.x) part += col[i] * col[i];
    const double nrm2 = block_sum(part, sh);
    const double x0 = col[j];
    const double nrm = sqrt(nrm2);
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vtv = nrm2 - x0 * x0 + v0 * v0;
    const double bt = (nrm2 > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
    if (b == 0 && tid == 0) { beta[j] = bt; vhead[j] = v0; rdiag[j] = (bt > 0.0) ? alpha : x0; }
    if (bt > 0.0) {
      const int l0 = j + 1 + ((b - (j + 1)) % G + G) % G;   // first owned column after j
      for (int l = l0 + wid * G; l < n; l += nw * G) {
        double* a = A + (size_t)l * m;
        double dot = (lane == 0) ? v0 * a[j] : 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) dot += col[i] * a[i];
        dot = warp_sum(dot);
        const double f = bt * dot;
        if (lane == 0) a[j] -= f * v0;
        for (int i = j + 1 + lane; i < m; i += 32) a[i] -= f * col[i];
      }
    }
    if (!grid_barrier(bar)) return false;
  }
  return true;
}

__global__ void __launch_bounds__(kCoopThreads)
qr_coop_kernel(Dev d, double* Q4, double* b4, double* h4, double* r4, double* Q6, double* b6,
               double* h6, double* r6, GridBar bar) {
  __shared__ double sh[33];
  const int na = d.meta[META_NACT], nn = d.meta[META_NNEW];
  if (!qr_coop(Q4, d.s, na, b4, h4, r4, bar, sh)) return;
  qr_coop(Q6, d.s, nn, b6, h6, r6, bar, sh);
}

// Householder QR of the m x n matrix A (column-major, lda = m), with the same outputs as
// qr_coop, on one thread-block cluster: CTA r holds the columns l with l % C == r in shared
// memory.  At step j every CTA reads column j (rows j..m-1) from its owner -- final since
// step j-1, and never written again -- forms reflector j (scalars on one thread), and applies
// it to its own columns l > j; one cluster barrier per step.  n is read on the device
// (meta[n_item]); control flow is uniform over the cluster.
__global__ void __launch_bounds__(kTriThreads, 1)
qr_cluster_kernel(Dev d, double* A, int n_item, double* beta, double* vhead, double* rdiag, int ncl) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int m = d.s, n = d.meta[n_item];
  if (n <= 0) return;                          // uniform over the cluster
  const int ldc = m | 1;
  extern __shared__ double qsm[];
  double* cols = qsm;                          // ncl x ldc
  double* x = cols + (size_t)ncl * ldc;        // column j, rows j..m-1
  __shared__ double sh[33];
  __shared__ double scal[2];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int nown = (n - rank + C - 1) / C;
  for (int lc = wid; lc < nown; lc += nw) {
    const double* src = A + (size_t)(lc * C + rank) * m;
    for (int i = lane; i < m; i += 32) cols[(size_t)lc * ldc + i] = src[i];
  }
  cl.sync();
  for (int j = 0; j < n; ++j) {
    const int mj = m - j;
    {
      const double* src = cl.map_shared_rank(cols, j % C) + (size_t)(j / C) * ldc + j;
      for (int i = tid; i < mj; i += blockDim.x) x[i] = src[i];
    }
    __syncthreads();
    if (wid < kRedWarps) {
      double part = 0.0;
      for (int i = tid; i < mj; i += 32 * kRedWarps) part += x[i] * x[i];
      part = warp_sum(part);
      if (lane == 0) sh[wid] = part;
    }
    __syncthreads();
    if (tid == 0) {
      double nrm2 = 0.0;
      for (int i = 0; i < kRedWarps; ++i) nrm2 += sh[i];
      const double x0 = x[0];
      const double nrm = sqrt(nrm2);
      const double alpha = (x0 >= 0.0) ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vtv = nrm2 - x0 * x0 + v0 * v0;
      const double bt = (nrm2 > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
      scal[0] = bt;
      scal[1] = v0;
      if (rank == 0) { beta[j] = bt; vhead[j] = v0; rdiag[j] = (bt > 0.0) ? alpha : x0; }
    }
    __syncthreads();
    const double bt = scal[0], v0 = scal[1];
    if (bt > 0.0) {
      const int lc0 = (j + 1 - rank + C - 1) / C;   // first owned column > j
      for (int lc = lc0 + wid; lc < nown; lc += nw) {
        double* a = cols + (size_t)lc * ldc;
        double dot = (lane == 0) ? v0 * a[j] : 0.0;
        for (int i = 1 + lane; i < mj; i += 32) dot += x[i] * a[j + i];
        dot = warp_sum(dot);
        const double f = bt * dot;
        if (lane == 0) a[j] -= f * v0;
        for (int i = 1 + lane; i < mj; i += 32) a[j + i] -= f * x[i];
      }
    }
    cl.sync();                                  // column j+1 is final; x may be overwritten
  }
  for (int lc = wid; lc < nown; lc += nw) {
    double* dst = A + (size_t)(lc * C + rank) * m;
    for (int i = lane; i < m; i += 32) dst[i] = cols[(size_t)lc * ldc + i];
  }
  cl.sync();                                    // no CTA leaves while its shared memory may be read
}

// Cluster size for qr_cluster_kernel with up to t columns of length m (0: not available).
int qr_cluster_size(int m, int t) {
  static int cached_m = -1, cached_t = -1, cached_c = 0;
  if (m == cached_m && t == cached_t) return cached_c;
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  int best = 0;
  if (cudaFuncGetAttributes(&fa, qr_cluster_kernel) == cudaSuccess) {
    max_smem -= (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(qr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(qr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) ==
            cudaSuccess) {
      for (int C : cluster_candidates("RID_QR_CLUSTER", {8, 16})) {
        if (C == 0) continue;
        const size_t smem = ((size_t)((t + C - 1) / C) * (m | 1) + m) * sizeof(double);
        if (smem + 1024 > (size_t)max_smem) continue;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kTriThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, qr_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0) {
          best = C;
          break;
        }
      }
    }
  }
  cudaGetLastError();
  cached_m = m;
  cached_t = t;
  cached_c = best;
  return best;
}

// Whether the current context -- a green context's SM partition -- can co-schedule the batch
// step's thread-block clusters at the sizes tri_cluster_size and qr_cluster_size chose (for s x s
// sketch Grams and t basis columns).  A partition that cannot would leave their launches waiting.
bool batch_clusters_fit(int s, int t) {
  const int ct = tri_cluster_size(s), cq = qr_cluster_size(s, t);
  if (ct <= 0 || cq <= 0) return false;
  auto fits = [](const void* fn, int C, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kTriThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();
    return ok;
  };
  const int ncl = (t + cq - 1) / cq;
  return fits((const void*)tridiag_cluster_kernel, ct, tri_cluster_smem(s, ct)) &&
         fits((const void*)qr_cluster_kernel, cq, ((size_t)ncl * (s | 1) + s) * sizeof(double));
}

int launch_qr_coop(const Dev& d, double* Q4, double* b4, double* h4, double* r4, double* Q6,
                   double* b6, double* h6, double* r6, unsigned int* bar_mem, cudaStream_t st) {
  const int C = qr_cluster_size(d.s, d.t);
  if (C > 0) {
    // one small cluster: unlike the grid version it needs no co-residency of ~t CTAs, which
    // the long-lived ingest CTAs running beside the batch step would delay
    const int ncl = (d.t + C - 1) / C;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kTriThreads);
    cfg.dynamicSmemBytes = ((size_t)ncl * (d.s | 1) + d.s) * sizeof(double);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, qr_cluster_kernel, d, Q4, (int)META_NACT, b4, h4, r4, ncl) != cudaSuccess) return 0;
    if (cudaLaunchKernelEx(&cfg, qr_cluster_kernel, d, Q6, (int)META_NNEW, b6, h6, r6, ncl) != cudaSuccess) return 0;
    return 1;
  }
  int grid = d.n_sm < d.t ? d.n_sm : d.t;
  if (grid < 1) grid = 1;
  cudaMemsetAsync(bar_mem, 0, 4 * sizeof(unsigned int), st);
  GridBar gb{bar_mem, bar_mem + 1, d.err, (int*)(bar_mem + 2)};
  Dev dd = d;
  void* args[] = {&dd, &Q4, &b4, &h4, &r4, &Q6, &b6, &h6, &r6, &gb};
  if (cudaLaunchCooperativeKernel((void*)qr_coop_kernel, grid, kCoopThreads, args, 0, st) != cudaSuccess)
    return 0;
  return 1;
}

}  // namespace rid
