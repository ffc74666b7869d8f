// Online column subset selection by residual-based sampling: the paper's Algorithm 1 (Sec. 2.2.1,
// from Bhaskara et al.), the comparison selector of the accuracy tables -- not part of the
// single-pass ID, which uses Algorithm 3.
//
// For each arriving column a (global index j): p_a = k ||Pi_perp a||^2 / xi with Pi_perp the
// projector onto the orthogonal complement of span(C_pre); a joins C_cur when u_j < min(p_a, 1)
// (u_j: the 53-bit uniform of Philox((j mod 2^32, j >> 32, 'RCS1', 0))); if p_a < 1 the residual
// mass sigma grows by p_a; if p_a >= 1 or sigma >= 1, C_pre takes C_cur's columns and sigma = 0.
//
// With stop_at_cap, the selection stops growing at cap columns (the treatment of the experiments,
// Sec. 4.1): a later keep decision adds nothing; p, sigma and the steps go on.
//
// Device state: an orthonormal basis Q of span(C_pre) (cap vectors of m_pad, the data's type),
// the raw columns of C_cur, and the selection list.  Per block of up to 64 columns:
//   1. rcss_norms_kernel: ||a||^2 of the block's columns; rcss_dots_kernel (for blocks of up to
//      16 columns rcss_thin_stage_kernel on FP32 data, rcss_thin_kernel on FP64): the dot products of
//      the basis with the block's columns (FP32 or FP64 products summed over runs of 128
//      coordinates, each run's sums added into per-CTA FP64 partials); rcss_reduce_kernel adds the
//      partials in CTA order into X (basis vector x block column);
//   2. rcss_decide_kernel (one thread, FP64): the decisions of Algorithm 1 for the block's columns
//      in order, ||Pi_perp a||^2 = ||a||^2 - ||Q^T a||^2; it stops after a column that ends a step;
//   3. the host copies the block's newly kept columns into the C_cur store and, after a step's
//      end, extends Q by each C_cur column in turn: two rounds of classical Gram-Schmidt (dots of Q
//      with the vector by rcss_gemv_kernel, rcss_axpy_kernel for v - Q c), a norm, and rcss_scale_kernel, which
//      normalizes the vector into the next basis slot unless its residual norm is at most tol
//      times its norm; the dots of the new basis vectors with the rest of the block are appended
//      to X, and the rest of the block is decided against the grown basis.
// The host reads the decide kernel's small result record after each decision pass: which columns
// to copy and whether a step ended (control flow only; every number is computed on the device).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "philox.cuh"
#include "rid.h"
#include "rid_internal.cuh"

namespace rid {

namespace {

constexpr uint32_t kTagRcss = 0x52435331u;   // 'RCS1'
constexpr int kRcBlock = 64;                  // columns per block
constexpr int kRcRun = 128;                   // coordinates per run
constexpr int kRcLd = 65;                     // shared row stride (coordinate-major, padded)
constexpr int kRcThreads = 256;
constexpr int kRcTile = 64;                   // V vectors per tile
constexpr int kRcMaxCap = 4096;               // largest selection (and basis) capacity

struct RcssRec {                              // the decide kernel's result for the host
  int stop;                                   // last column index of the block decided
  int step_end;                               // 1: that column ended a step (C_pre takes C_cur)
  int nkeep;                                  // block columns kept (C_cur members), in order
  int keep[kRcBlock];                         // their positions in the block
  int overflow;                               // the selection would exceed its capacity
};

struct RcssDevState {
  double sigma;
  int64_t n_obs;
  int nsel;                                   // selection list length
  int pad;
};

// Stage n vectors' coordinates i0 .. i0 + kRcRun - 1 (zero past m) into dst[ii * kRcLd + v]:
// element e = v * kRcRun + ii, kRcThreads apart per thread, 8 loads in flight before the stores.
template <typename T>
__device__ __forceinline__ void rcss_stage(T* dst, const T* const* __restrict__ src, int n, int64_t i0, int64_t m) {
  constexpr int U = 8;
  const int tid = threadIdx.x;
  for (int e0 = 0; e0 < n * kRcRun; e0 += U * kRcThreads) {
    T val[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kRcThreads + tid;
      const int v = e / kRcRun, ii = e - v * kRcRun;
      val[u] = (e < n * kRcRun && i0 + ii < m) ? src[v][i0 + ii] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kRcThreads + tid;
      const int v = e / kRcRun, ii = e - v * kRcRun;
      if (e < n * kRcRun) dst[ii * kRcLd + v] = val[u];
    }
  }
}

// V_v . A_a over this CTA's coordinate range for v < nv, a < na: per run of kRcRun coordinates the
// block's columns and a tile of kRcTile vectors are staged in shared memory, coordinate-major with
// a padded row (kRcLd) so that neither the staging stores nor the 4-wide reads conflict; thread t
// owns a 4 x 4 register tile of (v, a) pairs; each run's sums are added into the CTA's FP64
// partials part[cta][v][a] (read-modify-write by the owning thread).
template <typename T>
__global__ void __launch_bounds__(kRcThreads)
rcss_dots_kernel(const T* const* __restrict__ V, int nv, const T* const* __restrict__ A, int na, int64_t m,
                 int64_t runs_per_cta, int vmax, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char rsm[];
  T* As = reinterpret_cast<T*>(rsm);                         // kRcRun x kRcLd
  T* Vs = As + (size_t)kRcRun * kRcLd;                       // kRcRun x kRcLd
  const int tid = threadIdx.x;
  const int ta = (tid & 15) * 4, tv = (tid >> 4) * 4;        // 16 x 16 threads, 4 x 4 each
  double* P = part + (size_t)blockIdx.x * vmax * kRcBlock;
  for (int idx = tid; idx < nv * kRcBlock; idx += kRcThreads) P[idx] = 0.0;
  const int64_t nruns = (m + kRcRun - 1) / kRcRun;
  const int64_t r0 = (int64_t)blockIdx.x * runs_per_cta;
  const int64_t r1 = r0 + runs_per_cta < nruns ? r0 + runs_per_cta : nruns;
  for (int64_t run = r0; run < r1; ++run) {
    const int64_t i0 = run * kRcRun;
    __syncthreads();
    rcss_stage(As, A, na, i0, m);
    for (int vt = 0; vt < nv; vt += kRcTile) {
      const int nvt = nv - vt < kRcTile ? nv - vt : kRcTile;
      __syncthreads();
      rcss_stage(Vs, V + vt, nvt, i0, m);
      __syncthreads();
      if (tv < nvt && ta < na) {
        T acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
        for (int ii = 0; ii < kRcRun; ++ii) {
          T vv[4], aa[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) vv[x] = Vs[ii * kRcLd + tv + x];
#pragma unroll
          for (int y = 0; y < 4; ++y) aa[y] = As[ii * kRcLd + ta + y];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(vv[x], aa[y], acc[x][y]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y)
            if (tv + x < nvt && ta + y < na) P[(size_t)(vt + tv + x) * kRcBlock + ta + y] += (double)acc[x][y];
      }
    }
  }
}

// The same products for thin blocks (na <= NA <= 16): thread t of vector group blockIdx.y owns
// vector v = 256 blockIdx.y + t and streams it with 16-byte loads (8 in flight); the block's
// columns are staged kThinRuns runs at a time, coordinate-major (As[i * NA + a], zero past na and
// m), and read as 16-byte broadcasts.  The coordinate partition (CTAs over runs), the per-run sums
// in the data's type (fma in coordinate order from zero) and their FP64 accumulation in run order
// are those of rcss_dots_kernel, so both write bit-identical partials.  V must be 16-byte aligned
// with zeros from m up to the next multiple of kRcRun (the basis slots are).
constexpr int kThinRuns = 4;

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ T v16_get(const typename Vec16<T>::type& q, int e);
template <>
__device__ __forceinline__ float v16_get<float>(const float4& q, int e) {
  return e == 0 ? q.x : e == 1 ? q.y : e == 2 ? q.z : q.w;
}
template <>
__device__ __forceinline__ double v16_get<double>(const double2& q, int e) { return e == 0 ? q.x : q.y; }

template <typename T, int NA>
__global__ void __launch_bounds__(kRcThreads)
rcss_thin_kernel(const T* const* __restrict__ V, int nv, const T* const* __restrict__ A, int na, int64_t m,
                 int64_t runs_per_cta, int vmax, double* __restrict__ part) {
  using VT = typename Vec16<T>::type;
  constexpr int EPV = Vec16<T>::n;                         // elements per 16-byte load
  constexpr int CH = kThinRuns * kRcRun;                   // coordinates staged at a time
  constexpr int LPR = kRcRun / EPV;                        // 16-byte loads per run
  constexpr int B = 8;                                     // loads in flight
  extern __shared__ __align__(16) unsigned char rsm[];
  T* As = reinterpret_cast<T*>(rsm);                       // CH x NA
  const int tid = threadIdx.x;
  const int v = blockIdx.y * kRcThreads + tid;
  const bool own = v < nv;
  const VT* vp = own ? reinterpret_cast<const VT*>(V[v]) : nullptr;
  double acc64[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) acc64[a] = 0.0;
  const int64_t nruns = (m + kRcRun - 1) / kRcRun;
  const int64_t r0 = (int64_t)blockIdx.x * runs_per_cta;
  const int64_t r1 = r0 + runs_per_cta < nruns ? r0 + runs_per_cta : nruns;
  for (int64_t rc = r0; rc < r1; rc += kThinRuns) {
    const int nr = (int)(r1 - rc < kThinRuns ? r1 - rc : kThinRuns);
    const int64_t c0 = rc * kRcRun;
    __syncthreads();
    for (int e0 = 0; e0 < NA * CH; e0 += 8 * kRcThreads) {
      T val[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kRcThreads + tid;
        const int a = e / CH, i = e - a * CH;
        val[u] = (e < NA * CH && a < na && i < nr * kRcRun && c0 + i < m) ? A[a][c0 + i] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kRcThreads + tid;
        const int a = e / CH, i = e - a * CH;
        if (e < NA * CH) As[i * NA + a] = val[u];
      }
    }
    __syncthreads();
    if (own) {
      for (int r = 0; r < nr; ++r) {
        T acc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = T(0);
        const VT* src = vp + ((c0 + (int64_t)r * kRcRun) / EPV);
        const T* arow = As + (size_t)r * kRcRun * NA;
        for (int l0 = 0; l0 < LPR; l0 += B) {
          VT q[B];
#pragma unroll
          for (int u = 0; u < B; ++u) q[u] = src[l0 + u];
#pragma unroll
          for (int u = 0; u < B; ++u)
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
              const T x = v16_get<T>(q[u], e);
              const VT* ab = reinterpret_cast<const VT*>(arow + ((l0 + u) * EPV + e) * NA);
#pragma unroll
              for (int g = 0; g < NA / EPV; ++g) {
                const VT y = ab[g];
#pragma unroll
                for (int h = 0; h < EPV; ++h) acc[g * EPV + h] = fma(x, v16_get<T>(y, h), acc[g * EPV + h]);
              }
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) acc64[a] += (double)acc[a];
      }
    }
  }
  if (own) {
    double* P = part + ((size_t)blockIdx.x * vmax + v) * kRcBlock;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (a < na) P[a] = acc64[a];
  }
}

// FP32 form of the thin-block products with coalesced basis reads: per run, the tile of up to
// kStTile basis vectors (kRcRun coordinates each) is copied into shared memory by 16-byte
// cp.async (32 consecutive threads per vector and run), padded to kStLd floats per row so that
// each thread's 16-byte reads of its own row do not conflict, and the block's columns by 4-byte
// cp.async (zero past na and m); two stages, the next run's copies in flight while the current one
// is used.  Thread t owns vector kStTile * blockIdx.y + t.  The arithmetic -- per-run fma in
// coordinate order from zero, FP64 accumulation in run order, the CTAs' partition of the runs --
// is rcss_dots_kernel's, so the partials are bit-identical.  Basis rows must be 16-byte aligned
// and zero from m up to the next multiple of kRcRun.
constexpr int kStTile = 128;
constexpr int kStLd = kRcRun + 4;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

template <int NA>
__global__ void __launch_bounds__(kStTile)
rcss_thin_stage_kernel(const float* const* __restrict__ V, int nv, const float* const* __restrict__ A, int na,
                       int64_t m, int64_t runs_per_cta, int vmax, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char rsm[];
  float* Vs = reinterpret_cast<float*>(rsm);                         // 2 x kStTile x kStLd
  float* As = Vs + 2 * kStTile * kStLd;                              // 2 x kRcRun x NA
  const int tid = threadIdx.x;
  const int vbase = blockIdx.y * kStTile;
  const int nvt = nv - vbase < kStTile ? nv - vbase : kStTile;
  const bool own = tid < nvt;
  double acc64[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) acc64[a] = 0.0;
  const int64_t nruns = (m + kRcRun - 1) / kRcRun;
  const int64_t r0 = (int64_t)blockIdx.x * runs_per_cta;
  const int64_t r1 = r0 + runs_per_cta < nruns ? r0 + runs_per_cta : nruns;
  const uint32_t vs0 = (uint32_t)__cvta_generic_to_shared(Vs);
  const uint32_t as0 = (uint32_t)__cvta_generic_to_shared(As);
  const float* any = A[0];
  auto issue = [&](int64_t run, int stage) {
    const int64_t i0 = run * kRcRun;
    for (int c = tid; c < nvt * (kRcRun / 4); c += kStTile) {
      const int row = c / (kRcRun / 4), q = c - row * (kRcRun / 4);
      cp_async16(vs0 + (uint32_t)(((stage * kStTile + row) * kStLd + 4 * q) * 4), V[vbase + row] + i0 + 4 * q);
    }
    for (int e = tid; e < NA * kRcRun; e += kStTile) {
      const int a = e / kRcRun, ii = e - a * kRcRun;
      const bool in = a < na && i0 + ii < m;
      cp_async4(as0 + (uint32_t)(((stage * kRcRun + ii) * NA + a) * 4), in ? A[a] + i0 + ii : any, in ? 4 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (r0 < r1) issue(r0, 0);
  for (int64_t run = r0; run < r1; ++run) {
    const int stage = (int)((run - r0) & 1);
    if (run + 1 < r1) {
      issue(run + 1, stage ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (own) {
      float acc[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) acc[a] = 0.f;
      const float4* vrow = reinterpret_cast<const float4*>(Vs + (stage * kStTile + tid) * kStLd);
      const float* arow = As + stage * kRcRun * NA;
#pragma unroll 4
      for (int l = 0; l < kRcRun / 4; ++l) {
        const float4 q = vrow[l];
        const float xs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4* ab = reinterpret_cast<const float4*>(arow + (4 * l + e) * NA);
#pragma unroll
          for (int g = 0; g < NA / 4; ++g) {
            const float4 y = ab[g];
            acc[4 * g + 0] = fmaf(xs[e], y.x, acc[4 * g + 0]);
            acc[4 * g + 1] = fmaf(xs[e], y.y, acc[4 * g + 1]);
            acc[4 * g + 2] = fmaf(xs[e], y.z, acc[4 * g + 2]);
            acc[4 * g + 3] = fmaf(xs[e], y.w, acc[4 * g + 3]);
          }
        }
      }
#pragma unroll
      for (int a = 0; a < NA; ++a) acc64[a] += (double)acc[a];
    }
    __syncthreads();                              // the stage is refilled by the next issue
  }
  if (own) {
    double* P = part + ((size_t)blockIdx.x * vmax + vbase + tid) * kRcBlock;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (a < na) P[a] = acc64[a];
  }
}

// out[(row0 + v) * kRcBlock + col0 + a] = sum over the CTAs of part[cta][v][a] (partials of
// vmax x kRcBlock per CTA), for v < nv, a < na: four sums over the CTAs of each residue mod 4, in
// CTA order, then added pairwise.
__global__ void rcss_reduce_kernel(const double* __restrict__ part, int nblk, int nv, int na, int vmax,
                                   double* __restrict__ out, int row0, int col0) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nv * na) return;
  const int v = idx / na, a = idx - v * na;
  double s[4] = {0.0, 0.0, 0.0, 0.0};             // CTAs b = 0, 1, 2, 3 mod 4, then added in order
  int b = 0;
  for (; b + 3 < nblk; b += 4)
#pragma unroll
    for (int u = 0; u < 4; ++u) s[u] += part[((size_t)(b + u) * vmax + v) * kRcBlock + a];
  for (; b < nblk; ++b) s[b & 3] += part[((size_t)b * vmax + v) * kRcBlock + a];
  out[(size_t)(row0 + v) * kRcBlock + col0 + a] = (s[0] + s[1]) + (s[2] + s[3]);
}

// Thin products: part[v][cta] = V_v . x over this CTA's coordinate range, for v < nv.  The range
// is cut into chunks of kGvChunk coordinates; each chunk of x is staged in shared memory once and
// warp w sums V_v . x over it for v = w, w + 8, ... (8 loads in flight per lane, lane sums in the
// data's type), a butterfly adds the lanes' sums in FP64, and the chunk's sum joins the FP64
// partial of (v, cta), which only lane 0 of that warp touches.
constexpr int kGvChunk = 4096;

template <typename T>
__global__ void __launch_bounds__(kRcThreads)
rcss_gemv_kernel(const T* const* __restrict__ V, int nv, const T* __restrict__ x, int64_t m, int64_t per_cta,
                 double* __restrict__ part) {
  __shared__ T xs[kGvChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = gridDim.x;
  const int64_t c_begin = (int64_t)blockIdx.x * per_cta;
  const int64_t c_end = c_begin + per_cta < m ? c_begin + per_cta : m;
  for (int v = warp; v < nv; v += kRcThreads / 32)
    if (lane == 0) part[(size_t)v * nblk + blockIdx.x] = 0.0;
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kGvChunk) {
    const int len = (int)(c_end - c0 < kGvChunk ? c_end - c0 : kGvChunk);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += kRcThreads) xs[i] = x[c0 + i];
    __syncthreads();
    for (int v = warp; v < nv; v += kRcThreads / 32) {
      const T* col = V[v] + c0;
      T sum = T(0);
      int i = lane;
      for (; i + 7 * 32 < len; i += 8 * 32) {
        T a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = col[i + 32 * u];
#pragma unroll
        for (int u = 0; u < 8; ++u) sum = fma(a[u], xs[i + 32 * u], sum);
      }
      for (; i < len; i += 32) sum = fma(col[i], xs[i], sum);
      double ds = (double)sum;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xFFFFFFFFu, ds, off);
      if (lane == 0) part[(size_t)v * nblk + blockIdx.x] += ds;
    }
  }
}

// out[v * ostride] = sum over the CTAs of part[v][cta] (nblk per v), v < nv: one warp per v, lane l
// adding the CTAs l, l + 32, ... in order, then a butterfly.
__global__ void rcss_gemv_reduce_kernel(const double* __restrict__ part, int nblk, int nv,
                                        double* __restrict__ out, int ostride) {
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)v * nblk + b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) out[(size_t)v * ostride] = s;
}

// ||A_a||^2 over this CTA's coordinate range (the thin products' partition): every thread sums
// its coordinates (8 loads in flight) in the data's type, the warps add their lanes in FP64 and
// thread 0 adds the 8 warps in order into part[a][cta].
template <typename T>
__global__ void __launch_bounds__(kRcThreads)
rcss_norms_kernel(const T* const* __restrict__ A, int na, int64_t m, int64_t per_cta, double* __restrict__ part) {
  __shared__ double red[kRcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t c_begin = (int64_t)blockIdx.x * per_cta;
  const int64_t c_end = c_begin + per_cta < m ? c_begin + per_cta : m;
  for (int a = 0; a < na; ++a) {
    const T* col = A[a];
    T sum = T(0);
    int64_t i = c_begin + tid;
    for (; i + 7 * kRcThreads < c_end; i += 8 * kRcThreads) {
      T x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = col[i + kRcThreads * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) sum = fma(x[u], x[u], sum);
    }
    for (; i < c_end; i += kRcThreads) sum = fma(col[i], col[i], sum);
    double ds = (double)sum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(0xFFFFFFFFu, ds, off);
    if (lane == 0) red[warp] = ds;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kRcThreads / 32; ++w) t += red[w];
      part[(size_t)a * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// Algorithm 1's decisions for the block's columns q0 .. nb - 1 (one thread, FP64).  X[i][q] holds
// the dot of basis vector i < nq with block column q, nrm[q] = ||a_q||^2.
__global__ void rcss_decide_kernel(const double* __restrict__ X, const double* __restrict__ nrm, int nq, int q0,
                                   int nb, int k, double xi, uint64_t seed, int cap, int stop_at_cap, int ncur0,
                                   RcssDevState* st, int64_t* sel, RcssRec* rec, double* pout) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  rec->stop = nb - 1;
  rec->step_end = 0;
  rec->nkeep = 0;
  rec->overflow = 0;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int q = q0; q < nb; ++q) {
    double proj = 0.0;
    for (int i = 0; i < nq; ++i) {
      const double c = X[(size_t)i * kRcBlock + q];
      proj = fma(c, c, proj);
    }
    double res = nrm[q] - proj;
    if (res < 0.0) res = 0.0;
    const double p = (double)k * res / xi;
    const int64_t j = st->n_obs;
    pout[q] = p;
    const u32x4 w = philox4x32_10((uint32_t)(j & 0xFFFFFFFFu), (uint32_t)(j >> 32), kTagRcss, 0, k0, k1);
    const double u = uniform53(w.x, w.y);
    if (u < (p < 1.0 ? p : 1.0)) {
      if (st->nsel >= cap || ncur0 + rec->nkeep >= cap) {
        if (!stop_at_cap) {
          rec->overflow = 1;
          rec->stop = q - 1;                  // column q is left undecided
          return;
        }
      } else {
        sel[st->nsel++] = j;
        rec->keep[rec->nkeep++] = q;
      }
    }
    if (p < 1.0) st->sigma += p;
    st->n_obs = j + 1;
    if (p >= 1.0 || st->sigma >= 1.0) {
      st->sigma = 0.0;
      rec->stop = q;
      rec->step_end = 1;
      return;
    }
  }
}

// v = c - Q coef (coef: FP64 dots, nq of them, coef[t * cstride], rounded to the data's type and
// staged in shared memory); v may be c.  Arithmetic in the data's type, 4 basis loads in flight.
constexpr int kAxMaxCoef = 4096;

template <typename T>
__global__ void __launch_bounds__(256)
rcss_axpy_kernel(const T* __restrict__ Q, int64_t ldq, int nq, const double* __restrict__ coef, int cstride,
                 const T* c, T* v, int64_t m) {
  __shared__ T cs[kAxMaxCoef];
  for (int t = threadIdx.x; t < nq; t += blockDim.x) cs[t] = (T)coef[(size_t)t * cstride];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    T s = c[i];
    int t = 0;
    for (; t + 3 < nq; t += 4) {
      T q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = Q[(size_t)(t + u) * ldq + i];
#pragma unroll
      for (int u = 0; u < 4; ++u) s = fma(-cs[t + u], q[u], s);
    }
    for (; t < nq; ++t) s = fma(-cs[t], Q[(size_t)t * ldq + i], s);
    v[i] = s;
  }
}

// Normalize v in place if ||v|| > tol ||c||; flag[0] = 1 when it does (a new basis direction).
template <typename T>
__global__ void rcss_scale_kernel(T* __restrict__ v, int64_t m, const double* __restrict__ vv,
                                  const double* __restrict__ cc, double tol, int* __restrict__ flag) {
  const double nv = sqrt(vv[0]), nc = sqrt(cc[0]);
  const bool add = nv > tol * nc && nv > 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = add ? 1 : 0;
  if (!add) return;
  const double s = 1.0 / nv;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (T)((double)v[i] * s);
}

}  // namespace
}  // namespace rid

struct rid_rcss {
  int64_t m, m_pad;
  int k;
  double xi;
  uint64_t seed;
  int dtype;                  // RID_F64 or RID_F32
  size_t es;
  int cap;                    // selection capacity (and basis capacity)
  int stop_at_cap;
  cudaStream_t st;
  int n_sm, nblk;
  int vmax;                   // vectors in one product: max(cap + 1, kRcBlock)
  int64_t runs_per_cta;
  void* Q;                    // cap x m_pad: the orthonormal basis, then one candidate slot
  void* C;                    // cap x m_pad: raw columns of C_cur
  void* stage;                // kRcBlock x m_pad: host columns (allocated at the first host ingest)
  const void** vptr;          // device pointer arrays for the dot pass: V (vmax), A (kRcBlock)
  const void** aptr;
  double* part;               // nblk x vmax x kRcBlock: per-CTA partial dots
  double* partn;              // kRcBlock x gblk: per-CTA partial norms
  double* partg;              // vmax x gblk: per-CTA partial thin products
  int gblk;                   // CTAs of a thin product
  int64_t g_per_cta;          // coordinates per CTA of a thin product (a multiple of kGvChunk)
  double* X;                  // cap x kRcBlock: basis x block-column dots of the current block
  double* Xe;                 // vmax x kRcBlock: dots of the extension step
  double* nrm;                // kRcBlock: squared norms of the current block's columns
  double* pv;                 // kRcBlock: p of the block's columns
  rid::RcssDevState* dst;
  rid::RcssRec* drec;
  rid::RcssRec* hrec;         // pinned
  int64_t* sel;
  int* dflag;
  int* hflag;                 // pinned
  double* hp_stage;           // pinned, kRcBlock
  int nq, ncur;               // host mirrors of the basis size and of C_cur's size
  std::vector<double> hp;     // p of every column so far (copied after each pass)
};

namespace rid {

void rcss_selection_view(const rid_rcss* g, const int64_t** sel, const int** nsel, int64_t* m, int* cap,
                         int* stop_at_cap, int* dtype, cudaStream_t* st) {
  *sel = g->sel;
  *nsel = &g->dst->nsel;
  *m = g->m;
  *cap = g->cap;
  *stop_at_cap = g->stop_at_cap;
  *dtype = g->dtype;
  *st = g->st;
}

}  // namespace rid

namespace {

int rc_fail(int code, const std::string& msg) {
  rid::set_global_error(msg.c_str());
  return code;
}

#define RCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return rc_fail(e_ == cudaErrorMemoryAllocation ? RID_ENOMEM : RID_ECUDA,                      \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

char* qcol(rid_rcss* h, int t) { return (char*)h->Q + (size_t)t * h->m_pad * h->es; }
char* ccol(rid_rcss* h, int t) { return (char*)h->C + (size_t)t * h->m_pad * h->es; }

// out[(row0 + v) * kRcBlock + col0 + a] = V_v . A_a (nv <= vmax vectors, na <= kRcBlock columns).
int rc_dots(rid_rcss* h, const std::vector<const void*>& V, const std::vector<const void*>& A, double* out,
            int row0, int col0) {
  const int nv = (int)V.size(), na = (int)A.size();
  if (nv == 0 || na == 0) return RID_OK;
  if (nv > h->vmax || na > rid::kRcBlock || col0 + na > rid::kRcBlock)
    return rc_fail(RID_EINVAL, "rcss: too many vectors in one dot pass");
  RCK(cudaMemcpyAsync(h->vptr, V.data(), sizeof(void*) * nv, cudaMemcpyHostToDevice, h->st));
  RCK(cudaMemcpyAsync(h->aptr, A.data(), sizeof(void*) * na, cudaMemcpyHostToDevice, h->st));
  bool aligned = true;
  for (const void* p : V) aligned = aligned && ((uintptr_t)p % 16 == 0);
  if (na <= 16 && aligned && h->dtype == RID_F32) {
    const int na_t = na <= 4 ? 4 : na <= 8 ? 8 : 16;
    const size_t smem = sizeof(float) * (2 * (size_t)rid::kStTile * rid::kStLd + 2 * (size_t)rid::kRcRun * na_t);
    const dim3 grid(h->nblk, (nv + rid::kStTile - 1) / rid::kStTile);
#define RC_STAGE(NA)                                                                                              \
  rid::rcss_thin_stage_kernel<NA><<<grid, rid::kStTile, smem, h->st>>>(                                          \
      reinterpret_cast<const float* const*>(h->vptr), nv, reinterpret_cast<const float* const*>(h->aptr), na,   \
      h->m, h->runs_per_cta, h->vmax, h->part)
    if (na_t == 4) RC_STAGE(4); else if (na_t == 8) RC_STAGE(8); else RC_STAGE(16);
#undef RC_STAGE
    rid::rcss_reduce_kernel<<<(nv * na + 255) / 256, 256, 0, h->st>>>(h->part, h->nblk, nv, na, h->vmax, out, row0,
                                                                     col0);
    RCK(cudaGetLastError());
    return RID_OK;
  }
  if (na <= 16 && aligned) {
    const int na_t = na <= 4 ? 4 : na <= 8 ? 8 : 16;
    const size_t smem = h->es * (size_t)rid::kThinRuns * rid::kRcRun * na_t;
    const dim3 grid(h->nblk, (nv + rid::kRcThreads - 1) / rid::kRcThreads);
#define RC_THIN(TT, NA)                                                                                           \
  rid::rcss_thin_kernel<TT, NA><<<grid, rid::kRcThreads, smem, h->st>>>(                                         \
      reinterpret_cast<const TT* const*>(h->vptr), nv, reinterpret_cast<const TT* const*>(h->aptr), na, h->m,     \
      h->runs_per_cta, h->vmax, h->part)
    if (h->dtype == RID_F64) {
      if (na_t == 4) RC_THIN(double, 4); else if (na_t == 8) RC_THIN(double, 8); else RC_THIN(double, 16);
    } else {
      if (na_t == 4) RC_THIN(float, 4); else if (na_t == 8) RC_THIN(float, 8); else RC_THIN(float, 16);
    }
#undef RC_THIN
    rid::rcss_reduce_kernel<<<(nv * na + 255) / 256, 256, 0, h->st>>>(h->part, h->nblk, nv, na, h->vmax, out, row0,
                                                                     col0);
    RCK(cudaGetLastError());
    return RID_OK;
  }
  const size_t smem = h->es * 2 * (size_t)rid::kRcRun * rid::kRcLd;
  if (h->dtype == RID_F64)
    rid::rcss_dots_kernel<double><<<h->nblk, rid::kRcThreads, smem, h->st>>>(
        reinterpret_cast<const double* const*>(h->vptr), nv, reinterpret_cast<const double* const*>(h->aptr), na,
        h->m, h->runs_per_cta, h->vmax, h->part);
  else
    rid::rcss_dots_kernel<float><<<h->nblk, rid::kRcThreads, smem, h->st>>>(
        reinterpret_cast<const float* const*>(h->vptr), nv, reinterpret_cast<const float* const*>(h->aptr), na,
        h->m, h->runs_per_cta, h->vmax, h->part);
  rid::rcss_reduce_kernel<<<(nv * na + 255) / 256, 256, 0, h->st>>>(h->part, h->nblk, nv, na, h->vmax, out, row0,
                                                                   col0);
  RCK(cudaGetLastError());
  return RID_OK;
}

// out[a] = ||A_a||^2 for a < na (na <= kRcBlock).
int rc_norms(rid_rcss* h, const std::vector<const void*>& A, double* out) {
  const int na = (int)A.size();
  if (na == 0) return RID_OK;
  RCK(cudaMemcpyAsync(h->aptr, A.data(), sizeof(void*) * na, cudaMemcpyHostToDevice, h->st));
  if (h->dtype == RID_F64)
    rid::rcss_norms_kernel<double><<<h->gblk, rid::kRcThreads, 0, h->st>>>(
        reinterpret_cast<const double* const*>(h->aptr), na, h->m, h->g_per_cta, h->partn);
  else
    rid::rcss_norms_kernel<float><<<h->gblk, rid::kRcThreads, 0, h->st>>>(
        reinterpret_cast<const float* const*>(h->aptr), na, h->m, h->g_per_cta, h->partn);
  rid::rcss_gemv_reduce_kernel<<<(na + 7) / 8, 256, 0, h->st>>>(h->partn, h->gblk, na, out, 1);
  RCK(cudaGetLastError());
  return RID_OK;
}

// out[v * ostride] = V_v . x (nv <= vmax vectors).
int rc_gemv(rid_rcss* h, const std::vector<const void*>& V, const void* x, double* out, int ostride) {
  const int nv = (int)V.size();
  if (nv == 0) return RID_OK;
  if (nv > h->vmax) return rc_fail(RID_EINVAL, "rcss: too many vectors in one product");
  RCK(cudaMemcpyAsync(h->vptr, V.data(), sizeof(void*) * nv, cudaMemcpyHostToDevice, h->st));
  if (h->dtype == RID_F64)
    rid::rcss_gemv_kernel<double><<<h->gblk, rid::kRcThreads, 0, h->st>>>(
        reinterpret_cast<const double* const*>(h->vptr), nv, (const double*)x, h->m, h->g_per_cta, h->partg);
  else
    rid::rcss_gemv_kernel<float><<<h->gblk, rid::kRcThreads, 0, h->st>>>(
        reinterpret_cast<const float* const*>(h->vptr), nv, (const float*)x, h->m, h->g_per_cta, h->partg);
  rid::rcss_gemv_reduce_kernel<<<(nv + 7) / 8, 256, 0, h->st>>>(h->partg, h->gblk, nv, out, ostride);
  RCK(cudaGetLastError());
  return RID_OK;
}

// Extend Q by the C_cur columns, in order (two rounds of Gram-Schmidt each), then empty C_cur.
int rc_extend(rid_rcss* h) {
  const double tol = h->dtype == RID_F64 ? 1e-12 : 1e-4;
  const int grid = 4 * h->n_sm;
  for (int t = 0; t < h->ncur; ++t) {
    if (h->nq >= h->cap) return rc_fail(RID_EINVAL, "rcss: basis capacity exceeded");
    const void* c = ccol(h, t);
    void* v = qcol(h, h->nq);                     // the candidate direction, in the next basis slot
    std::vector<const void*> V;
    for (int i = 0; i < h->nq; ++i) V.push_back(qcol(h, i));
    const void* src = c;
    for (int round = 0; round < 2; ++round) {
      if (h->nq > 0) {
        int rc = rc_gemv(h, V, src, h->Xe, rid::kRcBlock);   // coefficients Xe[i * kRcBlock], i < nq
        if (rc != RID_OK) return rc;
        if (h->dtype == RID_F64)
          rid::rcss_axpy_kernel<double><<<grid, 256, 0, h->st>>>((const double*)h->Q, h->m_pad, h->nq, h->Xe,
                                                                 rid::kRcBlock, (const double*)src, (double*)v, h->m);
        else
          rid::rcss_axpy_kernel<float><<<grid, 256, 0, h->st>>>((const float*)h->Q, h->m_pad, h->nq, h->Xe,
                                                                rid::kRcBlock, (const float*)src, (float*)v, h->m);
      } else if (round == 0) {
        RCK(cudaMemcpyAsync(v, c, h->es * (size_t)h->m, cudaMemcpyDeviceToDevice, h->st));
      }
      src = v;
    }
    int rc = rc_norms(h, {v, c}, h->Xe);          // Xe[0] = ||v||^2, Xe[1] = ||c||^2
    if (rc != RID_OK) return rc;
    if (h->dtype == RID_F64)
      rid::rcss_scale_kernel<double><<<grid, 256, 0, h->st>>>((double*)v, h->m, h->Xe, h->Xe + 1, tol, h->dflag);
    else
      rid::rcss_scale_kernel<float><<<grid, 256, 0, h->st>>>((float*)v, h->m, h->Xe, h->Xe + 1, tol, h->dflag);
    RCK(cudaMemcpyAsync(h->hflag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    RCK(cudaStreamSynchronize(h->st));
    if (h->hflag[0]) ++h->nq;                     // else the slot is reused by the next candidate
  }
  h->ncur = 0;
  return RID_OK;
}

// One block of at most kRcBlock device columns.
int rc_block(rid_rcss* h, const void* const* cols, int nb) {
  std::vector<const void*> A(cols, cols + nb), V;
  int rc = rc_norms(h, A, h->nrm);
  if (rc != RID_OK) return rc;
  for (int i = 0; i < h->nq; ++i) V.push_back(qcol(h, i));
  rc = rc_dots(h, V, A, h->X, 0, 0);
  if (rc != RID_OK) return rc;
  int q0 = 0;
  while (q0 < nb) {
    rid::rcss_decide_kernel<<<1, 32, 0, h->st>>>(h->X, h->nrm, h->nq, q0, nb, h->k, h->xi, h->seed, h->cap,
                                                 h->stop_at_cap, h->ncur, h->dst, h->sel, h->drec, h->pv);
    RCK(cudaGetLastError());
    RCK(cudaMemcpyAsync(h->hrec, h->drec, sizeof(rid::RcssRec), cudaMemcpyDeviceToHost, h->st));
    RCK(cudaMemcpyAsync(h->hp_stage, h->pv, sizeof(double) * nb, cudaMemcpyDeviceToHost, h->st));
    RCK(cudaStreamSynchronize(h->st));
    const rid::RcssRec r = *h->hrec;
    for (int q = q0; q <= r.stop; ++q) h->hp.push_back(h->hp_stage[q]);   // the decided columns
    if (r.overflow) return rc_fail(RID_EINVAL, "rcss: selection capacity exceeded (raise cap)");
    for (int i = 0; i < r.nkeep; ++i) {
      RCK(cudaMemcpyAsync(ccol(h, h->ncur), cols[r.keep[i]], h->es * (size_t)h->m, cudaMemcpyDeviceToDevice, h->st));
      ++h->ncur;
    }
    q0 = r.stop + 1;
    if (r.step_end) {
      const int nq0 = h->nq;
      rc = rc_extend(h);
      if (rc != RID_OK) return rc;
      if (q0 < nb) {                              // dots of the new basis vectors with the rest
        std::vector<const void*> An(cols + q0, cols + nb);
        for (int i = nq0; i < h->nq; ++i) {
          rc = rc_gemv(h, An, qcol(h, i), h->X + (size_t)i * rid::kRcBlock + q0, 1);
          if (rc != RID_OK) return rc;
        }
      }
    }
  }
  return RID_OK;
}

}  // namespace

extern "C" {

int rid_rcss_init(rid_rcss** out, int64_t m, int32_t k, double xi, uint64_t seed, int32_t data_dtype, int32_t cap,
                  int32_t stop_at_cap, void* cuda_stream) {
  if (!out) return rc_fail(RID_EINVAL, "rcss: NULL argument");
  *out = nullptr;
  if (m < 1 || k < 1 || !(xi > 0.0) || cap < 1 || cap > rid::kRcMaxCap ||
      (data_dtype != RID_F64 && data_dtype != RID_F32))
    return rc_fail(RID_EINVAL, "rcss: need m >= 1, k >= 1, xi > 0, 1 <= cap <= 4096, dtype F32 or F64");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return rc_fail(RID_ENOLIB, "no CUDA device");
  }
  rid_rcss* h = new rid_rcss();
  h->m = m;
  h->m_pad = (m + rid::kRcRun - 1) / rid::kRcRun * rid::kRcRun;
  h->k = k;
  h->xi = xi;
  h->seed = seed;
  h->dtype = data_dtype;
  h->es = data_dtype == RID_F64 ? 8 : 4;
  h->cap = cap;
  h->stop_at_cap = stop_at_cap ? 1 : 0;
  h->st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nruns = (m + rid::kRcRun - 1) / rid::kRcRun;
  const int64_t per_sm = data_dtype == RID_F32 ? 3 : 1;    // dots CTAs resident per SM (shared memory)
  h->nblk = (int)(nruns < per_sm * h->n_sm ? nruns : per_sm * h->n_sm);
  h->runs_per_cta = (nruns + h->nblk - 1) / h->nblk;
  h->vmax = cap + 1 > rid::kRcBlock ? cap + 1 : rid::kRcBlock;
  {
    const int64_t chunks = (m + rid::kGvChunk - 1) / rid::kGvChunk;
    const int64_t want = 4 * (int64_t)h->n_sm;
    h->gblk = (int)(chunks < want ? chunks : want);
    h->g_per_cta = (chunks + h->gblk - 1) / h->gblk * rid::kGvChunk;
  }
  bool ok = true;
  auto al = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  al(&h->Q, (size_t)(cap + 1) * h->m_pad * h->es);
  al(&h->C, (size_t)cap * h->m_pad * h->es);
  al((void**)&h->vptr, sizeof(void*) * h->vmax);
  al((void**)&h->aptr, sizeof(void*) * rid::kRcBlock);
  al((void**)&h->part, sizeof(double) * (size_t)h->nblk * h->vmax * rid::kRcBlock);
  al((void**)&h->partn, sizeof(double) * (size_t)h->gblk * rid::kRcBlock);
  al((void**)&h->partg, sizeof(double) * (size_t)h->gblk * h->vmax);
  al((void**)&h->X, sizeof(double) * (size_t)cap * rid::kRcBlock);
  al((void**)&h->Xe, sizeof(double) * (size_t)h->vmax * rid::kRcBlock);
  al((void**)&h->nrm, sizeof(double) * rid::kRcBlock);
  al((void**)&h->pv, sizeof(double) * rid::kRcBlock);
  al((void**)&h->dst, sizeof(rid::RcssDevState));
  al((void**)&h->drec, sizeof(rid::RcssRec));
  al((void**)&h->sel, sizeof(int64_t) * (size_t)cap);
  al((void**)&h->dflag, sizeof(int));
  if (ok && (cudaMallocHost((void**)&h->hrec, sizeof(rid::RcssRec)) != cudaSuccess ||
             cudaMallocHost((void**)&h->hflag, sizeof(int)) != cudaSuccess ||
             cudaMallocHost((void**)&h->hp_stage, sizeof(double) * rid::kRcBlock) != cudaSuccess))
    ok = false;
  if (!ok) {
    cudaGetLastError();
    rid_rcss_destroy(h);
    return rc_fail(RID_ENOMEM, "rcss: device allocation failed");
  }
  {
    const int s64 = 8 * 2 * rid::kRcRun * rid::kRcLd;
    const int s32 = 4 * 2 * rid::kRcRun * rid::kRcLd;
    const int t64 = 8 * rid::kThinRuns * rid::kRcRun * 16;
    ok = cudaFuncSetAttribute(rid::rcss_dots_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64) ==
             cudaSuccess &&
         cudaFuncSetAttribute(rid::rcss_dots_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32) ==
             cudaSuccess &&
         cudaFuncSetAttribute(rid::rcss_thin_kernel<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, t64) ==
             cudaSuccess;
    for (int na_t : {4, 8, 16}) {
      const int st = (int)sizeof(float) * (2 * rid::kStTile * rid::kStLd + 2 * rid::kRcRun * na_t);
      const void* f = na_t == 4 ? (const void*)rid::rcss_thin_stage_kernel<4>
                      : na_t == 8 ? (const void*)rid::rcss_thin_stage_kernel<8>
                                  : (const void*)rid::rcss_thin_stage_kernel<16>;
      ok = ok && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, st) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      rid_rcss_destroy(h);
      return rc_fail(RID_ECUDA, "rcss: kernel shared-memory attributes refused");
    }
  }
  {
    ok = cudaMemsetAsync(h->Q, 0, (size_t)(cap + 1) * h->m_pad * h->es, h->st) == cudaSuccess &&
         cudaMemsetAsync(h->dst, 0, sizeof(rid::RcssDevState), h->st) == cudaSuccess &&
         cudaMemsetAsync(h->sel, 0xFF, sizeof(int64_t) * (size_t)cap, h->st) == cudaSuccess &&   // -1
         cudaStreamSynchronize(h->st) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    rid_rcss_destroy(h);
    return rc_fail(RID_ECUDA, "rcss: device initialization failed");
  }
  *out = h;
  return RID_OK;
}

int rid_rcss_ingest(rid_rcss* h, const void* cols, int64_t ld, int32_t ncols, int32_t on_device) {
  if (!h || (!cols && ncols > 0) || ncols < 0 || ld < h->m) return rc_fail(RID_EINVAL, "rcss: bad argument");
  if (!on_device && ncols > 0 && !h->stage) {
    if (cudaMalloc(&h->stage, (size_t)rid::kRcBlock * h->m_pad * h->es) != cudaSuccess) {
      cudaGetLastError();
      h->stage = nullptr;
      return rc_fail(RID_ENOMEM, "rcss: staging allocation failed");
    }
  }
  for (int32_t q0 = 0; q0 < ncols; q0 += rid::kRcBlock) {
    const int nb = ncols - q0 < rid::kRcBlock ? ncols - q0 : rid::kRcBlock;
    std::vector<const void*> ptrs((size_t)nb);
    for (int q = 0; q < nb; ++q) {
      const char* src = (const char*)cols + (size_t)(q0 + q) * ld * h->es;
      if (on_device) {
        ptrs[q] = src;
      } else {
        char* dst = (char*)h->stage + (size_t)q * h->m_pad * h->es;
        RCK(cudaMemcpyAsync(dst, src, (size_t)h->m * h->es, cudaMemcpyHostToDevice, h->st));
        ptrs[q] = dst;
      }
    }
    const int rc = rc_block(h, ptrs.data(), nb);
    if (rc != RID_OK) return rc;
  }
  return RID_OK;
}

int rid_rcss_selection(rid_rcss* h, int64_t* idx, int32_t max_out, int32_t* n_out, double* sigma,
                       int32_t* basis_size) {
  if (!h) return rc_fail(RID_EINVAL, "rcss: NULL handle");
  rid::RcssDevState s;
  RCK(cudaMemcpyAsync(&s, h->dst, sizeof(s), cudaMemcpyDeviceToHost, h->st));
  RCK(cudaStreamSynchronize(h->st));
  if (n_out) *n_out = s.nsel;
  if (sigma) *sigma = s.sigma;
  if (basis_size) *basis_size = h->nq;
  if (idx && max_out > 0) {
    const int n = s.nsel < max_out ? s.nsel : max_out;
    if (n > 0) {
      RCK(cudaMemcpyAsync(idx, h->sel, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, h->st));
      RCK(cudaStreamSynchronize(h->st));
    }
  }
  return RID_OK;
}

int rid_rcss_probabilities(rid_rcss* h, double* p, int64_t max_out, int64_t* n_out) {
  if (!h) return rc_fail(RID_EINVAL, "rcss: NULL handle");
  const int64_t n = (int64_t)h->hp.size();
  if (n_out) *n_out = n;
  if (p && max_out > 0) memcpy(p, h->hp.data(), sizeof(double) * (size_t)(n < max_out ? n : max_out));
  return RID_OK;
}

int rid_rcss_basis(rid_rcss* h, void* out, int64_t ld, int32_t on_device) {
  if (!h || !out || ld < h->m) return rc_fail(RID_EINVAL, "rcss: bad argument");
  if (h->nq == 0) return RID_OK;
  RCK(cudaMemcpy2DAsync(out, h->es * (size_t)ld, h->Q, h->es * (size_t)h->m_pad, h->es * (size_t)h->m, h->nq,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  RCK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_rcss_destroy(rid_rcss* h) {
  if (!h) return RID_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  void* ptrs[] = {h->Q, h->C, h->stage, (void*)h->vptr, (void*)h->aptr, h->part, h->partn, h->partg, h->X, h->Xe, h->nrm,
                  h->pv, h->dst, h->drec, h->sel, h->dflag};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->hrec) cudaFreeHost(h->hrec);
  if (h->hflag) cudaFreeHost(h->hflag);
  if (h->hp_stage) cudaFreeHost(h->hp_stage);
  delete h;
  return RID_OK;
}

}  // extern "C"
