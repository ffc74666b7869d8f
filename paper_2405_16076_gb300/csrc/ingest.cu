// Ingest path of Algorithm 3: for a block of nb columns, one read of each
// column produces (i) the copy into its buffer slot d_count, (ii) the squared
// norms for ||A_obs||_F^2 and (iii) the sketch s_j = Omega a_j for all s left
// rows and h probe rows, with Omega generated on chip from the counter-based
// generator (Rademacher) or read from its materialized transpose (Gaussian).
// A deterministic split-K reduction then appends the sketches to S and
// updates SS^T and ||A_obs||^2 in column order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "rid.h"
#include "rid_internal.cuh"

namespace rid {

template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

__device__ __forceinline__ double flip_sign(double x, uint32_t bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((unsigned long long)bit << 63));
}
__device__ __forceinline__ float flip_sign(float x, uint32_t bit) {
  return __int_as_float(__float_as_int(x) ^ (bit << 31));
}

// grid: (n_sketch_blocks, ceil(rows/256)); block: 256 threads.
// Thread tid of row-group y owns sketch row r = 256*y + tid.
struct SimtCols {
  const void* p[kMaxB];
};

template <typename T, int NB>
__global__ void __launch_bounds__(kSketchThreads)
ingest_sketch_kernel(Dev d, SimtCols cols, int nb, int count) {
  __shared__ T X[NB][kChunk];
  __shared__ int dst[NB];
  __shared__ double red[kSketchThreads / 32][NB];
  const int tid = threadIdx.x;
  const int r = blockIdx.y * kSketchThreads + tid;
  const bool row_ok = r < d.rows;
  const bool lead = blockIdx.y == 0;
  if (tid < NB) dst[tid] = (tid < nb) ? d.dslot[count + tid] : 0;
  __syncthreads();
  T* pool = (T*)d.pool;
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);

  double acc64[NB];
  T acc[NB];
  double nrm[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) { acc64[q] = 0.0; acc[q] = T(0); nrm[q] = 0.0; }

  const int64_t nchunks = (d.m + kChunk - 1) / kChunk;
  int since_flush = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t i0 = c * kChunk;
    const int64_t i = i0 + tid;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (q < nb) {
        T v = T(0);
        if (i < d.m) {
          v = ((const T*)cols.p[q])[i];
          if (lead) pool[(int64_t)dst[q] * d.m_pad + i] = v;
        }
        X[q][tid] = v;
        nrm[q] += (double)v * (double)v;
      }
    }
    __syncthreads();
    if (row_ok) {
      if (d.omega_kind == 1) {
        // Rademacher: 2 Philox calls cover the 256 coordinates of the chunk
#pragma unroll 1
        for (int half = 0; half < kChunk / 128; ++half) {
          const uint32_t blk = (uint32_t)(((i0 + d.row_offset) >> 7) + half);   // global row
          const u32x4 w = philox4x32_10(blk, (uint32_t)r, kTagRademacher, 0, k0, k1);
          const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int wi = 0; wi < 4; ++wi) {
            const uint32_t bits = words[wi];
#pragma unroll 8
            for (int e = 0; e < 32; ++e) {
              // coordinate pair p = e/2 takes bit 15-p (even e) or 31-p (odd e) of the word
              const int bpos = (e & 1) ? 31 - (e >> 1) : 15 - (e >> 1);
              const uint32_t bit = (bits >> bpos) & 1u;
              const int ii = half * 128 + wi * 32 + e;
#pragma unroll
              for (int q = 0; q < NB; ++q)
                if (q < nb) acc[q] += flip_sign(X[q][ii], bit);
            }
          }
        }
      } else {
        const double* om = d.omegaT + (size_t)i0 * d.rows + r;
#pragma unroll 4
        for (int ii = 0; ii < kChunk; ++ii) {
          if (i0 + ii >= d.m) break;
          const T w = (T)om[(size_t)ii * d.rows];
#pragma unroll
          for (int q = 0; q < NB; ++q)
            if (q < nb) acc[q] += w * X[q][ii];
        }
      }
    }
    if (++since_flush == 4) {
#pragma unroll
      for (int q = 0; q < NB; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      since_flush = 0;
    }
    __syncthreads();
  }
  if (row_ok) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < nb)
        d.spart[((size_t)blockIdx.x * nb + q) * d.rows + r] = acc64[q] + (double)acc[q];
  }
  if (lead) {
    // deterministic block reduction of the squared norms
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      double v = nrm[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (tid < nb) {
      double v = 0.0;
      for (int w = 0; w < kSketchThreads / 32; ++w) v += red[w][tid];
      d.npart[(size_t)blockIdx.x * nb + tid] = v;
    }
  }
}

// One thread per (q, r): sum the split-K partials in block order, append S(:, n_obs+q).
__global__ void sketch_reduce_kernel(Dev d, int nb, int64_t n_obs, int nblk) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nb * d.rows) {
    const int q = idx / d.rows, r = idx % d.rows;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += d.spart[((size_t)b * nb + q) * d.rows + r];
    d.S[(size_t)(n_obs + q) * d.rows + r] = v;
  }
  if (idx == 0) {
    for (int q = 0; q < nb; ++q) {
      double v = 0.0;
      for (int b = 0; b < nblk; ++b) v += d.npart[(size_t)b * nb + q];
      if (d.gnorm) {                        // row shard: summed over the shards first
        d.gnorm[q] = v;
        continue;
      }
      if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
      d.fro2[0] += v;
      d.fro2[1] += v;
    }
  }
}

// Row sharding: the group's squared norms, summed over the shards, into ||A_obs||^2 (column order).
__global__ void add_norms_kernel(Dev d, int nb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < nb; ++q) {
    const double v = d.gnorm[q];
    if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
    d.fro2[0] += v;
    d.fro2[1] += v;
  }
}

int shard_exchange_sketch(const Dev& d, int ncols, int64_t n_obs, cudaStream_t st) {
  const rid_allreduce_fn f = (rid_allreduce_fn)d.allreduce;
  if (f(d.S + (size_t)n_obs * d.rows, (int64_t)ncols * d.rows, (void*)st, d.allreduce_user) != 0) return -1;
  if (f(d.gnorm, ncols, (void*)st, d.allreduce_user) != 0) return -1;
  add_norms_kernel<<<1, 32, 0, st>>>(d, ncols);
  return 0;
}

// SS^T += sum_q l_q l_q^T over the new leverage-sketch columns, in column order.
__global__ void gram_update_kernel(Dev d, int nb, int64_t n_obs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = d.s;
  if (idx >= (int64_t)s * s) return;
  const int i = (int)(idx % s), j = (int)(idx / s);
  double v = d.SSt[idx];
  for (int q = 0; q < nb; ++q) {
    const double* l = d.Slev + (size_t)(n_obs + q) * d.lev_ld;
    v += l[i] * l[j];
  }
  d.SSt[idx] = v;
}

__global__ void materialize_omega_kernel(Dev d) {
  const int64_t n = d.m_pad * d.rows;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / d.rows;
    const int r = (int)(idx % d.rows);
    d.omegaT[idx] = (i < d.m) ? gauss_entry(d.seed, kTagGauss, (uint32_t)r, (uint64_t)(i + d.row_offset)) : 0.0;
  }
}

// ---------------------------------------------------------------- gradient mode (Sec. 3.4)
// G a (Eq. 42) by grad_stencil (rid_internal.cuh): the least-squares gradient of Eqs. 39-43 on
// the grid graph, central inside and one-sided at the boundary.
// Omega_g (G a_q) for the s leverage rows and ||G a_q||^2, split-K over the d m gradient
// entries like the ingest sketch (working-precision sums over four chunks, then FP64): grid
// (nblk, ceil(s / 256)), 256 threads, thread tid of row group y owns row r = 256 y + tid;
// partials to d.spart / d.npart.
template <typename T, int NB>
__global__ void __launch_bounds__(kSketchThreads)
grad_sketch_kernel(Dev d, SimtCols cols, int nb) {
  __shared__ T X[NB][kChunk];
  __shared__ double red[kSketchThreads / 32][NB];
  const int tid = threadIdx.x;
  const int r = blockIdx.y * kSketchThreads + tid;
  const bool row_ok = r < d.s;
  const bool lead = blockIdx.y == 0;
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  const int64_t dm = 2 * d.m;
  double acc64[NB], nrm[NB];
  T acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) { acc64[q] = 0.0; acc[q] = T(0); nrm[q] = 0.0; }
  const int64_t nchunks = (dm + kChunk - 1) / kChunk;
  int pending = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t j0 = c * kChunk;
    const int64_t j = j0 + tid;
    if (j < dm) {
      const GradStencil g = grad_stencil(j, d.m, d.nx, d.ny);
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nb) {
          const T* a = (const T*)cols.p[q];
          T v = (T)g.wc * a[g.i];
          if (g.wm != 0.0) v += (T)g.wm * a[g.i - g.st];
          if (g.wp != 0.0) v += (T)g.wp * a[g.i + g.st];
          X[q][tid] = v;
          nrm[q] += (double)v * (double)v;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nb) X[q][tid] = T(0);
    }
    __syncthreads();
    if (row_ok) {
      if (d.omega_kind == 1) {
#pragma unroll 1
        for (int half = 0; half < kChunk / 128; ++half) {
          const u32x4 w = philox4x32_10((uint32_t)((j0 >> 7) + half), (uint32_t)r, kTagGradRademacher, 0, k0, k1);
          const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int wi = 0; wi < 4; ++wi) {
#pragma unroll 8
            for (int e = 0; e < 32; ++e) {
              const int bpos = (e & 1) ? 31 - (e >> 1) : 15 - (e >> 1);
              const uint32_t bit = (words[wi] >> bpos) & 1u;
              const int ii = half * 128 + wi * 32 + e;
#pragma unroll
              for (int q = 0; q < NB; ++q)
                if (q < nb) acc[q] += flip_sign(X[q][ii], bit);
            }
          }
        }
      } else {
#pragma unroll 1
        for (int ii = 0; ii < kChunk; ++ii) {
          if (j0 + ii >= dm) break;
          const T w = (T)gauss_entry(d.seed, kTagGradGauss, (uint32_t)r, (uint64_t)(j0 + ii));
#pragma unroll
          for (int q = 0; q < NB; ++q)
            if (q < nb) acc[q] += w * X[q][ii];
        }
      }
    }
    if (++pending == 4) {
#pragma unroll
      for (int q = 0; q < NB; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      pending = 0;
    }
    __syncthreads();
  }
  if (row_ok) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < nb) d.spart[((size_t)blockIdx.x * nb + q) * d.rows + r] = acc64[q] + (double)acc[q];
  }
  if (lead) {
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      double v = nrm[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (tid < nb) {
      double v = 0.0;
      for (int w = 0; w < kSketchThreads / 32; ++w) v += red[w][tid];
      d.npart[(size_t)blockIdx.x * nb + tid] = v;
    }
  }
}

// Leverage sketch column n_obs + q: the s left rows of Omega a_q plus Omega_g (G a_q), and
// ||G a_q||^2 added to the leverage norm, in column order.
__global__ void grad_reduce_kernel(Dev d, int nb, int64_t n_obs, int nblk) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nb * d.s) {
    const int q = idx / d.s, r = idx % d.s;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += d.spart[((size_t)b * nb + q) * d.rows + r];
    d.Slev[(size_t)(n_obs + q) * d.lev_ld + r] = d.S[(size_t)(n_obs + q) * d.rows + r] + v;
  }
  if (idx == 0) {
    for (int q = 0; q < nb; ++q) {
      double v = 0.0;
      for (int b = 0; b < nblk; ++b) v += d.npart[(size_t)b * nb + q];
      if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
      d.fro2[1] += v;
    }
  }
}

// Omega (G^p a_q) for the s left rows of Omega (the main stream) and direction p: the sketches
// of Sec. 3.4's gradient-augmented coefficient problem.  Split-K over the m coordinates like the
// ingest sketch (working-precision sums over four chunks, then FP64); partials to d.spart.
template <typename T, int NB>
__global__ void __launch_bounds__(kSketchThreads)
gradc_sketch_kernel(Dev d, SimtCols cols, int nb, int p) {
  __shared__ T X[NB][kChunk];
  const int tid = threadIdx.x;
  const int r = blockIdx.y * kSketchThreads + tid;
  const bool row_ok = r < d.s;
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  double acc64[NB];
  T acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) { acc64[q] = 0.0; acc[q] = T(0); }
  const int64_t nchunks = (d.m + kChunk - 1) / kChunk;
  int pending = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t i0 = c * kChunk;
    const int64_t i = i0 + tid;
    if (i < d.m) {
      const GradStencil g = grad_stencil((int64_t)p * d.m + i, d.m, d.nx, d.ny);
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nb) {
          const T* a = (const T*)cols.p[q];
          T v = (T)g.wc * a[g.i];
          if (g.wm != 0.0) v += (T)g.wm * a[g.i - g.st];
          if (g.wp != 0.0) v += (T)g.wp * a[g.i + g.st];
          X[q][tid] = v;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nb) X[q][tid] = T(0);
    }
    __syncthreads();
    if (row_ok) {
      if (d.omega_kind == 1) {
#pragma unroll 1
        for (int half = 0; half < kChunk / 128; ++half) {
          const u32x4 w = philox4x32_10((uint32_t)((i0 >> 7) + half), (uint32_t)r, kTagRademacher, 0, k0, k1);
          const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int wi = 0; wi < 4; ++wi) {
#pragma unroll 8
            for (int e = 0; e < 32; ++e) {
              const int bpos = (e & 1) ? 31 - (e >> 1) : 15 - (e >> 1);
              const uint32_t bit = (words[wi] >> bpos) & 1u;
              const int ii = half * 128 + wi * 32 + e;
#pragma unroll
              for (int q = 0; q < NB; ++q)
                if (q < nb) acc[q] += flip_sign(X[q][ii], bit);
            }
          }
        }
      } else {
#pragma unroll 1
        for (int ii = 0; ii < kChunk; ++ii) {
          if (i0 + ii >= d.m) break;
          const T w = (T)gauss_entry(d.seed, kTagGauss, (uint32_t)r, (uint64_t)(i0 + ii));
#pragma unroll
          for (int q = 0; q < NB; ++q)
            if (q < nb) acc[q] += w * X[q][ii];
        }
      }
    }
    if (++pending == 4) {
#pragma unroll
      for (int q = 0; q < NB; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      pending = 0;
    }
    __syncthreads();
  }
  if (row_ok) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q < nb) d.spart[((size_t)blockIdx.x * nb + q) * d.rows + r] = acc64[q] + (double)acc[q];
  }
}

// Coefficient sketch column n_obs + q, direction p: Sg[((n_obs + q) 2 + p) s + r].
__global__ void gradc_reduce_kernel(Dev d, int nb, int64_t n_obs, int nblk, int p) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * d.s) return;
  const int q = idx / d.s, r = idx % d.s;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += d.spart[((size_t)b * nb + q) * d.rows + r];
  d.Sg[((size_t)(n_obs + q) * 2 + p) * d.s + r] = v;
}

int launch_grad(const Dev& d, const void* const* colp, int nb, int64_t n_obs, cudaStream_t st) {
  SimtCols cols;
  for (int q = 0; q < kMaxB; ++q) cols.p[q] = q < nb ? colp[q] : nullptr;
  const int64_t nchunks = (2 * d.m + kChunk - 1) / kChunk;
  const int nblk = (int)(nchunks < d.n_sketch_blocks ? nchunks : d.n_sketch_blocks);
  dim3 grid(nblk, (d.s + kSketchThreads - 1) / kSketchThreads);
  if (d.dtype == 0) {
    if (nb == 1) grad_sketch_kernel<double, 1><<<grid, kSketchThreads, 0, st>>>(d, cols, nb);
    else grad_sketch_kernel<double, kMaxB><<<grid, kSketchThreads, 0, st>>>(d, cols, nb);
  } else {
    if (nb == 1) grad_sketch_kernel<float, 1><<<grid, kSketchThreads, 0, st>>>(d, cols, nb);
    else grad_sketch_kernel<float, kMaxB><<<grid, kSketchThreads, 0, st>>>(d, cols, nb);
  }
  const int n = nb * d.s;
  grad_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, nb, n_obs, nblk);
  if (!d.grad_coeff) return 2;
  // the coefficient sketches Omega G^p a (the partial buffer is free again after the reduce)
  const int64_t mchunks = (d.m + kChunk - 1) / kChunk;
  const int mblk = (int)(mchunks < d.n_sketch_blocks ? mchunks : d.n_sketch_blocks);
  dim3 gm(mblk, (d.s + kSketchThreads - 1) / kSketchThreads);
  for (int p = 0; p < 2; ++p) {
    if (d.dtype == 0) {
      if (nb == 1) gradc_sketch_kernel<double, 1><<<gm, kSketchThreads, 0, st>>>(d, cols, nb, p);
      else gradc_sketch_kernel<double, kMaxB><<<gm, kSketchThreads, 0, st>>>(d, cols, nb, p);
    } else {
      if (nb == 1) gradc_sketch_kernel<float, 1><<<gm, kSketchThreads, 0, st>>>(d, cols, nb, p);
      else gradc_sketch_kernel<float, kMaxB><<<gm, kSketchThreads, 0, st>>>(d, cols, nb, p);
    }
    gradc_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, nb, n_obs, mblk, p);
  }
  return 6;
}

void launch_materialize_omega(const Dev& d, cudaStream_t st) {
  materialize_omega_kernel<<<4 * 152, 256, 0, st>>>(d);
}

void launch_gram_update(const Dev& d, int nb, int64_t n_obs, cudaStream_t st) {
  const int64_t ns = (int64_t)d.s * d.s;
  gram_update_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(d, nb, n_obs);
}

int launch_ingest(const Dev& d, const void* const* colp, int nb, int count, int64_t n_obs,
                  cudaStream_t st, cudaEvent_t* ev) {
  SimtCols cols;
  for (int q = 0; q < kMaxB; ++q) cols.p[q] = q < nb ? colp[q] : nullptr;
  if (ev) cudaEventRecord(ev[0], st);
  dim3 grid(d.n_sketch_blocks, (d.rows + kSketchThreads - 1) / kSketchThreads);
  if (d.dtype == 0) {
    if (nb == 1)
      ingest_sketch_kernel<double, 1><<<grid, kSketchThreads, 0, st>>>(d, cols, nb, count);
    else
      ingest_sketch_kernel<double, kMaxB><<<grid, kSketchThreads, 0, st>>>(d, cols, nb, count);
  } else {
    if (nb == 1)
      ingest_sketch_kernel<float, 1><<<grid, kSketchThreads, 0, st>>>(d, cols, nb, count);
    else
      ingest_sketch_kernel<float, kMaxB><<<grid, kSketchThreads, 0, st>>>(d, cols, nb, count);
  }
  if (ev) cudaEventRecord(ev[1], st);
  const int n = nb * d.rows;
  sketch_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, nb, n_obs, d.n_sketch_blocks);
  return 2;
}

}  // namespace rid
