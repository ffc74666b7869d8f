// Allocation-free sketch of a block of columns: rid_sketch_noalloc.
//
// Who needs it: a simulation that compresses its own snapshots in situ usually
// reserves nearly all of HBM for its fields through its own allocator, and its
// time-stepping loop must not be held up by the device-wide synchronisation
// that cudaMalloc / cudaFree imply.  Such a caller cannot let this library
// allocate per call; it passes the inputs and the outputs, and the library uses
// only the fixed scratch array below, which the CUDA runtime places in device
// memory when it loads this library's device code.
//
// What it computes: S(:, q) = Omega a_q for the s left rows and h probe rows of
// the Rademacher Omega of the streaming sketch (the counter-based generator with
// the same seed, rows and coordinates as a handle), and ||a_q||^2, for up to
// kNaMaxCols columns.  It is the split-K sketch of the ingest path without its
// buffer copy: a sketch kernel writes per-block partial sums into the scratch
// array and a reduction kernel adds them in block order into the caller's
// output.
//
// Scratch: file-scope, 8 MiB + 16 KiB per GPU, held from the first call until
// the process exits.  Every call on a device shares it and it keeps the last
// call's contents; nothing in it needs to start at zero, because every entry
// the reduction reads is first written by the same call's sketch kernel.  Two
// calls whose kernels overlap on the GPU (different streams with no ordering
// between them) race on the scratch and give wrong results; calls on one
// stream run one after the other and are safe.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "philox.cuh"
#include "rid.h"
#include "rid_internal.cuh"

namespace rid {

namespace {

constexpr int kNaMaxCols = 16;        // columns per call
constexpr int kNaMaxRows = 512;       // s + h
constexpr int kNaBlocks = 128;        // split-K blocks (partials kept per block)
constexpr int kNaThreads = 256;       // one sketch row per thread
constexpr int kNaChunk = 256;         // coordinates staged per block iteration
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaPartDoubles = (size_t)kNaBlocks * kNaMaxCols * kNaMaxRows;
constexpr size_t kNaNormDoubles = (size_t)kNaBlocks * kNaMaxCols;

// The only device memory this entry point uses besides the caller's buffers.
static __device__ __align__(256) double g_noalloc_scratch[kNaPartDoubles + kNaNormDoubles];

std::atomic<double*> g_scratch_ptr[kNaMaxDevices];
std::mutex g_setup_mu;

__device__ __forceinline__ double na_signed(double x, uint32_t bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((unsigned long long)bit << 63));
}
__device__ __forceinline__ float na_signed(float x, uint32_t bit) {
  return __int_as_float(__float_as_int(x) ^ (bit << 31));
}

// grid (nblk, ceil(rows / 256)), 256 threads; thread tid of row group y owns row
// r = 256 y + tid.  Block b takes the 256-coordinate chunks b, b + nblk, ...
// and writes its partial sums part[(b * nb + q) * rows + r] for every q < nb and
// row r < rows, and (row group 0) the partial squared norms npart[b * nb + q].
template <typename T>
__global__ void __launch_bounds__(kNaThreads)
noalloc_sketch_kernel(const T* __restrict__ cols, int64_t ld, int nb, int64_t m, int rows, uint64_t seed,
                      double* __restrict__ part, double* __restrict__ npart) {
  __shared__ T X[kNaMaxCols][kNaChunk];
  __shared__ double red[kNaThreads / 32][kNaMaxCols];
  const int tid = threadIdx.x;
  const int r = blockIdx.y * kNaThreads + tid;
  const bool row_ok = r < rows;
  const bool lead = blockIdx.y == 0;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

  double acc64[kNaMaxCols];
  T acc[kNaMaxCols];
  double nrm[kNaMaxCols];
#pragma unroll
  for (int q = 0; q < kNaMaxCols; ++q) { acc64[q] = 0.0; acc[q] = T(0); nrm[q] = 0.0; }

  const int64_t nchunks = (m + kNaChunk - 1) / kNaChunk;
  int pending = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t i0 = c * kNaChunk;
    const int64_t i = i0 + tid;
#pragma unroll
    for (int q = 0; q < kNaMaxCols; ++q) {
      if (q < nb) {
        const T v = (i < m) ? cols[(int64_t)q * ld + i] : T(0);
        X[q][tid] = v;
        nrm[q] += (double)v * (double)v;
      }
    }
    __syncthreads();
    if (row_ok) {
      // Omega(r, i) = -1 where the generator's bit for (r, i) is set, else +1.  One
      // Philox call (block i / 128, row r) gives the bits of 128 coordinates; within
      // its 32-bit word i / 32 % 4, coordinate pair p = (i % 32) / 2 takes bit 15 - p
      // (even i) or 31 - p (odd i).
#pragma unroll 1
      for (int half = 0; half < kNaChunk / 128; ++half) {
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
            for (int q = 0; q < kNaMaxCols; ++q)
              if (q < nb) acc[q] += na_signed(X[q][ii], bit);
          }
        }
      }
    }
    // working-precision sums over four chunks, then FP64
    if (++pending == 4) {
#pragma unroll
      for (int q = 0; q < kNaMaxCols; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      pending = 0;
    }
    __syncthreads();
  }
  if (row_ok) {
#pragma unroll
    for (int q = 0; q < kNaMaxCols; ++q)
      if (q < nb) part[((size_t)blockIdx.x * nb + q) * rows + r] = acc64[q] + (double)acc[q];
  }
  if (lead) {
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < kNaMaxCols; ++q) {
      double v = nrm[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (tid < nb) {
      double v = 0.0;
      for (int wq = 0; wq < kNaThreads / 32; ++wq) v += red[wq][tid];
      npart[(size_t)blockIdx.x * nb + tid] = v;
    }
  }
}

// One thread per (q, r): S_out(r, q) = sum of the nblk partials in block order;
// threads q < nb also add the norm partials.
__global__ void noalloc_reduce_kernel(const double* __restrict__ part, const double* __restrict__ npart, int nb,
                                      int rows, int nblk, double* __restrict__ S_out, int64_t lds,
                                      double* __restrict__ norms_out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nb * rows) {
    const int q = idx / rows, r = idx % rows;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += part[((size_t)b * nb + q) * rows + r];
    S_out[(int64_t)q * lds + r] = v;
  }
  if (idx < nb) {
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += npart[(size_t)b * nb + idx];
    norms_out[idx] = v;
  }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int na_fail(int code, const char* msg) {
  set_global_error(msg);
  return code;
}

}  // namespace

}  // namespace rid

extern "C" int rid_sketch_noalloc(const rid_config* cfg, const void* cols, int64_t ld, int32_t ncols,
                                  double* S_out, int64_t lds, double* norms_out) {
  using namespace rid;
  if (!cfg || !cols || !S_out || !norms_out) return na_fail(RID_EINVAL, "rid_sketch_noalloc: NULL argument");
  if (ncols < 1 || ncols > kNaMaxCols)
    return na_fail(RID_EINVAL, "rid_sketch_noalloc: ncols must be in [1, 16] (fixed scratch limit)");
  if (cfg->m < 1) return na_fail(RID_EINVAL, "rid_sketch_noalloc: m must be >= 1");
  if (cfg->s < 1 || cfg->h < 0) return na_fail(RID_EINVAL, "rid_sketch_noalloc: need s >= 1 and h >= 0");
  const int64_t rows64 = (int64_t)cfg->s + cfg->h;
  if (rows64 > kNaMaxRows)
    return na_fail(RID_EINVAL, "rid_sketch_noalloc: s + h must be <= 512 (fixed scratch limit)");
  const int rows = (int)rows64;
  if (ld < cfg->m) return na_fail(RID_EINVAL, "rid_sketch_noalloc: ld must be >= m");
  if (lds < rows) return na_fail(RID_EINVAL, "rid_sketch_noalloc: lds must be >= s + h");
  if (cfg->omega_kind != RID_OMEGA_RADEMACHER)
    return na_fail(RID_EINVAL, "rid_sketch_noalloc: only the Rademacher Omega is generated without allocation");
  if (cfg->data_dtype != RID_F64 && cfg->data_dtype != RID_F32)
    return na_fail(RID_EINVAL, "rid_sketch_noalloc: unknown data_dtype");

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return na_fail(RID_ENOLIB, "rid_sketch_noalloc: no CUDA device");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return na_fail(RID_ECUDA, "rid_sketch_noalloc: cannot query the current device");
  if (!is_device_pointer(cols) || !is_device_pointer(S_out) || !is_device_pointer(norms_out))
    return na_fail(RID_EINVAL, "rid_sketch_noalloc: cols, S_out and norms_out must be device memory");

  // Set-up, once per device, with that device current: the address of the scratch.
  double* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    scratch = g_scratch_ptr[dev].load(std::memory_order_relaxed);
    if (!scratch) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return na_fail(RID_ECUDA, "rid_sketch_noalloc: cudaGetSymbolAddress of the scratch array failed");
      }
      scratch = static_cast<double*>(p);
      g_scratch_ptr[dev].store(scratch, std::memory_order_release);
    }
  }

  cudaStream_t st = (cudaStream_t)cfg->cuda_stream;
  // The scratch address above is the current device's; the kernels run on cfg->cuda_stream, which
  // must therefore belong to that device (the legacy default stream always does).
  if (st != nullptr) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return na_fail(RID_EINVAL, "rid_sketch_noalloc: cannot query the device of cfg->cuda_stream");
    }
    if (sdev != dev)
      return na_fail(RID_EINVAL,
                     "rid_sketch_noalloc: cfg->cuda_stream belongs to another device than the current one "
                     "(make the stream's device current first)");
  }
  const int64_t nchunks = (cfg->m + kNaChunk - 1) / kNaChunk;
  const int nblk = (int)(nchunks < kNaBlocks ? nchunks : kNaBlocks);
  double* part = scratch;
  double* npart = scratch + kNaPartDoubles;
  const dim3 grid((unsigned)nblk, (unsigned)((rows + kNaThreads - 1) / kNaThreads));
  if (cfg->data_dtype == RID_F64)
    noalloc_sketch_kernel<double><<<grid, kNaThreads, 0, st>>>(static_cast<const double*>(cols), ld, ncols,
                                                                cfg->m, rows, cfg->seed, part, npart);
  else
    noalloc_sketch_kernel<float><<<grid, kNaThreads, 0, st>>>(static_cast<const float*>(cols), ld, ncols,
                                                               cfg->m, rows, cfg->seed, part, npart);
  const int nred = ncols * rows;
  noalloc_reduce_kernel<<<(nred + 255) / 256, 256, 0, st>>>(part, npart, ncols, rows, nblk, S_out, lds,
                                                             norms_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(RID_ECUDA, cudaGetErrorString(e));
  return RID_OK;
}
