// Optional right sketch Y (m x l) += sum_q a_q omega_{j0+q}^T over a group of ingested columns.
//
// Not part of the paper's method: a running m x l sketch of the stream's range (each snapshot's
// l-vector omega_j is drawn from its own Philox stream, keyed by the snapshot index j).  Y is
// read and written once per group of up to 64 (FP32) or 32 (FP64) columns, so its traffic is
// 2 x (bytes of Y) / (group size) per snapshot; the arithmetic is l FMAs per coordinate and
// column, about the FP32 pipe's balance point against HBM.
//
// Kernels: right_w_kernel draws the group's W (G x lw, zero-padded to lw = l rounded up to 8);
// right_sketch_kernel is persistent (one CTA per SM) over a block of up to 256 sketch columns:
// it stages that block of W once, then for each tile of 256 C coordinates stages the group's
// columns in shared memory and updates Y in runs of 16 sketch columns -- each thread keeps C
// coordinates x 16 columns of Y in registers, adds sum_q a_q[i] W[q][r] in snapshot order, and
// has the next run's Y loads in flight meanwhile.
#include "rid_internal.cuh"
#include "philox.cuh"

namespace rid {

constexpr uint32_t kTagRightRademacher = 0x52534B31u;   // 'RSK1'
constexpr uint32_t kTagRightGauss = 0x52534731u;        // 'RSG1'

namespace {

constexpr int kRThreads = 256;
constexpr int kRBlock = 256;                          // sketch columns per pass over a tile
constexpr int kRR = 16;                               // sketch columns per register run

template <typename T> struct RTraits;
template <> struct RTraits<float> { static constexpr int kC = 2, kQ = 64; };
template <> struct RTraits<double> { static constexpr int kC = 1, kQ = 32; };

struct RCols {
  const void* p[64];
};

template <typename T>
__global__ void right_w_kernel(Dev d, int64_t j0, int G, int lw, T* __restrict__ W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G * lw) return;
  const int q = idx / lw, r = idx % lw;
  double v = 0.0;
  if (r < d.right_l)
    v = d.omega_kind == 1 ? rademacher_entry(d.seed, kTagRightRademacher, (uint32_t)r, (uint64_t)(j0 + q))
                          : gauss_entry(d.seed, kTagRightGauss, (uint32_t)r, (uint64_t)(j0 + q));
  W[idx] = (T)v;
}

// Sketch columns rb .. rb + rl - 1 (rl <= kRBlock) of Y for the group; W columns staged with
// row stride lwb = rl rounded up to kRR (zero-padded).  Thread t owns coordinates
// i0 + C t .. i0 + C t + C - 1 of each tile; a run of kRR sketch columns of Y lives in its
// registers while the next run's values are already being loaded.
template <typename T>
__global__ void __launch_bounds__(kRThreads, 1)
right_sketch_kernel(Dev d, RCols cols, int G, int lw, const T* __restrict__ Wg, int rb, int rl, int vec) {
  constexpr int C = RTraits<T>::kC;
  constexpr int TW = kRThreads * C;                     // coordinates per tile
  extern __shared__ __align__(16) unsigned char rsm[];
  const int lwb = (rl + kRR - 1) / kRR * kRR;
  T* Ws = reinterpret_cast<T*>(rsm);                    // G x lwb
  T* As = Ws + (size_t)RTraits<T>::kQ * kRBlock;        // G x TW
  const int tid = threadIdx.x;
  const int64_t m = d.m, m_pad = d.m_pad, ldy = d.m_pad;
  T* Y = reinterpret_cast<T*>(d.Y) + (int64_t)rb * ldy;
  for (int idx = tid; idx < G * lwb; idx += kRThreads) {
    const int q = idx / lwb, r = idx - q * lwb;
    Ws[idx] = (r < rl) ? Wg[q * lw + rb + r] : T(0);
  }
  const int ic = tid * C;
  for (int64_t tile = blockIdx.x; tile * TW < m; tile += gridDim.x) {
    const int64_t i0 = tile * TW;
    __syncthreads();                                    // W staged; the previous tile's A consumed
    if (vec && i0 + TW <= m) {
      // 16-byte loads (every column 16-byte aligned, the tile inside m)
      constexpr int V = 16 / sizeof(T), TV = TW / V;
#pragma unroll 8
      for (int idx = tid; idx < G * TV; idx += kRThreads) {
        const int q = idx / TV, iv = idx - q * TV;
        const float4 v = *reinterpret_cast<const float4*>(reinterpret_cast<const T*>(cols.p[q]) + i0 + iv * V);
        *reinterpret_cast<float4*>(As + q * TW + iv * V) = v;
      }
    } else {
#pragma unroll 8
      for (int idx = tid; idx < G * TW; idx += kRThreads) {
        const int q = idx / TW, ii = idx - q * TW;
        const int64_t i = i0 + ii;
        As[idx] = (i < m) ? reinterpret_cast<const T*>(cols.p[q])[i] : T(0);
      }
    }
    __syncthreads();
    const int64_t ib = i0 + ic;                         // C consecutive coordinates, all < m_pad or none
    if (ib >= m_pad) continue;
    T ynext[kRR][C];
#pragma unroll
    for (int rr = 0; rr < kRR; ++rr)
#pragma unroll
      for (int c = 0; c < C; ++c) ynext[rr][c] = (rr < rl) ? Y[ib + c + (int64_t)rr * ldy] : T(0);
    for (int r0 = 0; r0 < rl; r0 += kRR) {
      T acc[kRR][C];
#pragma unroll
      for (int rr = 0; rr < kRR; ++rr)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[rr][c] = ynext[rr][c];
      if (r0 + kRR < rl) {                              // the next run's Y, in flight during this run
#pragma unroll
        for (int rr = 0; rr < kRR; ++rr)
#pragma unroll
          for (int c = 0; c < C; ++c)
            ynext[rr][c] = (r0 + kRR + rr < rl) ? Y[ib + c + (int64_t)(r0 + kRR + rr) * ldy] : T(0);
      }
#pragma unroll 2
      for (int q = 0; q < G; ++q) {
        T a[C], w[kRR];
#pragma unroll
        for (int c = 0; c < C; ++c) a[c] = As[q * TW + ic + c];
#pragma unroll
        for (int rr = 0; rr < kRR; ++rr) w[rr] = Ws[q * lwb + r0 + rr];
#pragma unroll
        for (int rr = 0; rr < kRR; ++rr)
#pragma unroll
          for (int c = 0; c < C; ++c) acc[rr][c] = fma(a[c], w[rr], acc[rr][c]);
      }
#pragma unroll
      for (int rr = 0; rr < kRR; ++rr)
        if (r0 + rr < rl)
#pragma unroll
          for (int c = 0; c < C; ++c) Y[ib + c + (int64_t)(r0 + rr) * ldy] = acc[rr][c];
    }
  }
}

template <typename T>
int launch_right_t(const Dev& d, const void* const* cols, int ncols, int64_t j0, cudaStream_t st) {
  constexpr int Q = RTraits<T>::kQ, C = RTraits<T>::kC;
  const int lw = (d.right_l + 7) / 8 * 8;
  const size_t smem = sizeof(T) * (size_t)Q * kRBlock + sizeof(T) * (size_t)Q * kRThreads * C;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(right_sketch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  const int64_t ntiles = (d.m + kRThreads * C - 1) / (kRThreads * C);
  const int grid = (int)(ntiles < d.n_sm ? ntiles : d.n_sm);
  int nk = 0;
  for (int q0 = 0; q0 < ncols; q0 += Q) {
    const int G = ncols - q0 < Q ? ncols - q0 : Q;
    RCols c{};
    int vec = 1;
    for (int q = 0; q < G; ++q) {
      c.p[q] = cols[q0 + q];
      if ((uintptr_t)cols[q0 + q] & 15u) vec = 0;
    }
    T* W = reinterpret_cast<T*>(d.Wr);
    right_w_kernel<T><<<(G * lw + 255) / 256, 256, 0, st>>>(d, j0 + q0, G, lw, W);
    nk += 1;
    if constexpr (sizeof(T) == 4) {
      if (d.tc_right) {
        const int nt = launch_tc_right(d, cols + q0, G, reinterpret_cast<const float*>(W), lw, st);
        if (nt < 0) return -1;
        nk += nt;
        continue;
      }
    }
    for (int rb = 0; rb < d.right_l; rb += kRBlock) {
      const int rl = d.right_l - rb < kRBlock ? d.right_l - rb : kRBlock;
      right_sketch_kernel<T><<<grid, kRThreads, smem, st>>>(d, c, G, lw, W, rb, rl, vec);
      nk += 1;
    }
  }
  return nk;
}

}  // namespace

size_t right_w_bytes(const Dev& d) {
  const int lw = (d.right_l + 7) / 8 * 8;
  return (d.dtype == 0 ? sizeof(double) * RTraits<double>::kQ : sizeof(float) * RTraits<float>::kQ) * (size_t)lw;
}

int launch_right_sketch(const Dev& d, const void* const* cols, int ncols, int64_t j0, cudaStream_t st) {
  if (d.right_l <= 0 || ncols <= 0) return 0;
  return d.dtype == 0 ? launch_right_t<double>(d, cols, ncols, j0, st) : launch_right_t<float>(d, cols, ncols, j0, st);
}

}  // namespace rid
