// Tensor-core ingest for FP32 snapshots (sm_103a, tcgen05 + TMEM).
//
// One launch sketches a group of G <= 64 (split) or <= 128 (hi only) columns:
//   S(:, q) = Omega a_q  for every left and probe row of Omega (Algorithm 3),
// while copying each column into its buffer slot and accumulating its squared
// norm -- one HBM read of each column.
//
// MMA mapping (kind::f16, BF16 operands, FP32 accumulation in TMEM):
//   A (M = 128, K-major): rows are the data columns, split a = hi + lo in BF16
//                         (row q = hi(a_q), row 64 + q = lo(a_q)), or hi only.
//   B (N <= 256 per tile, K-major): rows of Omega, +-1 exactly representable in
//                         BF16, generated on chip from the counter-based generator.
//   D (128 x R16 FP32 in TMEM): D[q][r] = sum_i A[q][i] Omega[r][i].
// The contraction runs over the coordinates; each CTA owns a contiguous range
// of 64-coordinate chunks and keeps its partial D in TMEM for the whole range
// (split-K over the SMs); a deterministic FP64 reduction adds the partials.
//
// Warp roles: warp 0 allocates TMEM and one lane issues the MMAs; warps 1..8
// produce both operands (HBM loads with a two-chunk register prefetch, the
// split into BF16, the copy to the buffer slot, Philox expansion of Omega) and
// then read the accumulators back.  Two SMEM stages, mbarrier hand-off, every
// wait bounded (on timeout: error flag, drain, free TMEM, return).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "rid_internal.cuh"

namespace rid {

namespace {

constexpr int kChunkK = 64;                 // coordinates per chunk: one 128-byte BF16 row
constexpr int kProducerWarps = 16;           // ingest: 4 producer warps per SM sub-partition
constexpr int kThreads = 32 * (1 + kProducerWarps);
constexpr int kGramProducerWarps = 8;        // basis Gram: 4 column segments x 64 tasks
constexpr int kGramThreads = 32 * (1 + kGramProducerWarps);
constexpr int kATile = 128 * 128;           // 128 rows x 128 bytes
constexpr int kBTile = 512 * 128;           // up to 512 Omega rows x 128 bytes
constexpr int kSmemBytes = 2 * kATile + 2 * kBTile + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kL2Ahead = 6;                 // L2 prefetch distance of the ingest, in chunks
constexpr int kMaxStages = 4;               // ingest ring stages (barrier slots)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls (or when another role gave up), raising the CTA
// abort flag and the device error word.  Pipeline waits take the handle's limit (d.ring_wait_limit,
// kRingWaitLimit unless a test shortened it); the final wait for the MMAs in flight always takes
// kWaitLimit, so that TMEM is freed only once they have completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 32) __nanosleep(128);
  }
  *abort_flag = 1;
  atomicOr(err, ERR_TIMEOUT);
  return false;
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
  d |= (uint64_t)1u << 16;                     // leading byte offset (unused when K fits the swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1u << 46;                     // descriptor version
  d |= (uint64_t)2u << 61;                     // SWIZZLE_128B
  return d;
}
// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of the 16-byte chunk c of row r in a K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const uint32_t a = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (b << 16);
}

struct Cols {
  const float* p[128];
};

}  // namespace

// One pass of the tensor-core sketch: rows [rlo, rlo + rows of the launch) of the test matrix
// with counter tag `tag`, over `len` coordinates of each column; `copy`: also copy the columns
// into their buffer slots (the first pass over the data).  The plain sketch of a stream with
// more than 512 rows takes several passes (the 512 TMEM accumulator columns of one CTA), and
// gradient mode sketches the 2m-long gradient field with the gradient test matrix.
struct TcPass {
  int64_t len;
  int rlo;
  uint32_t tag;
  int copy;
};

namespace {

// 16 coordinates of one column: 4 float4 (aligned) or guarded scalars.
__device__ __forceinline__ void load16(const float* src, int64_t i, int64_t m, bool vec, float4 (&v)[4]) {
  if (vec && i + 16 <= m) {
    const float4* s = reinterpret_cast<const float4*>(src + i);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __ldcs(s + j);
  } else {
    float t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) t[j] = (i + j < m) ? src[i + j] : 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = make_float4(t[4 * j], t[4 * j + 1], t[4 * j + 2], t[4 * j + 3]);
  }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1)
tc_ingest_kernel(Dev d, Cols cols, int ncols, int split, int count, int nrows16, int n1, int n2,
                 int64_t chunks_per_cta, int vec, float* __restrict__ part, double* __restrict__ npart,
                 int nstage, uint32_t btile, TcPass ps) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  // nstage ring stages of one A tile (16 KB) and one B tile (btile = nrows16 x 128 bytes)
  const uint32_t sA = base;
  const uint32_t sB = base + (uint32_t)nstage * kATile;
  const uint32_t sBar = sB + (uint32_t)nstage * btile;   // full[4], empty[4], done
  uint8_t* gbar = gbase + (sBar - base);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 96);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 104);
  const uint32_t bar_full0 = sBar, bar_empty0 = sBar + 32, bar_done = sBar + 64;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nchunks = (ps.len + kChunkK - 1) / kChunkK;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_cta;
  int64_t c1 = c0 + chunks_per_cta;
  if (c1 > nchunks) c1 = nchunks;
  const int64_t nch = c1 > c0 ? c1 - c0 : 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) {
      mbar_init(bar_full0 + 8 * i, 32 * kProducerWarps);
      mbar_init(bar_empty0 + 8 * i, 1);
    }
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t id1 = idesc_bf16(128, n1);
      const uint32_t id2 = idesc_bf16(128, n2 > 0 ? n2 : 16);
      int st = 0;
      uint32_t par = 0;
      for (int64_t c = 0; c < nch; ++c) {
        if (!mbar_wait(bar_full0 + 8 * st, par, abort_flag, d.err, d.ring_wait_limit)) break;
        tc_fence_after();
        const uint64_t da = desc_sw128(sA + st * kATile);
        const uint64_t db1 = desc_sw128(sB + st * btile);
        const uint64_t db2 = desc_sw128(sB + st * btile + 256 * 128);
#pragma unroll
        for (int kk = 0; kk < kChunkK / 16; ++kk) {
          const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
          const uint64_t adv = (uint64_t)(kk * 2);            // +32 bytes along K
          tc_mma(tmem, da + adv, db1 + adv, id1, acc);
          if (n2 > 0) tc_mma(tmem + (uint32_t)n1, da + adv, db2 + adv, id2, acc);
        }
        tc_commit(bar_empty0 + 8 * st);
        if (++st == nstage) { st = 0; par ^= 1u; }
      }
      tc_commit(bar_done);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- producers
    // 512 producer threads: thread pt moves coordinates 8g..8g+7 of every chunk of column
    // q = pt / 8 (g = pt % 8: one 16-byte BF16 unit of the 128-byte A row) and expands
    // Omega row pt.  Every producer thread arrives once per chunk.
    const int pt = threadIdx.x - 32;          // 0..511
    const int q = pt >> 3, g = pt & 7;
    const bool has_col = q < ncols;
    const float* src = has_col ? cols.p[q] : nullptr;
    float* dstp = (has_col && ps.copy) ? (float*)d.pool + (int64_t)d.dslot[count + q] * d.m_pad : nullptr;
    const int r0 = pt;                        // Omega row of this thread
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    // squared norm: compensated FP32 sum (Kahan) over this CTA's coordinates, converted to FP64
    // at the end: its error stays at a few FP32 roundings of the total, and the loop issues no
    // FP64 instruction (this GPU issues about one per warp per 64 cycles)
    float ks = 0.f, kc = 0.f;
    uint32_t keep[2] = {0u, 0u};
    float4 bufA[2], bufB[2];
    // Loads run two chunks ahead in registers; one lane per column also asks L2 for the
    // column's chunk kL2Ahead chunks ahead (a bulk prefetch), so that those loads hit L2.
    auto load_chunk = [&](int64_t c, float4 (&v)[2]) {
      if (has_col && c < nch) {
        const int64_t i = (c0 + c) * kChunkK + 8 * g;
        if (vec && i + 8 <= ps.len) {
          const float4* s4 = reinterpret_cast<const float4*>(src + i);
          v[0] = __ldcs(s4);
          v[1] = __ldcs(s4 + 1);
        } else {
          float t[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) t[j] = (i + j < ps.len) ? src[i + j] : 0.f;
          v[0] = make_float4(t[0], t[1], t[2], t[3]);
          v[1] = make_float4(t[4], t[5], t[6], t[7]);
        }
      }
      if (has_col && g == 0 && vec && c + kL2Ahead < nch && (c0 + c + kL2Ahead + 1) * kChunkK <= ps.len)
        prefetch_l2(src + (c0 + c + kL2Ahead) * kChunkK, kChunkK * 4);
    };
    int pst = 0;
    uint32_t ppar = 1u;                       // first pass over the ring: stages start empty
    auto process = [&](int64_t c, const float4 (&v)[2]) -> bool {
      const int st = pst;
      if (!mbar_wait(bar_empty0 + 8 * st, ppar, abort_flag, d.err, d.ring_wait_limit)) return false;
      if (++pst == nstage) { pst = 0; ppar ^= 1u; }
      const int64_t cg = c0 + c;
      const uint32_t ast = sA + st * kATile;
      if (has_col) {
        const int64_t i0 = cg * kChunkK + 8 * g;
        const float x[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
        // copy into the buffer slot (first pass only)
        if (dstp) {
          if (i0 + 8 <= d.m) {
            float4* o = reinterpret_cast<float4*>(dstp + i0);
            __stcs(o, v[0]);
            __stcs(o + 1, v[1]);
          } else {
            for (int j = 0; j < 8; ++j) if (i0 + j < d.m) dstp[i0 + j] = x[j];
          }
        }
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s2 = fmaf(x[j], x[j], s2);
        {
          const float y = s2 - kc;
          const float tsum = ks + y;
          kc = (tsum - ks) - y;
          ks = tsum;
        }
        // a = hi + lo with hi = bf16(a) and lo = bf16(a - hi), two coordinates per 32-bit word
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
          const uint32_t hv = *reinterpret_cast<const uint32_t*>(&h2);
          hw[j] = hv;
          const float ra = x[2 * j] - __uint_as_float(hv << 16);
          const float rb = x[2 * j + 1] - __uint_as_float(hv & 0xFFFF0000u);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(ra, rb);
          lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        sts128(ast + sw128_off(q, g), hw[0], hw[1], hw[2], hw[3]);
        if (split) sts128(ast + sw128_off(64 + q, g), lw[0], lw[1], lw[2], lw[3]);
      }
      if (r0 < nrows16) {
        const uint32_t bst = sB + st * btile;
        uint32_t wa, wb;
        if ((cg & 1) == 0) {
          // counter block of 128 global rows (the shard offset is a multiple of 128)
          const u32x4 w = philox4x32_10((uint32_t)((cg >> 1) + (d.row_offset >> 7)), (uint32_t)(ps.rlo + r0), ps.tag,
                                        0, k0, k1);
          wa = w.x; wb = w.y; keep[0] = w.z; keep[1] = w.w;
        } else {
          wa = keep[0]; wb = keep[1];
        }
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const uint32_t w = (cc < 4) ? wa : wb;
          const int p0 = 4 * (cc & 3);
          const uint32_t v0 = ((w << (p0 + 0)) & 0x80008000u) | 0x3F803F80u;
          const uint32_t v1 = ((w << (p0 + 1)) & 0x80008000u) | 0x3F803F80u;
          const uint32_t v2 = ((w << (p0 + 2)) & 0x80008000u) | 0x3F803F80u;
          const uint32_t v3 = ((w << (p0 + 3)) & 0x80008000u) | 0x3F803F80u;
          sts128(bst + sw128_off(r0, cc), v0, v1, v2, v3);
        }
      }
      fence_async_smem();
      mbar_arrive(bar_full0 + 8 * st);
      return true;
    };
    if (has_col && g == 0 && vec)
      for (int64_t c = 2; c < kL2Ahead && c < nch; ++c)
        if ((c0 + c + 1) * kChunkK <= ps.len) prefetch_l2(src + (c0 + c) * kChunkK, kChunkK * 4);
    load_chunk(0, bufA);
    load_chunk(1, bufB);
    for (int64_t c = 0; c < nch; c += 2) {
      if (!process(c, bufA)) break;
      load_chunk(c + 2, bufA);
      if (c + 1 < nch) {
        if (!process(c + 1, bufB)) break;
        load_chunk(c + 3, bufB);
      }
    }
    double nrm = (double)ks - (double)kc;
    // squared norms: the eight segment threads of a column are adjacent lanes
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 1);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 2);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 4);
    if (has_col && g == 0) npart[(size_t)blockIdx.x * 128 + q] = nrm;

    // ---------------------------------------------------------------- epilogue (warps 1..4)
    if (warp <= 4) {
      const bool ok = mbar_wait(bar_done, 0, abort_flag, d.err);
      tc_fence_after();
      if (ok && !*abort_flag) {
        const int quarter = warp & 3;           // TMEM lanes 32*quarter .. +31
        const int L = 32 * quarter + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
        for (int cb = 0; cb < nrows16; cb += 32) {
          uint32_t r[32];
          tc_ld32(taddr + (uint32_t)cb, r);
          tc_wait_ld();
          float* o = part + ((size_t)blockIdx.x * nrows16 + cb) * 128 + L;
          const int jn = (nrows16 - cb < 32) ? nrows16 - cb : 32;   // rows of this CTA's slice only
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < jn) o[(size_t)j * 128] = (nch > 0) ? __uint_as_float(r[j]) : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// S(:, n_obs + q) = sum over CTAs of the hi (and lo) rows; norms in CTA order.
// grid: d.rows + 1 CTAs of 256 threads.  CTA r < rows: S(r, n_obs + q) = sum over the split-K
// blocks of the hi and lo partials of column q; thread (j, q) sums the blocks b = j (mod 4) in
// order, and the four partial sums are added in the fixed order j = 0..3 (deterministic).
// CTA rows: the squared norms, added to ||A_obs||^2 in column order.
__global__ void __launch_bounds__(256) tc_reduce_kernel(Dev d, const float* __restrict__ part,
                                                        const double* __restrict__ npart, int nblk,
                                                        int ncols, int split, int nrows16, int64_t n_obs) {
  __shared__ double red[4][64];
  const int q = threadIdx.x & 63, j = threadIdx.x >> 6;
  if ((int)blockIdx.x < d.rows) {
    const int r = blockIdx.x;
    double v = 0.0;
    if (q < ncols) {
      for (int b = j; b < nblk; b += 4) {
        const float* p = part + ((size_t)b * nrows16 + r) * 128;
        v += (double)p[q];
        if (split) v += (double)p[64 + q];
      }
    }
    red[j][q] = v;
    __syncthreads();
    if (j == 0 && q < ncols)
      d.S[(size_t)(n_obs + q) * d.rows + r] = ((red[0][q] + red[1][q]) + red[2][q]) + red[3][q];
  } else {
    if (j == 0) {
      double v = 0.0;
      if (q < ncols)
        for (int b = 0; b < nblk; ++b) v += npart[(size_t)b * 128 + q];
      red[0][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int c = 0; c < ncols; ++c) {
        const double v = red[0][c];
        if (d.gnorm) {                      // row shard: summed over the shards first
          d.gnorm[c] = v;
          continue;
        }
        if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
        d.fro2[0] += v;
        d.fro2[1] += v;
      }
    }
  }
}

// ---------------------------------------------------------------- basis Gram on tensor cores
// G(x, y) = <pool[gnew[x0 + x]], pool[gtgt[y0 + y]]> for x < nx <= 64, y < ny <= 128, over
// all m coordinates: A rows are the new columns split hi/lo (rows x, 64 + x), B rows the
// target columns split hi/lo (rows y, 128 + y), so that the four BF16 cross products of
// (hi + lo)(hi + lo) land in D(x | 64 + x, y | 128 + y); the split leaves an error of
// at most ~2^-16 |a_i b_i| per term.  Same pipeline as the ingest kernel, no Omega.
constexpr int kGramN = 256;

__global__ void __launch_bounds__(kGramThreads, 1)
tc_gram_kernel(Dev d, int x0, int y0, int64_t chunks_per_cta, float* __restrict__ part) {
  extern __shared__ uint8_t smem_raw[];
  const int nx = min(64, d.meta[META_NNEW] - x0);     // counts are decided on the device
  const int ny = min(128, d.meta[META_NTGT] - y0);
  if (nx <= 0 || ny <= 0) return;                     // uniform over the CTA, before any TMEM use
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sA = base;
  const uint32_t sB = base + 2 * kATile;
  const uint32_t sBar = sB + 2 * kBTile;
  uint8_t* gbar = gbase + (sBar - base);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 64);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 72);
  const uint32_t bar_full0 = sBar, bar_empty0 = sBar + 16, bar_done = sBar + 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nchunks = (d.m + kChunkK - 1) / kChunkK;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_cta;
  int64_t c1 = c0 + chunks_per_cta;
  if (c1 > nchunks) c1 = nchunks;
  const int64_t nch = c1 > c0 ? c1 - c0 : 0;
  if (threadIdx.x == 0) {
    mbar_init(bar_full0, 32 * kGramProducerWarps);
    mbar_init(bar_full0 + 8, 32 * kGramProducerWarps);
    mbar_init(bar_empty0, 1);
    mbar_init(bar_empty0 + 8, 1);
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      const uint32_t id = idesc_bf16(128, kGramN);
      for (int64_t c = 0; c < nch; ++c) {
        const int st = (int)(c & 1);
        if (!mbar_wait(bar_full0 + 8 * st, (uint32_t)((c >> 1) & 1), abort_flag, d.err, d.ring_wait_limit)) break;
        tc_fence_after();
        const uint64_t da = desc_sw128(sA + st * kATile);
        const uint64_t db = desc_sw128(sB + st * kBTile);
#pragma unroll
        for (int kk = 0; kk < kChunkK / 16; ++kk)
          tc_mma(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), id, (c > 0 || kk > 0) ? 1u : 0u);
        tc_commit(bar_empty0 + 8 * st);
      }
      tc_commit(bar_done);
    }
    __syncwarp();
  } else {
    const int pt = threadIdx.x - 32;
    const float* pool = (const float*)d.pool;
    // task 0: new column qa (A rows qa, 64 + qa); tasks 1, 2: target columns (B rows)
    const int qa = pt >> 2, g = pt & 3;
    const bool tasks = pt < 256;               // 64 A columns and 2 x 64 B columns, 4 segments each
    const bool hasA = tasks && qa < nx;
    const float* srcA = hasA ? pool + (int64_t)d.gnew[x0 + qa] * d.m_pad : nullptr;
    const int qb0 = pt >> 2, qb1 = 64 + (pt >> 2);
    const bool hasB0 = tasks && qb0 < ny, hasB1 = tasks && qb1 < ny;
    const float* srcB0 = hasB0 ? pool + (int64_t)d.gtgt[y0 + qb0] * d.m_pad : nullptr;
    const float* srcB1 = hasB1 ? pool + (int64_t)d.gtgt[y0 + qb1] * d.m_pad : nullptr;
    float4 a0[4], a1[4], b00[4], b01[4], b10[4], b11[4];
    auto ld = [&](const float* src, bool has, int64_t c, float4 (&v)[4]) {
      if (has && c < nch) load16(src, (c0 + c) * kChunkK + 16 * g, d.m, true, v);
    };
    auto put = [&](uint32_t tile, int row_hi, int row_lo, const float4 (&v)[4]) {
      float xv[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) { xv[4 * j] = v[j].x; xv[4 * j + 1] = v[j].y; xv[4 * j + 2] = v[j].z; xv[4 * j + 3] = v[j].w; }
      uint32_t hw[8], lw[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float a = xv[2 * j], bb = xv[2 * j + 1];
        const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(bb);
        hw[j] = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
        lw[j] = pack_bf16(a - __bfloat162float(ha), bb - __bfloat162float(hb));
      }
      sts128(tile + sw128_off(row_hi, 2 * g), hw[0], hw[1], hw[2], hw[3]);
      sts128(tile + sw128_off(row_hi, 2 * g + 1), hw[4], hw[5], hw[6], hw[7]);
      sts128(tile + sw128_off(row_lo, 2 * g), lw[0], lw[1], lw[2], lw[3]);
      sts128(tile + sw128_off(row_lo, 2 * g + 1), lw[4], lw[5], lw[6], lw[7]);
    };
    auto process = [&](int64_t c, const float4 (&va)[4], const float4 (&vb0)[4], const float4 (&vb1)[4]) -> bool {
      const int st = (int)(c & 1);
      if (!mbar_wait(bar_empty0 + 8 * st, (uint32_t)(((c >> 1) & 1) ^ 1), abort_flag, d.err, d.ring_wait_limit)) return false;
      const uint32_t ast = sA + st * kATile, bst = sB + st * kBTile;
      if (hasA) put(ast, qa, 64 + qa, va);
      if (hasB0) put(bst, qb0, 128 + qb0, vb0);
      if (hasB1) put(bst, qb1, 128 + qb1, vb1);
      fence_async_smem();
      mbar_arrive(bar_full0 + 8 * st);
      return true;
    };
    ld(srcA, hasA, 0, a0); ld(srcB0, hasB0, 0, b00); ld(srcB1, hasB1, 0, b10);
    ld(srcA, hasA, 1, a1); ld(srcB0, hasB0, 1, b01); ld(srcB1, hasB1, 1, b11);
    for (int64_t c = 0; c < nch; c += 2) {
      if (!process(c, a0, b00, b10)) break;
      ld(srcA, hasA, c + 2, a0); ld(srcB0, hasB0, c + 2, b00); ld(srcB1, hasB1, c + 2, b10);
      if (c + 1 < nch) {
        if (!process(c + 1, a1, b01, b11)) break;
        ld(srcA, hasA, c + 3, a1); ld(srcB0, hasB0, c + 3, b01); ld(srcB1, hasB1, c + 3, b11);
      }
    }
    if (warp <= 4) {
      const bool ok = mbar_wait(bar_done, 0, abort_flag, d.err);
      tc_fence_after();
      if (ok && !*abort_flag) {
        const int quarter = warp & 3;
        const int L = 32 * quarter + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
        for (int cb = 0; cb < kGramN; cb += 32) {
          uint32_t r[32];
          tc_ld32(taddr + (uint32_t)cb, r);
          tc_wait_ld();
          float* o = part + ((size_t)blockIdx.x * kGramN + cb) * 128 + L;
#pragma unroll
          for (int j = 0; j < 32; ++j) o[(size_t)j * 128] = (nch > 0) ? __uint_as_float(r[j]) : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

__global__ void tc_gram_reduce_kernel(Dev d, const float* __restrict__ part, int nblk, int x0, int y0) {
  const int nx = min(64, d.meta[META_NNEW] - x0);
  const int ny = min(128, d.meta[META_NTGT] - y0);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (nx <= 0 || ny <= 0 || idx >= nx * ny) return;
  const int x = idx % nx, y = idx / nx;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const float* p = part + (size_t)b * kGramN * 128;
    v += (double)p[(size_t)y * 128 + x] + (double)p[(size_t)y * 128 + 64 + x] +
         (double)p[(size_t)(128 + y) * 128 + x] + (double)p[(size_t)(128 + y) * 128 + 64 + x];
  }
  const int np = d.npool;
  const int a = d.gnew[x0 + x], bb = d.gtgt[y0 + y];
  // a pair of two new columns is computed twice; only the one with a <= bb writes it, so
  // that the stored Gram is symmetric and independent of the order of the writes
  const int nnew = d.meta[META_NNEW];
  bool b_new = false;
  for (int z = 0; z < nnew; ++z) b_new |= d.gnew[z] == bb;
  if (b_new && a > bb) return;
  d.Gp[a + (size_t)bb * np] = v;
  d.Gp[bb + (size_t)a * np] = v;
}

// Gram of every (new, target) pool-slot pair, in tiles of 64 x 128.  The counts live on the
// device, so every tile is launched for the largest possible counts and exits early.
// Basis Gram of every new element against every target in one pass over the pool.  The
// targets (new elements first) are staged per chunk as one B tile of 64-target blocks (64 hi
// rows, then the 64 lo rows of the same targets); the A operand of the MMA is the 128-row
// block holding new elements x0 .. x0+63, read from the same tile.  D[L][c] accumulates in
// TMEM over this CTA's chunks; the reduction adds the split-K partials and the four
// hi/lo products.  Requires ntgt <= 256 (2t <= 256).
constexpr int kGramRowsMax = 512;            // 4 blocks x (64 hi + 64 lo) rows

// Both 64-blocks of new elements (nnew > 64) in one pass over the targets: their two
// accumulators, 128 lanes x nbrows columns each, fit the 512 TMEM columns together when
// nbrows = 128 ceil(ntgt / 64) <= 256.
__device__ __forceinline__ bool gram_merged(int nnew, int ntgt) {
  return nnew > 64 && nnew <= 128 && ntgt <= 128;
}

// Warp roles of the basis Gram: warp 0 issues the MMAs, warps 1..16 convert, warps 17..28 load.
constexpr int kGramLoadWarp = 1 + kProducerWarps;
constexpr int kGramLoadWarps = 12;
constexpr int kGramAllThreads = 32 * (1 + kProducerWarps + kGramLoadWarps);
constexpr int kGramMaxStages = 8;                       // barrier slots of the staging ring
constexpr uint32_t kGramStageArea = 3u * kGramRowsMax * 128u;   // 192 KB of stages

// The targets' FP32 chunks are staged by asynchronous copies: warp 17 copies each target's chunk
// to byte 256 y of the stage (target y), completing on the stage's load barrier, as soon as the
// MMAs are done with the stage; the converters read the stage, meet at a
// named barrier, and write the BF16 hi / lo rows of the MMA tile over the same bytes (the FP32
// chunk of ntgt targets and its hi + lo tile take the same room).  The stage size follows the
// device-side target count: nbrows x 128 bytes, so that smaller counts keep more chunks in
// flight (up to kGramMaxStages within kGramStageArea).
__global__ void __launch_bounds__(kGramAllThreads, 1)
tc_gram_all_kernel(Dev d, int x0, int64_t chunks_per_cta, float* __restrict__ part) {
  extern __shared__ uint8_t smem_raw[];
  const int nnew = d.meta[META_NNEW], ntgt_all = d.meta[META_NTGT];
  if (x0 >= nnew || ntgt_all <= 0) return;              // uniform over the CTA, before any TMEM use
  // both 64-blocks of new elements in one pass when their accumulators fit TMEM together
  const bool merged = gram_merged(nnew, ntgt_all);
  if (merged && x0 > 0) return;                           // done by the x0 = 0 pass
  const int nablk = (merged && x0 == 0) ? 2 : 1;
  // targets before x0 are new elements of earlier blocks, whose pairs with this block those
  // blocks' passes computed: the tile starts at target x0 (the A block is its first 128 rows)
  const int ybase = merged ? 0 : x0;
  const int ntgt = ntgt_all - ybase;
  const int nbrows = 128 * ((ntgt + 63) / 64);            // B rows in use (multiple of 128, <= 512)
  const uint32_t btile = (uint32_t)nbrows * 128u;         // >= 256 ntgt: the FP32 chunk fits
  int nstage = (int)(kGramStageArea / btile);
  if (nstage > kGramMaxStages) nstage = kGramMaxStages;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sB = base;
  const uint32_t sBar = sB + kGramStageArea;              // full[8], empty[8], loaded[8], done; slot offsets
  uint8_t* gbar = gbase + (sBar - base);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 208);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 216);
  const uint32_t bar_full0 = sBar, bar_empty0 = sBar + 64, bar_load0 = sBar + 128, bar_done = sBar + 192;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nchunks = (d.m + kChunkK - 1) / kChunkK;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_cta;
  int64_t c1 = c0 + chunks_per_cta;
  if (c1 > nchunks) c1 = nchunks;
  const int64_t nch = c1 > c0 ? c1 - c0 : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) {
      mbar_init(bar_full0 + 8 * i, 32 * kProducerWarps);
      mbar_init(bar_empty0 + 8 * i, 1);
      mbar_init(bar_load0 + 8 * i, 32 * kGramLoadWarps);   // one arrival per loader thread
    }
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      const int n1 = nbrows < 256 ? nbrows : 256, n2 = nbrows - n1;
      const uint32_t id1 = idesc_bf16(128, n1);
      const uint32_t id2 = idesc_bf16(128, n2 > 0 ? n2 : 16);
      int st = 0;
      uint32_t par = 0;
      for (int64_t c = 0; c < nch; ++c) {
        if (!mbar_wait(bar_full0 + 8 * st, par, abort_flag, d.err, d.ring_wait_limit)) break;
        tc_fence_after();
        const uint32_t bst = sB + st * btile;
        const uint64_t db1 = desc_sw128(bst);
        const uint64_t db2 = desc_sw128(bst + 256 * 128);
        for (int ab = 0; ab < nablk; ++ab) {
          // A block ab: the 128 tile rows of new elements x0 + 64 ab .. (hi, then lo); its
          // accumulator at TMEM columns ab nbrows
          const uint64_t da = desc_sw128(bst + (uint32_t)ab * 128u * 128u);
          const uint32_t dcol = tmem + (uint32_t)(ab * nbrows);
#pragma unroll
          for (int kk = 0; kk < kChunkK / 16; ++kk) {
            const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
            const uint64_t adv = (uint64_t)(kk * 2);
            tc_mma(dcol, da + adv, db1 + adv, id1, acc);
            if (n2 > 0) tc_mma(dcol + (uint32_t)n1, da + adv, db2 + adv, id2, acc);
          }
        }
        tc_commit(bar_empty0 + 8 * st);
        if (++st == nstage) { st = 0; par ^= 1u; }
      }
      tc_commit(bar_done);
    }
    __syncwarp();
  } else if (warp >= kGramLoadWarp) {
    // ---------------------------------------------------------------- loads: 16-byte async copies
    // (ntgt x 16 of them per chunk, about 13 per lane for 100 targets), each lane's completing on
    // the stage's load barrier (128 arrivals); 256-byte bulk copies, one per target, were measured
    // 2.7x slower (the copy engine's cost per transfer dominates at that size), and one loader
    // warp 1.7x slower (its issue rate).
    const int lt = threadIdx.x - 32 * kGramLoadWarp;        // loader thread 0..127
    const float* pool = (const float*)d.pool;
    int64_t* soff = reinterpret_cast<int64_t*>(gbar + 256);   // element offset of each target's slot
    for (int y = lt; y < ntgt; y += 32 * kGramLoadWarps) soff[y] = (int64_t)d.gtgt[ybase + y] * d.m_pad;
    asm volatile("bar.sync 2, %0;" ::"n"(32 * kGramLoadWarps) : "memory");
    int st = 0;
    uint32_t epar = 1u;                                   // first pass over the ring: stages start empty
    for (int64_t c = 0; c < nch; ++c) {
      // every lane waits (the same barrier and phase), so the warp leaves the loop together
      const bool okw = mbar_wait(bar_empty0 + 8 * st, epar, abort_flag, d.err, d.ring_wait_limit);
      if (!__all_sync(0xffffffffu, okw)) break;
      const uint32_t dst = sB + st * btile;
      const int64_t off = (c0 + c) * kChunkK;               // < m_pad: the slot tail beyond m is zero
      for (int idx = lt; idx < ntgt * 16; idx += 32 * kGramLoadWarps) {
        const int y = idx >> 4, seg = idx & 15;
        const float* src = pool + soff[y] + off + 4 * seg;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (uint32_t)y * 256u + 16u * seg),
                     "l"(src)
                     : "memory");
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar_load0 + 8 * st) : "memory");
      if (++st == nstage) { st = 0; epar ^= 1u; }
    }
    // no copy may still be landing when the CTA exits
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- converters (warps 1..16)
    // thread pt converts, for u = 0..3, coordinates 8g..8g+7 of target y = y0t + 64 u
    const int pt = threadIdx.x - 32;
    const int g = pt & 7;
    const int y0t = pt >> 3;
    int st = 0;
    uint32_t lpar = 0;
    for (int64_t c = 0; c < nch; ++c) {
      const bool okw = mbar_wait(bar_load0 + 8 * st, lpar, abort_flag, d.err, d.ring_wait_limit);
      const uint32_t bst = sB + st * btile;
      float x[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int y = y0t + 64 * u;
        if (okw && y < ntgt) {
          const float* rp = reinterpret_cast<const float*>(gbase + (bst - base) + (uint32_t)y * 256u + 32u * g);
          const float4 a0 = *reinterpret_cast<const float4*>(rp);
          const float4 a1 = *reinterpret_cast<const float4*>(rp + 4);
          x[u][0] = a0.x; x[u][1] = a0.y; x[u][2] = a0.z; x[u][3] = a0.w;
          x[u][4] = a1.x; x[u][5] = a1.y; x[u][6] = a1.z; x[u][7] = a1.w;
        }
      }
      // every converter has read its FP32 values before any writes the tile over them; the
      // barrier also takes the AND of the waits, so that all converters leave together
      uint32_t all_ok;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\t"
          "setp.ne.u32 q, %1, 0;\n\t"
          "bar.red.and.pred p, 1, %2, q;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(all_ok)
          : "r"(okw ? 1u : 0u), "n"(32 * kProducerWarps)
          : "memory");
      if (!all_ok) break;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int y = y0t + 64 * u;
        if (y >= ntgt) continue;
        const int rhi = 128 * u + y0t;                    // hi row of target y0t + 64 u
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[u][2 * j], x[u][2 * j + 1]);
          const uint32_t hv = *reinterpret_cast<const uint32_t*>(&h2);
          hw[j] = hv;
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(x[u][2 * j] - __uint_as_float(hv << 16),
                                                          x[u][2 * j + 1] - __uint_as_float(hv & 0xFFFF0000u));
          lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
        }
        sts128(bst + sw128_off(rhi, g), hw[0], hw[1], hw[2], hw[3]);
        sts128(bst + sw128_off(rhi + 64, g), lw[0], lw[1], lw[2], lw[3]);
      }
      fence_async_smem();
      mbar_arrive(bar_full0 + 8 * st);
      if (++st == nstage) { st = 0; lpar ^= 1u; }
    }
    if (warp <= 4) {
      const bool ok = mbar_wait(bar_done, 0, abort_flag, d.err);
      tc_fence_after();
      if (ok && !*abort_flag) {
        const int quarter = warp & 3;
        const int L = 32 * quarter + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16);
        for (int cb = 0; cb < nablk * nbrows; cb += 32) {
          uint32_t r[32];
          tc_ld32(taddr + (uint32_t)cb, r);
          tc_wait_ld();
          float* o = part + ((size_t)blockIdx.x * kGramRowsMax + cb) * 128 + L;
#pragma unroll
          for (int j = 0; j < 32; ++j) o[(size_t)j * 128] = (nch > 0) ? __uint_as_float(r[j]) : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// One CTA per target y, 256 threads: thread (j, x) adds the partials of blocks b = j (mod 4) in
// order; the four sums are combined in the fixed order j = 0..3.  G(new x0 + x, target y).
__global__ void __launch_bounds__(256) tc_gram_all_reduce_kernel(Dev d, const float* __restrict__ part, int nblk,
                                                                 int x0) {
  __shared__ double red[4][64];
  const int nnew = d.meta[META_NNEW], ntgt = d.meta[META_NTGT];
  const int y = blockIdx.x;
  if (x0 >= nnew || y >= ntgt) return;
  const bool merged = gram_merged(nnew, ntgt);
  // a separate pass of block x0 starts its tile at target x0; in a merged pass the
  // accumulators of the second 64-block follow those of the first
  const int ybase = merged ? 0 : x0;
  if (y < ybase) return;                                  // pair computed by an earlier block's pass
  const int nx = min(64, nnew - x0);
  const int x = threadIdx.x & 63, j = threadIdx.x >> 6;
  const int cofs = (merged && x0 > 0) ? 128 * ((ntgt + 63) / 64) : 0;
  const int yl = y - ybase;
  const int chi = cofs + 128 * (yl >> 6) + (yl & 63), clo = chi + 64;
  double v = 0.0;
  if (x < nx) {
    for (int b = j; b < nblk; b += 4) {
      const float* p = part + (size_t)b * kGramRowsMax * 128;
      v += (double)p[(size_t)chi * 128 + x] + (double)p[(size_t)clo * 128 + x] +
           (double)p[(size_t)chi * 128 + 64 + x] + (double)p[(size_t)clo * 128 + 64 + x];
    }
  }
  red[j][x] = v;
  __syncthreads();
  if (j != 0 || x >= nx) return;
  const double g = ((red[0][x] + red[1][x]) + red[2][x]) + red[3][x];
  const int np = d.npool;
  const int a = d.gnew[x0 + x], bb = d.gtgt[y];
  // target y < nnew is a new element: its pair with x0 + x is computed twice; the smaller
  // new-element index writes it, so the stored Gram is symmetric and deterministic
  if (y < nnew && x0 + x > y) return;
  d.Gp[a + (size_t)bb * np] = g;
  d.Gp[bb + (size_t)a * np] = g;
}

int launch_tc_gram(const Dev& d, int nblk, float* part, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
        cudaSuccess)
      return -1;
    attr_set = true;
  }
  const int64_t nchunks = (d.m + kChunkK - 1) / kChunkK;
  int64_t per = (nchunks + nblk - 1) / nblk;
  int nk = 0;
  if (2 * d.t <= 256) {
    // one pass over the targets per 64 new elements
    static int max_smem = 0;
    if (max_smem == 0) {
      int dev = 0, v = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
          cudaFuncSetAttribute(tc_gram_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, v) != cudaSuccess)
        return -1;
      max_smem = v;
    }
    // align slack + barriers + the targets' slot offsets (256 x 8 bytes) + stages
    const size_t smem = 1024 + 256 + 2048 + (size_t)kGramStageArea;
    if (smem > (size_t)max_smem) return -1;
    for (int x0 = 0; x0 < d.t; x0 += 64) {
      tc_gram_all_kernel<<<nblk, kGramAllThreads, smem, st>>>(d, x0, per, part);
      tc_gram_all_reduce_kernel<<<2 * d.t, 256, 0, st>>>(d, part, nblk, x0);
      nk += 2;
    }
    return nk;
  }
  for (int x0 = 0; x0 < d.t; x0 += 64)
    for (int y0 = 0; y0 < 2 * d.t; y0 += 128) {
      tc_gram_kernel<<<nblk, kGramThreads, kSmemBytes, st>>>(d, x0, y0, per, part);
      tc_gram_reduce_kernel<<<(64 * 128 + 255) / 256, 256, 0, st>>>(d, part, nblk, x0, y0);
      nk += 2;
    }
  return nk;
}

int tc_smem_bytes() { return kSmemBytes; }

// ---------------------------------------------------------------- right sketch on tensor cores
// Y(:, rb .. rb + rl - 1) += A_group W(:, rb .. rb + rl - 1) for a group of G <= 64 FP32 columns
// and a +-1 W (the optional right sketch; not part of the paper's method).  MMA mapping
// (kind::f16, FP32 accumulation): M = 128 coordinates of a tile, N = nW >= rl sketch columns
// (a multiple of 16, <= 256), K = the group's columns, split a = hi + lo: one K block of 64
// columns for the hi parts and one for the lo parts, both against the same B tile (W^T rows,
// +-1 exact in BF16).  The CTA is persistent over its tiles of 128 coordinates: 16 producer
// warps transpose each tile into the K-major A tiles (thread: one coordinate, 16 columns; every
// warp writes 32 consecutive rows of one 16-byte chunk, conflict-free), the MMA warp fills one of
// two TMEM accumulators, and the same 16 warps then add the accumulator to Y (lane = coordinate:
// coalesced 128-byte rows of each Y column) -- so Y is read and written once per group, the
// bound of this update (2 x 4 m l bytes per group against 4 m G of data).
constexpr int kRtTile = 128;                          // coordinates per tile
constexpr int kRtStages = 3;
constexpr uint32_t kRtATile = 128u * 128u;            // 128 rows x 64 BF16
constexpr uint32_t kRtBTile = 256u * 128u;            // up to 256 W rows x 64 BF16

__global__ void __launch_bounds__(kThreads, 1)
tc_right_kernel(Dev d, Cols cols, int G, const float* __restrict__ Wg, int lw, int rb, int rl, int nW) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sW = base;                                         // B tile
  const uint32_t sA = sW + kRtBTile;                                // stages: A hi, A lo
  const uint32_t sBar = sA + (uint32_t)kRtStages * 2u * kRtATile;   // full[3], empty[3], tfull[2], tempty[2]
  uint8_t* gbar = gbase + (sBar - base);
  const float** colptr = reinterpret_cast<const float**>(gbar + 128);   // the group's 64 column pointers
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 96);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 104);
  const uint32_t bar_full0 = sBar, bar_empty0 = sBar + 24, bar_tfull0 = sBar + 48, bar_tempty0 = sBar + 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m = d.m, ldy = d.m_pad;
  const int64_t ntiles = (m + kRtTile - 1) / kRtTile;
  const int64_t nmine = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kRtStages; ++i) {
      mbar_init(bar_full0 + 8 * i, 32 * kProducerWarps);
      mbar_init(bar_empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar_tfull0 + 8 * i, 1);
      mbar_init(bar_tempty0 + 8 * i, 32 * kProducerWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 64) colptr[threadIdx.x] = threadIdx.x < G ? cols.p[threadIdx.x] : nullptr;
  // the B tile: row n = sketch column rb + n, K entry q = W(q, rb + n), zero past G and rl
  for (int idx = threadIdx.x; idx < nW * 8; idx += blockDim.x) {
    const int n = idx >> 3, ch = idx & 7;            // 16-byte chunk ch: columns 8 ch .. 8 ch + 7
    uint32_t w4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int q0 = 8 * ch + 2 * e;
      const float v0 = (q0 < G && n < rl) ? Wg[q0 * lw + rb + n] : 0.f;
      const float v1 = (q0 + 1 < G && n < rl) ? Wg[(q0 + 1) * lw + rb + n] : 0.f;
      w4[e] = pack_bf16(v0, v1);
    }
    sts128(sW + sw128_off(n, ch), w4[0], w4[1], w4[2], w4[3]);
  }
  fence_async_smem();
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t id = idesc_bf16(128, nW);
      const uint64_t db = desc_sw128(sW);
      int st = 0;
      uint32_t par = 0;
      for (int64_t t = 0; t < nmine; ++t) {
        const int buf = (int)(t & 1);
        const uint32_t tpar = (uint32_t)(((t >> 1) & 1) ^ 1);   // the buffers start empty
        if (!mbar_wait(bar_tempty0 + 8 * buf, tpar, abort_flag, d.err, d.ring_wait_limit)) break;
        if (!mbar_wait(bar_full0 + 8 * st, par, abort_flag, d.err, d.ring_wait_limit)) break;
        tc_fence_after();
        const uint32_t sst = sA + (uint32_t)st * 2u * kRtATile;
        const uint32_t dcol = tmem + (uint32_t)(256 * buf);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
          const uint64_t da = desc_sw128(sst + (uint32_t)kb * kRtATile);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 2);            // +32 bytes along K
            tc_mma(dcol, da + adv, db + adv, id, (kb > 0 || kk > 0) ? 1u : 0u);
          }
        }
        tc_commit(bar_empty0 + 8 * st);
        tc_commit(bar_tfull0 + 8 * buf);
        if (++st == kRtStages) { st = 0; par ^= 1u; }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- producers, then epilogue
    const int pt = threadIdx.x - 32;                  // 0..511
    const int rr = pt & 127;                          // coordinate (A row) of this thread
    const int qb = pt >> 7;                           // columns 16 qb .. 16 qb + 15
    const int quarter = warp & 3, cq = (warp - 1) >> 2;  // TMEM lanes 32 quarter .., column chunks cq, cq + 4, ..
    int st = 0;
    uint32_t ppar = 1u;                               // stages start empty
    bool ok = true;
    auto produce = [&](int64_t t) -> bool {
      if (!mbar_wait(bar_empty0 + 8 * st, ppar, abort_flag, d.err, d.ring_wait_limit)) return false;
      const int64_t i = (int64_t)(blockIdx.x + t * gridDim.x) * kRtTile + rr;
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int q = 16 * qb + e;
        v[e] = (q < G && i < m) ? __ldcs(colptr[q] + i) : 0.f;
      }
      const uint32_t sst = sA + (uint32_t)st * 2u * kRtATile;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {                // chunk 2 qb + h2: columns 16 qb + 8 h2 ..
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float x0 = v[8 * h2 + 2 * e], x1 = v[8 * h2 + 2 * e + 1];
          const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
          const uint32_t hv = *reinterpret_cast<const uint32_t*>(&hb);
          hw[e] = hv;
          const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - __uint_as_float(hv << 16),
                                                          x1 - __uint_as_float(hv & 0xFFFF0000u));
          lw[e] = *reinterpret_cast<const uint32_t*>(&lb);
        }
        sts128(sst + sw128_off(rr, 2 * qb + h2), hw[0], hw[1], hw[2], hw[3]);
        sts128(sst + kRtATile + sw128_off(rr, 2 * qb + h2), lw[0], lw[1], lw[2], lw[3]);
      }
      fence_async_smem();
      mbar_arrive(bar_full0 + 8 * st);
      if (++st == kRtStages) { st = 0; ppar ^= 1u; }
      return true;
    };
    auto epilogue = [&](int64_t t) -> bool {
      const int buf = (int)(t & 1);
      const uint32_t fpar = (uint32_t)((t >> 1) & 1);
      if (!mbar_wait(bar_tfull0 + 8 * buf, fpar, abort_flag, d.err, d.ring_wait_limit)) return false;
      tc_fence_after();
      const int64_t i = (int64_t)(blockIdx.x + t * gridDim.x) * kRtTile + 32 * quarter + lane;
      const uint32_t taddr = tmem + (uint32_t)(256 * buf) + ((uint32_t)(32 * quarter) << 16);
      float* __restrict__ Y = reinterpret_cast<float*>(d.Y) + (int64_t)rb * ldy;
      for (int cb = 16 * cq; cb < nW; cb += 64) {     // 16 columns per load; 4 warps share a lane quarter
        uint32_t r[16];
        tc_ld16(taddr + (uint32_t)cb, r);
        tc_wait_ld();
        if (i < ldy) {                                 // rows m .. m_pad - 1 of Y stay 0 (the data is 0 there)
          float y[16];                                 // 16 loads in flight, then their 16 stores
#pragma unroll
          for (int j = 0; j < 16; ++j) y[j] = cb + j < rl ? Y[(int64_t)(cb + j) * ldy + i] : 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < rl) Y[(int64_t)(cb + j) * ldy + i] = y[j] + __uint_as_float(r[j]);
        }
      }
      tc_fence_before();
      mbar_arrive(bar_tempty0 + 8 * buf);
      return true;
    };
    // tile t's epilogue runs after tile t + 1 is staged, so that the MMAs of t + 1 overlap it
    for (int64_t t = 0; t < nmine && ok; ++t) {
      ok = produce(t);
      if (ok && t >= 1) ok = epilogue(t - 1);
    }
    if (ok && nmine >= 1) epilogue(nmine - 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

int launch_tc_right(const Dev& d, const void* const* colp, int ncols, const float* W, int lw, cudaStream_t st) {
  const size_t smem = 1024 + kRtBTile + (size_t)kRtStages * 2 * kRtATile + 128 + 512;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc_right_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    attr = true;
  }
  if (ncols > 64) return -1;
  Cols c;
  for (int q = 0; q < 128; ++q) c.p[q] = q < ncols ? (const float*)colp[q] : nullptr;
  const int64_t ntiles = (d.m + kRtTile - 1) / kRtTile;
  const int grid = (int)(ntiles < d.n_sm ? ntiles : d.n_sm);
  int nk = 0;
  for (int rb = 0; rb < d.right_l; rb += 256) {
    const int rl = d.right_l - rb < 256 ? d.right_l - rb : 256;
    const int nW = (rl + 15) / 16 * 16;
    tc_right_kernel<<<grid, kThreads, smem, st>>>(d, c, ncols, W, lw, rb, rl, nW);
    ++nk;
  }
  return nk;
}

// ---------------------------------------------------------------- FP8 (E4M3, block-scaled) ingest
// The same sketch S(:, q) = Omega a_q with the data quantized to E4M3 with one power-of-two scale
// per 32 consecutive coordinates of a column (the microscaling layout: UE8M0 exponents), as one
// term (hi) or two (hi + lo, lo quantizing the residual a - hi with its own block scales).
// Omega's +-1 entries are exact in E4M3.  MMA: tcgen05.mma kind::mxf8f6f4 with block scaling
// (scale_vec::1X: one scale per row and 32-element K step), A = the 128 data rows (hi rows
// 0..63, lo rows 64..127), B = the Omega rows, FP32 accumulation in TMEM.
// A chunk is 128 coordinates (one 128-byte E4M3 row, four K steps of 32).  The A scales of a
// chunk live in TMEM: row m's four exponent bytes (one per K step, selected by the
// instruction's scale-factor id) at lane m, column sfa + m / 32 -- each lane quarter's 32 rows in
// its own column.  Four scale-writer warps (one per lane quarter, no other work) copy them from
// the producers' shared-memory staging into TMEM once every producer has staged its column's
// scales (an mbarrier, so that every wait stays bounded), then release the stage to the MMA;
// the producers never wait for them, so the ring keeps its overlap.  The B scales are 1.0
// everywhere, written once.
constexpr int kChunk8 = 128;                // coordinates per chunk
constexpr int kSfbCol = 504;                // TMEM columns 504..511: B scales (all 1.0)
constexpr int kSfaCol0 = 488;               // TMEM columns 488 + 4 st .. + 3: A scales of ring stage st
constexpr int kMaxStages8 = 3;
constexpr int kScaleBytes = 128 * 4;        // staged A scale words of one stage
constexpr int kWriterWarps = 4;             // warps 17..20: the A scales into TMEM
constexpr int kThreads8 = 32 * (1 + kProducerWarps + kWriterWarps);

__device__ __forceinline__ void tc_st32x1(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_mma_mx8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t sfa, uint32_t sfb, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accum)
      : "memory");
}
// Instruction descriptor, kind::mxf8f6f4 with block scaling: A and B E4M3 (format 0), K-major,
// UE8M0 scales (bit 23), N >> 3 at bit 17, M >> 4 at bit 24, scale-factor ids of A (bits 29-30)
// and B (bits 4-5).
__host__ __device__ constexpr uint32_t idesc_mx8(int M, int N, int a_sf_id) {
  return ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24) | ((uint32_t)a_sf_id << 29);
}
// Block exponent X of a 32-coordinate block: the smallest 2^X with amax / 2^X <= 448 (E4M3's
// largest finite value), 0 for an all-zero block; clamped to [-127, 126] (UE8M0's range; only
// blocks below 2^-118 in magnitude reach the lower clamp).  amax = (1 + f) 2^e with f the
// fraction: amax / 448 = (1 + f) / 1.75 * 2^(e - 8), at most 2^(e - 8) iff 1 + f <= 1.75.
__device__ __forceinline__ int e4m3_block_exp(float amax) {
  const uint32_t b = __float_as_uint(amax);
  const int ef = (int)((b >> 23) & 0xFFu);
  if (!(amax > 0.f)) return 0;
  int x;
  if (ef == 0) {
    x = -127;                                    // subnormal amax: below every representable scale
  } else {
    x = ef - 127 - 8 + (((b & 0x7FFFFFu) > 0x600000u) ? 1 : 0);
  }
  return x < -127 ? -127 : (x > 126 ? 126 : x);
}
// 2^X as a float, X in [-127, 126] (2^-127 is subnormal).
__device__ __forceinline__ float pow2f(int x) {
  return x >= -126 ? __uint_as_float((uint32_t)(x + 127) << 23) : __uint_as_float(0x00400000u);
}
// Quantize 16 values to E4M3 at scale 2^X (round to nearest even, satfinite): 16 bytes in
// coordinate order, and the quantized values scaled back (exact in FP32).
__device__ __forceinline__ void e4m3_quant16(const float (&x)[16], int X, uint32_t (&w)[4], float (&back)[16]) {
  const float inv = pow2f(-X), sc = pow2f(X);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const __nv_fp8x2_storage_t p =
        __nv_cvt_float2_to_fp8x2(make_float2(x[2 * j] * inv, x[2 * j + 1] * inv), __NV_SATFINITE, __NV_E4M3);
    const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(p, __NV_E4M3);
    __half_raw h0, h1;
    h0.x = hr.x;
    h1.x = hr.y;
    back[2 * j] = __half2float(__half(h0)) * sc;
    back[2 * j + 1] = __half2float(__half(h1)) * sc;
    const uint32_t pv = (uint32_t)p;
    if (j & 1) w[j >> 1] |= pv << 16; else w[j >> 1] = pv;
  }
}
// Four E4M3 +-1 Omega entries (coordinates 4j .. 4j+3 of a 32-coordinate word of the counter-based
// bits): coordinate e takes bit 15 - e/2 (even e) or 31 - e/2 (odd e), set = -1; after a shift by
// 2j the four bits sit at 15, 31, 14, 30 and a byte permutation puts them at the sign bits.
__device__ __forceinline__ uint32_t omega_e4m3x4(uint32_t w, int j) {
  const uint32_t x = w << (2 * j);
  const uint32_t y = x & 0x80008000u;
  const uint32_t z = (x << 1) & 0x80008000u;
  return __byte_perm(y, z, 0x7531) | 0x38383838u;
}

__global__ void __launch_bounds__(kThreads8, 1)
tc_ingest_fp8_kernel(Dev d, Cols cols, int ncols, int split, int count, int nrows16, int n1, int n2,
                     int64_t chunks_per_cta, int vec, float* __restrict__ part, double* __restrict__ npart,
                     int nstage, uint32_t btile) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  // ring stage st: A tile (16 KB) at sA + st * kATile, B tile at sB + st * btile, staged A
  // scale words at sS + st * kScaleBytes
  const uint32_t sA = base;
  const uint32_t sB = base + (uint32_t)nstage * kATile;
  const uint32_t sS = sB + (uint32_t)nstage * btile;
  uint32_t* scale_stage = reinterpret_cast<uint32_t*>(gbase + (sS - base));
  const uint32_t sBar = sS + (uint32_t)nstage * kScaleBytes;   // full[4], empty[4], done, ready[4]
  uint8_t* gbar = gbase + (sBar - base);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 112);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbar + 120);
  const uint32_t bar_full0 = sBar, bar_empty0 = sBar + 32, bar_done = sBar + 64, bar_ready0 = sBar + 72;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nchunks = (d.m + kChunk8 - 1) / kChunk8;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_cta;
  int64_t c1 = c0 + chunks_per_cta;
  if (c1 > nchunks) c1 = nchunks;
  const int64_t nch = c1 > c0 ? c1 - c0 : 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nstage; ++i) {
      mbar_init(bar_full0 + 8 * i, 32 * (kProducerWarps + kWriterWarps));
      mbar_init(bar_empty0 + 8 * i, 1);
      mbar_init(bar_ready0 + 8 * i, 32 * kProducerWarps);
    }
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // the scale writers: warps 17..20 cover the lane quarters 1, 2, 3, 0
  const bool writer = warp > kProducerWarps;
  const int quarter = warp & 3;
  if (writer) {
    const uint32_t lq = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) tc_st32x1(lq + (uint32_t)(kSfbCol + cc), 0x7F7F7F7Fu);   // 2^0
    tc_wait_st();
    tc_fence_before();
  }

  if (warp == 0) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      int st = 0;
      uint32_t par = 0;
      for (int64_t c = 0; c < nch; ++c) {
        if (!mbar_wait(bar_full0 + 8 * st, par, abort_flag, d.err, d.ring_wait_limit)) break;
        tc_fence_after();
        const uint64_t da = desc_sw128(sA + st * kATile);
        const uint64_t db1 = desc_sw128(sB + st * btile);
        const uint64_t db2 = desc_sw128(sB + st * btile + 256 * 128);
        const uint32_t sfa = tmem + (uint32_t)(kSfaCol0 + 4 * st);
        const uint32_t sfb = tmem + (uint32_t)kSfbCol;
#pragma unroll
        for (int kk = 0; kk < kChunk8 / 32; ++kk) {
          const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
          const uint64_t adv = (uint64_t)(kk * 2);            // +32 bytes along K
          tc_mma_mx8(tmem, da + adv, db1 + adv, idesc_mx8(128, n1, kk), sfa, sfb, acc);
          if (n2 > 0) tc_mma_mx8(tmem + (uint32_t)n1, da + adv, db2 + adv, idesc_mx8(128, n2, kk), sfa, sfb, acc);
        }
        tc_commit(bar_empty0 + 8 * st);
        if (++st == nstage) { st = 0; par ^= 1u; }
      }
      tc_commit(bar_done);
    }
    __syncwarp();
  } else if (writer) {
    // ---------------------------------------------------------------- A scales into TMEM
    int st = 0;
    uint32_t par = 0;
    const uint32_t lq = tmem + ((uint32_t)(32 * quarter) << 16);
    for (int64_t c = 0; c < nch; ++c) {
      if (!__all_sync(0xffffffffu, mbar_wait(bar_ready0 + 8 * st, par, abort_flag, d.err, d.ring_wait_limit))) break;
      const uint32_t v = scale_stage[(size_t)st * 128 + 32 * quarter + lane];
      tc_st32x1(lq + (uint32_t)(kSfaCol0 + 4 * st + quarter), v);
      tc_wait_st();
      tc_fence_before();
      mbar_arrive(bar_full0 + 8 * st);
      if (++st == nstage) { st = 0; par ^= 1u; }
    }
  } else {
    // ---------------------------------------------------------------- producers
    // thread pt moves coordinates 16g .. 16g+15 of every chunk of column q = pt / 8 (g = pt % 8:
    // one 16-byte E4M3 unit of the 128-byte A row; 32-coordinate block g / 2 shared with the
    // neighbouring lane) and expands Omega row pt (one counter-based call per chunk).
    const int pt = threadIdx.x - 32;
    const int q = pt >> 3, g = pt & 7;
    const bool has_col = q < ncols;
    const float* src = has_col ? cols.p[q] : nullptr;
    float* dstp = has_col ? (float*)d.pool + (int64_t)d.dslot[count + q] * d.m_pad : nullptr;
    const int r0 = pt;
    const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
    float ks = 0.f, kc = 0.f;
    float bufA[16], bufB[16];
    auto load_chunk = [&](int64_t c, float (&v)[16]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;
      if (has_col && c < nch) {
        const int64_t i = (c0 + c) * kChunk8 + 16 * g;
        if (vec && i + 16 <= d.m) {
          const float4* s4 = reinterpret_cast<const float4*>(src + i);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 t = __ldcs(s4 + j);
            v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = (i + j < d.m) ? src[i + j] : 0.f;
        }
      }
      if (has_col && g == 0 && vec && c + kL2Ahead < nch && (c0 + c + kL2Ahead + 1) * kChunk8 <= d.m)
        prefetch_l2(src + (c0 + c + kL2Ahead) * kChunk8, kChunk8 * 4);
    };
    int pst = 0;
    uint32_t ppar = 1u;                       // first pass over the ring: stages start empty
    auto process = [&](int64_t c, const float (&x)[16]) -> bool {
      const int st = pst;
      // warp-uniform outcome of the bounded wait: the shuffles below need every lane
      if (!__all_sync(0xffffffffu, mbar_wait(bar_empty0 + 8 * st, ppar, abort_flag, d.err, d.ring_wait_limit))) return false;
      const int64_t cg = c0 + c;
      const uint32_t ast = sA + st * kATile;
      if (has_col) {
        const int64_t i0 = cg * kChunk8 + 16 * g;
        if (i0 + 16 <= d.m && vec) {
          float4* o = reinterpret_cast<float4*>(dstp + i0);
#pragma unroll
          for (int j = 0; j < 4; ++j) __stcs(o + j, make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]));
        } else {
          for (int j = 0; j < 16; ++j) if (i0 + j < d.m) dstp[i0 + j] = x[j];
        }
        float s2 = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) s2 = fmaf(x[j], x[j], s2);
        const float y = s2 - kc;
        const float tsum = ks + y;
        kc = (tsum - ks) - y;
        ks = tsum;
      }
      // block scales and E4M3 terms (every lane takes part in the shuffles; rows of absent
      // columns are not stored)
      float am = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) am = fmaxf(am, fabsf(x[j]));
      am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 1));
      const int Xh = e4m3_block_exp(am);
      uint32_t wh[4], wl[4];
      float back[16];
      e4m3_quant16(x, Xh, wh, back);
      float rres[16];
      float amr = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) { rres[j] = x[j] - back[j]; amr = fmaxf(amr, fabsf(rres[j])); }
      amr = fmaxf(amr, __shfl_xor_sync(0xffffffffu, amr, 1));
      const int Xl = e4m3_block_exp(amr);
      e4m3_quant16(rres, Xl, wl, back);
      // the four block exponents of the column's row, one byte per K step, gathered over its 8 lanes
      uint32_t sh = (uint32_t)(Xh + 127) << (8 * (g >> 1));
      uint32_t sl = split ? (uint32_t)(Xl + 127) << (8 * (g >> 1)) : 0x7Fu << (8 * (g >> 1));
      sh |= __shfl_xor_sync(0xffffffffu, sh, 2);
      sh |= __shfl_xor_sync(0xffffffffu, sh, 4);
      sl |= __shfl_xor_sync(0xffffffffu, sl, 2);
      sl |= __shfl_xor_sync(0xffffffffu, sl, 4);
      uint32_t* ss = scale_stage + (size_t)st * 128;
      if (g == 0) { ss[q] = has_col ? sh : 0x7F7F7F7Fu; ss[64 + q] = has_col ? sl : 0x7F7F7F7Fu; }
      if (has_col) {
        sts128(ast + sw128_off(q, g), wh[0], wh[1], wh[2], wh[3]);
        if (split) sts128(ast + sw128_off(64 + q, g), wl[0], wl[1], wl[2], wl[3]);
      }
      if (r0 < nrows16) {
        const uint32_t bst = sB + st * btile;
        const u32x4 w = philox4x32_10((uint32_t)(cg + (d.row_offset >> 7)), (uint32_t)r0, kTagRademacher, 0, k0, k1);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t ww = words[u >> 1];
          const int j0 = 4 * (u & 1);             // 4-coordinate groups 4 j0 .. of the 32-bit word
          sts128(bst + sw128_off(r0, u), omega_e4m3x4(ww, j0), omega_e4m3x4(ww, j0 + 1), omega_e4m3x4(ww, j0 + 2),
                 omega_e4m3x4(ww, j0 + 3));
        }
      }
      fence_async_smem();
      mbar_arrive(bar_ready0 + 8 * st);
      mbar_arrive(bar_full0 + 8 * st);
      if (++pst == nstage) { pst = 0; ppar ^= 1u; }
      return true;
    };
    load_chunk(0, bufA);
    load_chunk(1, bufB);
    for (int64_t c = 0; c < nch; c += 2) {
      if (!process(c, bufA)) break;
      load_chunk(c + 2, bufA);
      if (c + 1 < nch) {
        if (!process(c + 1, bufB)) break;
        load_chunk(c + 3, bufB);
      }
    }
    double nrm = (double)ks - (double)kc;
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 1);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 2);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, 4);
    if (has_col && g == 0) npart[(size_t)blockIdx.x * 128 + q] = nrm;

    // ---------------------------------------------------------------- epilogue (warps 1..4)
    if (warp <= 4) {
      const bool ok = mbar_wait(bar_done, 0, abort_flag, d.err);
      tc_fence_after();
      if (ok && !*abort_flag) {
        const int qtr = warp & 3;
        const int L = 32 * qtr + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * qtr) << 16);
        for (int cb = 0; cb < nrows16; cb += 32) {
          uint32_t r[32];
          tc_ld32(taddr + (uint32_t)cb, r);
          tc_wait_ld();
          float* o = part + ((size_t)blockIdx.x * nrows16 + cb) * 128 + L;
          const int jn = (nrows16 - cb < 32) ? nrows16 - cb : 32;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < jn) o[(size_t)j * 128] = (nch > 0) ? __uint_as_float(r[j]) : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- multi-pass sketch (row slices, gradient mode)
constexpr int kMaxSliceRows = 512;          // TMEM accumulator columns of one CTA

// Rows [rlo, rlo + gridDim.x) of the destination column block: dst(rlo + r, col0 + q) = the sum
// over the split-K blocks of the hi (and lo) partial rows r of column q, blocks b = j (mod 4)
// summed in order by thread (j, q) and the four sums added in the fixed order j = 0..3.
__global__ void __launch_bounds__(256) tc_reduce_rows_kernel(const float* __restrict__ part, int nblk, int ncols,
                                                             int split, int nrows16, int rlo,
                                                             double* __restrict__ dst, int64_t ldd, int64_t col0) {
  __shared__ double red[4][64];
  const int q = threadIdx.x & 63, j = threadIdx.x >> 6;
  const int r = blockIdx.x;
  double v = 0.0;
  if (q < ncols) {
    for (int b = j; b < nblk; b += 4) {
      const float* p = part + ((size_t)b * nrows16 + r) * 128;
      v += (double)p[q];
      if (split) v += (double)p[64 + q];
    }
  }
  red[j][q] = v;
  __syncthreads();
  if (j == 0 && q < ncols)
    dst[(size_t)(col0 + q) * ldd + rlo + r] = ((red[0][q] + red[1][q]) + red[2][q]) + red[3][q];
}

// The group's squared norms (split-K blocks in order, one thread per column): with out ==
// nullptr added to ||A_obs||^2 and to the leverage norm in column order, else stored in out.
__global__ void __launch_bounds__(128) tc_norms_kernel(Dev d, const double* __restrict__ npart, int nblk, int ncols,
                                                      double* out) {
  __shared__ double nv[128];
  const int c = threadIdx.x;
  if (c < ncols) {
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += npart[(size_t)b * 128 + c];
    if (out) out[c] = v;
    nv[c] = v;
  }
  __syncthreads();
  if (out || c != 0) return;
  for (int q = 0; q < ncols; ++q) {
    const double v = nv[q];
    if (d.gnorm) {                            // row shard: summed over the shards first
      d.gnorm[q] = v;
      continue;
    }
    if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
    d.fro2[0] += v;
    d.fro2[1] += v;
  }
}

// One entry of G a with grad_stencil's weights (central inside, one-sided at either end of the
// line of length len, position c along it, neighbours st apart) in the native path's FP32
// arithmetic and order: the centre product first, then the lower and the upper neighbour.
__device__ __forceinline__ float stencil_fp32(const float* __restrict__ a, int64_t i, int64_t st, int c, int len) {
  if (c == 0) {
    float v = -1.0f * a[i];
    v += 1.0f * a[i + st];
    return v;
  }
  if (c == len - 1) {
    float v = 1.0f * a[i];
    v += -1.0f * a[i - st];
    return v;
  }
  float v = 0.0f * a[i];
  v += -0.5f * a[i - st];
  v += 0.5f * a[i + st];
  return v;
}

// Gradient mode (Sec. 3.4, Eqs. 38-43): the stacked gradient fields G a_q (2m entries each, the
// x then the y differences of every field) into g (column q at g + q ldg).  A CTA takes one grid
// line (field f, row y) of one column at a time, so an entry's position along its line (x) and
// down its field (y) come from the loop indices: no division per entry.  With vec (16-byte
// aligned columns, nx a multiple of 4) a thread takes four consecutive entries of the line: one
// 16-byte load of the line and of each neighbouring line, the two neighbours along the line from
// L1, 16-byte stores; otherwise one entry per thread.
__global__ void __launch_bounds__(256) grad_field_kernel(Dev d, Cols c, int ncols, float* __restrict__ g, int64_t ldg,
                                                         int vec) {
  const int nx = d.nx, ny = d.ny;
  const int lines = d.nfields * ny;               // grid lines of one column (m = lines nx)
  const int64_t nline = (int64_t)lines * ncols;
  for (int64_t lb = blockIdx.x; lb < nline; lb += gridDim.x) {
    const int q = (int)(lb / lines);
    const int line = (int)(lb - (int64_t)q * lines);
    const int y = line % ny;
    const float* a = c.p[q];
    const int64_t i0 = (int64_t)line * nx;
    float* gx = g + (size_t)q * ldg + i0;         // x differences: entries i0 .. i0 + nx - 1
    float* gy = gx + d.m;                         // y differences: entries m + i0 ..
    if (vec) {
      for (int x = 4 * threadIdx.x; x < nx; x += 4 * blockDim.x) {
        const float4 cv = *reinterpret_cast<const float4*>(a + i0 + x);
        const float v[4] = {cv.x, cv.y, cv.z, cv.w};
        const float left = x > 0 ? a[i0 + x - 1] : 0.f;          // read only where used
        const float right = x + 4 < nx ? a[i0 + x + 4] : 0.f;
        float ox[4], oy[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int xe = x + e;
          const float lo = e > 0 ? v[e - 1] : left, hi = e < 3 ? v[e + 1] : right;
          // grad_stencil's weights in the native path's FP32 order (centre, lower, upper)
          if (xe == 0) { float t = -1.0f * v[e]; t += 1.0f * hi; ox[e] = t; }
          else if (xe == nx - 1) { float t = 1.0f * v[e]; t += -1.0f * lo; ox[e] = t; }
          else { float t = 0.0f * v[e]; t += -0.5f * lo; t += 0.5f * hi; ox[e] = t; }
        }
        const float4 dn = y > 0 ? *reinterpret_cast<const float4*>(a + i0 + x - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 up = y < ny - 1 ? *reinterpret_cast<const float4*>(a + i0 + x + nx) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float vd[4] = {dn.x, dn.y, dn.z, dn.w}, vu[4] = {up.x, up.y, up.z, up.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (y == 0) { float t = -1.0f * v[e]; t += 1.0f * vu[e]; oy[e] = t; }
          else if (y == ny - 1) { float t = 1.0f * v[e]; t += -1.0f * vd[e]; oy[e] = t; }
          else { float t = 0.0f * v[e]; t += -0.5f * vd[e]; t += 0.5f * vu[e]; oy[e] = t; }
        }
        *reinterpret_cast<float4*>(gx + x) = make_float4(ox[0], ox[1], ox[2], ox[3]);
        *reinterpret_cast<float4*>(gy + x) = make_float4(oy[0], oy[1], oy[2], oy[3]);
      }
    } else {
      for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        gx[x] = stencil_fp32(a, i0 + x, 1, x, nx);
        gy[x] = stencil_fp32(a, i0 + x, nx, y, ny);
      }
    }
  }
}

// Leverage sketch columns n_obs + q: the s left rows of the sketch plus Omega_g (G a_q), and
// ||G a_q||^2 added to the leverage norm in column order.
__global__ void lev_combine_kernel(Dev d, int ncols, int64_t n_obs) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < ncols * d.s) {
    const int q = idx / d.s, r = idx % d.s;
    d.Slev[(size_t)(n_obs + q) * d.lev_ld + r] = d.S[(size_t)(n_obs + q) * d.rows + r] + d.glev[(size_t)q * d.s + r];
  }
  if (idx == 0) {
    for (int q = 0; q < ncols; ++q) {
      const double v = d.gnorm2[q];
      if (!isfinite(v)) atomicOr(d.err, ERR_NONFINITE);
      d.fro2[1] += v;
    }
  }
}

// One pass of the BF16 tensor-core sketch over rows [ps.rlo, ps.rlo + nrows) of the test matrix.
static int tc_pass(const Dev& d, const Cols& c, int ncols, int split, int count, TcPass ps, int nrows, int vec,
                   int nblk, float* part, double* npart, int max_smem, cudaStream_t st) {
  const int nrows16 = (nrows + 15) / 16 * 16;
  if (nrows16 > kMaxSliceRows) return -1;
  const int n1 = nrows16 < 256 ? nrows16 : 256;
  const int n2 = nrows16 - n1;
  const int64_t nchunks = (ps.len + kChunkK - 1) / kChunkK;
  int64_t per = (nchunks + nblk - 1) / nblk;
  per = (per + 1) / 2 * 2;                      // even: Philox words are shared by chunk pairs
  // as many ring stages as fit (align slack + barrier block + stages)
  const uint32_t btile = (uint32_t)nrows16 * 128u;
  const int stage_bytes = kATile + (int)btile;
  int nstage = (max_smem - 1024 - 128) / stage_bytes;
  if (nstage > kMaxStages) nstage = kMaxStages;
  if (nstage < 2) return -1;
  const size_t smem = 1024 + 128 + (size_t)nstage * stage_bytes;
  tc_ingest_kernel<<<nblk, kThreads, smem, st>>>(d, c, ncols, split, count, nrows16, n1, n2, per, vec ? 1 : 0, part,
                                                 npart, nstage, btile, ps);
  return 0;
}

// Launch the tensor-core sketch of ncols columns; returns 0 on success.
int launch_tc_ingest(const Dev& d, const void* const* colp, int ncols, int split, int count,
                     int64_t n_obs, int nblk, float* part, double* npart, cudaStream_t st,
                     cudaEvent_t* ev, int fp8) {
  static int max_smem = 0;
  if (max_smem == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return -1;
    if (cudaFuncSetAttribute(tc_ingest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, v) != cudaSuccess ||
        cudaFuncSetAttribute(tc_ingest_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, v) != cudaSuccess)
      return -1;
    max_smem = v;
  }
  Cols c;
  bool vec = true;
  for (int q = 0; q < 128; ++q) {
    c.p[q] = q < ncols ? (const float*)colp[q] : nullptr;
    if (q < ncols && ((uintptr_t)colp[q] & 15u)) vec = false;
  }
  const int nrows16 = (d.rows + 15) / 16 * 16;
  const int n1 = nrows16 < 256 ? nrows16 : 256;
  const int n2 = nrows16 - n1;
  if (fp8) {
    // E4M3 with block scales: 128-coordinate chunks, the A scales beside each stage, the
    // accumulator below the scale columns of TMEM
    if (nrows16 > kSfaCol0) return -1;
    const int64_t nch8 = (d.m + kChunk8 - 1) / kChunk8;
    const int64_t per8 = (nch8 + nblk - 1) / nblk;
    const uint32_t btile8 = (uint32_t)nrows16 * 128u;
    const int stage8 = kATile + (int)btile8 + kScaleBytes;
    int ns8 = (max_smem - 1024 - 128) / stage8;
    if (ns8 > kMaxStages8) ns8 = kMaxStages8;
    if (ns8 < 2) return -1;
    const size_t smem8 = 1024 + 128 + (size_t)ns8 * stage8;
    if (ev) cudaEventRecord(ev[0], st);
    tc_ingest_fp8_kernel<<<nblk, kThreads8, smem8, st>>>(d, c, ncols, split, count, nrows16, n1, n2, per8,
                                                        vec ? 1 : 0, part, npart, ns8, btile8);
    if (ev) cudaEventRecord(ev[1], st);
    tc_reduce_kernel<<<d.rows + 1, 256, 0, st>>>(d, part, npart, nblk, ncols, split, nrows16, n_obs);
    return 0;
  }
  if (nrows16 <= kMaxSliceRows && !d.grad) {
    // one pass: the whole test matrix in one CTA's TMEM
    if (ev) cudaEventRecord(ev[0], st);
    if (tc_pass(d, c, ncols, split, count, TcPass{d.m, 0, kTagRademacher, 1}, d.rows, vec, nblk, part, npart,
                max_smem, st) != 0)
      return -1;
    if (ev) cudaEventRecord(ev[1], st);
    tc_reduce_kernel<<<d.rows + 1, 256, 0, st>>>(d, part, npart, nblk, ncols, split, nrows16, n_obs);
    return 0;
  }
  // Several passes over the columns: row slices of the test matrix (at most 512 rows each), then
  // in gradient mode the gradient field G a (materialized per group) sketched with Omega_g.
  if (ev) cudaEventRecord(ev[0], st);
  const int nsl = (nrows16 + kMaxSliceRows - 1) / kMaxSliceRows;
  const int per_sl = ((d.rows + nsl - 1) / nsl + 15) / 16 * 16;
  for (int sl = 0; sl < nsl; ++sl) {
    const int rlo = sl * per_sl;
    const int rc = d.rows - rlo < per_sl ? d.rows - rlo : per_sl;
    if (rc <= 0) break;
    if (tc_pass(d, c, ncols, split, count, TcPass{d.m, rlo, kTagRademacher, sl == 0 ? 1 : 0}, rc, vec, nblk, part,
                npart, max_smem, st) != 0)
      return -1;
    tc_reduce_rows_kernel<<<rc, 256, 0, st>>>(part, nblk, ncols, split, (rc + 15) / 16 * 16, rlo, d.S, d.rows,
                                                n_obs);
    if (sl == 0) tc_norms_kernel<<<1, 128, 0, st>>>(d, npart, nblk, ncols, nullptr);
  }
  if (d.grad) {
    // Omega_g (G a): the stencil writes the 2m-long gradient fields of the group into gbuf (the
    // same FP32 arithmetic as the native path), sketched like data with the gradient test matrix
    const int64_t len = 2 * d.m, ldg = d.gfield_ld;
    const int gvec = vec && d.nx % 4 == 0 && ldg % 4 == 0 && d.m % 4 == 0;
    grad_field_kernel<<<8 * d.n_sm, 256, 0, st>>>(d, c, ncols, d.gfield, ldg, gvec ? 1 : 0);
    Cols gc;
    for (int q = 0; q < 128; ++q) gc.p[q] = q < ncols ? d.gfield + (size_t)q * ldg : nullptr;
    const int s16 = (d.s + 15) / 16 * 16;
    const int gns = (s16 + kMaxSliceRows - 1) / kMaxSliceRows;
    const int gper = ((d.s + gns - 1) / gns + 15) / 16 * 16;
    for (int sl = 0; sl < gns; ++sl) {
      const int rlo = sl * gper;
      const int rc = d.s - rlo < gper ? d.s - rlo : gper;
      if (rc <= 0) break;
      if (tc_pass(d, gc, ncols, split, count, TcPass{len, rlo, kTagGradRademacher, 0}, rc, 1, nblk, part, npart,
                  max_smem, st) != 0)
        return -1;
      tc_reduce_rows_kernel<<<rc, 256, 0, st>>>(part, nblk, ncols, split, (rc + 15) / 16 * 16, rlo, d.glev, d.s,
                                                  0);
      if (sl == 0) tc_norms_kernel<<<1, 128, 0, st>>>(d, npart, nblk, ncols, d.gnorm2);
    }
    const int n = ncols * d.s;
    lev_combine_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, ncols, n_obs);
  }
  if (ev) cudaEventRecord(ev[1], st);
  return 0;
}

}  // namespace rid
