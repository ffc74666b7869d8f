// Batch step of Algorithm 3, run on the device whenever t columns are
// buffered (and once more for the tail): lambda (Eq. 23), sketched ridge
// scores of C and D (Eq. 23), prune/refill of the basis slots, the basis Gram
// G = A_J^T A_J and A_J^T A_Jprev, the coefficient candidates of Algorithms
// 4-7, the NA-Hutch++ estimate of each (Algorithm 8, Eqs. 36-37) and the
// commit of P = P_{q*}.  Every decision stays on the device, so the whole
// ingest loop needs no host round trip.
#include <cuda_runtime.h>
#include <stdint.h>

#include "linalg.cuh"
#include "philox.cuh"
#include "rid.h"
#include "rid_internal.cuh"

namespace rid {

// ---------------------------------------------------------------- work layout
struct WorkLayout {
  int64_t eigA, eigR, eigD, eigE, eigV, eigP;   // tridiagonalization of the sketch Gram
  int64_t beta, vhead, mu, ldld, ldll;    // reflectors, top-k eigenvalues, LDL^T of T + lambda I
  // every array of the lambda part has a second copy: batch b uses copy b % 2, so that the
  // lambda parts of consecutive batches run concurrently (two lambda streams) and the lambda
  // part of batch b+1 may run while the scores of batch b still read theirs
  int64_t eigR2, beta2, vhead2, ldld2, ldll2;
  int64_t eigA2, eigD2, eigE2, eigP2, mu2;
  int64_t svec;                           // per-warp vectors of the scores (their own stream)
  int64_t unif;                           // uniforms of the prune/refill decisions
  int64_t vec;                            // per-warp vectors (scores / applies)
  int64_t SJ, HJ, G, Gq, Gc, T;           // gathered sketch data and Grams
  int64_t QR4, b4, h4, r4, QR6, b6, h6, r6;   // Householder factors (r: diagonal of R)
  int64_t Lcinv, r4inv, r6inv;            // reciprocal diagonals of the triangular factors
  int64_t Q4x, Q6x, M6;                   // explicit thin Q factors (s x t) and Q6^T (Omega A_J) (t x t)
  int64_t Z, trgpp, hut, hut_stride;      // Hutch++
  int64_t total;
};

// Per-warp scratch of the apply / coefficient kernels: an s-vector, or two t-vectors.
__host__ __device__ inline int64_t vec_stride(int64_t s, int64_t t) { return s > 2 * t ? s : 2 * t; }

static constexpr int kApplyBlocks = 2 * 152;
static constexpr int kApplyThreads = 256;
static constexpr int kHutChunk = 32;

// per-candidate scratch of hutch_finish_kernel: X, W (h1 x h2), ZG (h1 x t), J (h1 x h1),
// Xp (h2 x h1), M1 (h1 x h3), F (h3 x h2), E (h2 x h3)
static int64_t hut_stride(const Dev& d) {
  const int64_t h1 = d.h1, h2 = d.h2, h3 = d.h3, t = d.t;
  return 3 * h1 * h2 + h1 * t + h1 * h1 + 2 * h1 * h3 + 2 * h2 * h3 + 64;
}

static WorkLayout layout(const Dev& d) {
  WorkLayout w{};
  const int64_t s = d.s, t = d.t, hh = d.h1 + d.h2 + d.h3;
  const int64_t nw = (int64_t)kApplyBlocks * (kApplyThreads / 32);
  int64_t o = 0;
  auto take = [&](int64_t n) { int64_t r = o; o += (n + 31) / 32 * 32; return r; };
  w.eigA = take(s * s); w.eigR = take(s * s); w.eigD = take(s); w.eigE = take(s); w.eigV = take(s);
  w.eigP = take(2 * s);
  w.beta = take(s); w.vhead = take(s); w.mu = take(t); w.ldld = take(s); w.ldll = take(s);
  w.eigR2 = take(s * s); w.beta2 = take(s); w.vhead2 = take(s); w.ldld2 = take(s); w.ldll2 = take(s);
  w.eigA2 = take(s * s); w.eigD2 = take(s); w.eigE2 = take(s); w.eigP2 = take(2 * s); w.mu2 = take(t);
  w.svec = take(2 * t * vec_stride(s, t));
  w.unif = take(t * (t + 2));
  w.vec = take(nw * vec_stride(s, t));
  w.SJ = take(s * t); w.HJ = take(hh * t); w.G = take(t * t); w.Gq = take(t * t);
  w.Gc = take(t * t); w.T = take(t * t);
  w.QR4 = take(s * t); w.b4 = take(t); w.h4 = take(t); w.r4 = take(t);
  w.QR6 = take(s * t); w.b6 = take(t); w.h6 = take(t); w.r6 = take(t);
  w.Lcinv = take(t); w.r4inv = take(t); w.r6inv = take(t);
  w.Q4x = take(s * t); w.Q6x = take(s * t); w.M6 = take(t * t);
  w.Z = take(4 * hh * t); w.trgpp = take(4);
  w.hut_stride = hut_stride(d);
  w.hut = take(4 * w.hut_stride);
  w.total = o;
  return w;
}

int64_t work_doubles(const Dev& d) { return layout(d).total; }

// ---------------------------------------------------------------- prune / refill
// The uniforms of every possible decision, u(batch, i, r), drawn in parallel: r = 0 the drop of
// slot i, r = 1..count the refill scan, r = count + 1 the proportional draw (R7p).
__global__ void uniforms_kernel(Dev d, double* unif, int count, int batch) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = count + 2;
  if (idx >= d.t * per) return;
  const int i = idx / per, r = idx % per;
  unif[idx] = sample_uniform(d.seed, (uint32_t)batch, (uint32_t)i, (uint32_t)r);
}

// Prune / refill of the basis slots (Algorithm 3) and the bookkeeping of the later kernels.
// One CTA: the slot state, the refill probabilities and (when they fit) the uniforms are
// staged in shared memory by all threads; warp 0 then takes the decisions slot by slot in
// slot order (a refill tests 32 buffered columns at a time and takes the first success in
// column order), and thread 0 writes the index lists.  A buffered column has a larger index
// than every column of the previous basis, so it can only be in C already if an earlier slot
// of this scan took it (the taken[] flags).  Buffered column q has global index jd0 + q.
// d holds the live selection state (JC, slotC, tau_old: read, then updated to the new basis);
// the step's record r receives the previous and the new basis (r.JC_prev / r.slotC_prev and
// r.JC / r.slotC) and the index lists its tail reads, so that the next step's scores and select
// may run while this step's tail still reads its record.
// Pool slots: the columns of batch + la go to the first t of the (la + 2) t slots that hold
// neither the previous nor the new basis nor the batches batch + 1 .. batch + la - 1 (their
// lists in d.dslot_all), written over this batch's list; so that batch's ingest may run while
// this step and the next la - 1 steps are in flight.
__global__ void __launch_bounds__(256) select_kernel(Dev d, Dev r, const double* unif, int count, int stage_u,
                                                     int64_t jd0, int batch) {
  extern __shared__ double ssm[];
  const int t = d.t, np = d.npool, per = count + 2;
  const int tid = threadIdx.x, lane = tid & 31;
  double* s_told = ssm;                                  // t
  double* s_tauC = s_told + t;                           // t
  double* s_p = s_tauC + t;                              // count: refill probabilities
  double* s_tauD = s_p + count;                          // count
  double* s_u = s_tauD + count;                          // t x per when staged
  int64_t* s_JC = reinterpret_cast<int64_t*>(s_u + (stage_u ? (size_t)t * per : 0));
  int64_t* s_JCp = s_JC + t;
  int64_t* s_JD = s_JCp + t;                             // count
  int* s_slot = reinterpret_cast<int*>(s_JD + count);    // t
  int* s_slotp = s_slot + t;                             // t
  int* s_dslot = s_slotp + t;                            // count
  int* s_taken = s_dslot + count;                        // count
  int* s_used = s_taken + count;                         // npool
  for (int i = tid; i < t; i += blockDim.x) {
    s_told[i] = d.tau_old[i]; s_tauC[i] = d.tauC[i];
    s_JC[i] = d.JC[i]; s_JCp[i] = d.JC[i];              // the previous basis is the live one
    s_slot[i] = d.slotC[i]; s_slotp[i] = d.slotC[i];
  }
  for (int q = tid; q < count; q += blockDim.x) {
    const double td = d.tauD[q];
    s_tauD[q] = td;
    s_p[q] = fmin(fmax(td * d.refill_scale, 0.0), 1.0);
    s_JD[q] = jd0 + q; s_dslot[q] = d.dslot[q]; s_taken[q] = 0;
  }
  for (int i = tid; i < np; i += blockDim.x) s_used[i] = 0;
  if (stage_u)
    for (int i = tid; i < t * per; i += blockDim.x) s_u[i] = unif[i];
  __syncthreads();
  if (d.ext_sel) {
    // Algorithm 1 as the selector: the columns it kept from this batch fill the empty slots in
    // order (it never drops a column, and its subset is capped at t).  Entries for later columns
    // (being appended concurrently) lie past jd0 + count or still read -1: both are skipped.
    if (tid == 0) {
      const int ns = *(volatile const int*)d.ext_nsel;
      int cur = 0;
      for (int i = 0; i < t; ++i) {
        if (s_JC[i] >= 0) continue;
        int rr = -1;
        while (cur < ns && rr < 0) {
          const int64_t j = ((volatile const int64_t*)d.ext_sel)[cur++];
          if (j >= jd0 && j < jd0 + count) rr = (int)(j - jd0);
        }
        if (rr < 0) break;
        s_taken[rr] = 1; s_JC[i] = s_JD[rr]; s_slot[i] = s_dslot[rr]; s_told[i] = 1.0;
      }
    }
  } else if (tid < 32) {
    for (int i = 0; i < t; ++i) {
      const double* u = stage_u ? s_u + (size_t)i * per : unif + (size_t)i * per;
      if (lane == 0 && s_JC[i] >= 0) {
        const double tc = fmin(s_told[i], s_tauC[i]);
        if (u[0] < 1.0 - tc / s_told[i]) { s_JC[i] = -1; s_slot[i] = -1; s_told[i] = 1.0; }
        else s_told[i] = tc;
      }
      __syncwarp();
      if (s_JC[i] < 0) {
        for (int r0 = 0; r0 < count; r0 += 32) {
          const int rr0 = r0 + lane;
          const bool ok = rr0 < count && u[1 + rr0] < s_p[rr0] && !s_taken[rr0];
          const unsigned msk = __ballot_sync(0xffffffffu, ok);
          if (msk) {
            int rr = r0 + __ffs(msk) - 1;
            if (lane == 0) {
              if (d.refill_mode == 1) {
                // R7p: the column is drawn among those not yet taken with probability proportional
                // to its score, by inverse CDF over the scores summed in column order (one lane, a
                // fixed order of the additions)
                double tot = 0.0;
                for (int q = 0; q < count; ++q) if (!s_taken[q]) tot += fmax(s_tauD[q], 0.0);
                if (tot > 0.0) {
                  const double x = u[1 + count] * tot;
                  double run = 0.0;
                  int pick = -1, last = -1;
                  for (int q = 0; q < count; ++q) {
                    if (s_taken[q]) continue;
                    run += fmax(s_tauD[q], 0.0);
                    last = q;
                    if (x < run) { pick = q; break; }
                  }
                  rr = pick >= 0 ? pick : last;
                }
              }
              s_taken[rr] = 1; s_JC[i] = s_JD[rr]; s_slot[i] = s_dslot[rr]; s_told[i] = s_tauD[rr];
            }
            break;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (tid == 0) {
    int na = 0, nn = 0, nk = 0;
    for (int i = 0; i < t; ++i) {
      r.posof[i] = -1;
      if (s_JC[i] >= 0) {
        const int is_new = !(s_JC[i] == s_JCp[i]);
        r.act[na] = i;
        r.posof[i] = na;
        r.isnew[na] = is_new;
        if (is_new) { r.newpos[nn] = na; r.gnew[nn++] = s_slot[i]; } else ++nk;
        ++na;
      }
    }
    int npa = 0;
    for (int i = 0; i < t; ++i) if (s_JCp[i] >= 0) r.pact[npa++] = i;
    // Gram targets: pool slots of the current and the previous basis (distinct); the new
    // elements first, in the order of gnew, so that target x < nnew is new element x
    int nt = 0;
    for (int i = 0; i < t; ++i)
      if (s_JC[i] >= 0 && s_JC[i] != s_JCp[i]) { const int ps = s_slot[i]; r.gtgt[nt++] = ps; s_used[ps] = 1; }
    for (int i = 0; i < t; ++i)
      if (s_JC[i] >= 0 && s_JC[i] == s_JCp[i]) { const int ps = s_slot[i]; r.gtgt[nt++] = ps; s_used[ps] = 1; }
    for (int i = 0; i < t; ++i) {
      if (s_JCp[i] < 0) continue;
      const int ps = s_slotp[i];
      if (!s_used[ps]) { r.gtgt[nt++] = ps; s_used[ps] = 2; }
    }
    for (int i = 0; i < META_LEN; ++i) r.meta[i] = 0;
    r.meta[META_NACT] = na; r.meta[META_NPACT] = npa; r.meta[META_NNEW] = nn;
    r.meta[META_NTGT] = nt; r.meta[META_NKEPT] = nk;
    // buffer slots of batch + la: the first t pool slots holding none of the new basis (flag 1),
    // the previous basis (flag 2) and the columns of the batches in between (flag 3)
    for (int k = 1; k < d.la; ++k) {
      const int* lst = d.dslot_all + (size_t)((batch + k) % d.la) * t;
      for (int q = 0; q < t; ++q) s_used[lst[q]] = 3;
    }
    int q = 0;
    for (int ps = 0; ps < np && q < t; ++ps)
      if (s_used[ps] == 0) d.dslot[q++] = ps;
  }
  for (int i = tid; i < t; i += blockDim.x) {
    d.JC[i] = s_JC[i]; d.slotC[i] = s_slot[i]; d.tau_old[i] = s_told[i];
    r.JC[i] = s_JC[i]; r.slotC[i] = s_slot[i];
    r.JC_prev[i] = s_JCp[i]; r.slotC_prev[i] = s_slotp[i];
  }
}

// Dynamic shared memory of select_kernel: doubles s_told, s_tauC (t), s_p, s_tauD (count) and the
// staged uniforms (t x (count + 2)); int64 s_JC, s_JCp (t), s_JD (count); ints s_slot, s_slotp
// (t), s_dslot, s_taken (count) and s_used (npool).
size_t select_smem_bytes(int t, int count, bool stage_u, int npool) {
  return (size_t)8 * (2 * t + 2 * count + (stage_u ? (size_t)t * (count + 2) : 0)) + (size_t)8 * (2 * t + count) +
         (size_t)4 * (2 * t + 2 * count + npool);
}

// ---------------------------------------------------------------- basis Gram
// C[x][y] = <pool[gnew[x]], pool[gtgt[y]]> over one K-range, 64x64 tile per CTA, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) basis_gram_kernel(Dev d) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const int nnew = d.meta[META_NNEW], ntgt = d.meta[META_NTGT];
  const int x0 = blockIdx.x * 64, y0 = blockIdx.y * 64;
  if (x0 >= nnew || y0 >= ntgt) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t per = (d.m + gridDim.z - 1) / gridDim.z;
  const int64_t k0 = (int64_t)blockIdx.z * per;
  const int64_t k1 = (k0 + per < d.m) ? k0 + per : d.m;
  const T* pool = (const T*)d.pool;
  double acc64[4][4];
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc64[a][b] = 0.0; acc[a][b] = T(0); }
  int since = 0;
  for (int64_t kk = k0; kk < k1; kk += 16) {
    // load 16 coordinates of 64 columns each: thread -> (coord = tid % 16, col = tid / 16 + 16 c)
    const int kc = threadIdx.x & 15, cc = threadIdx.x >> 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = cc + 16 * c;
      const int64_t i = kk + kc;
      T va = T(0), vb = T(0);
      if (i < k1) {
        if (x0 + col < nnew) va = pool[(int64_t)d.gnew[x0 + col] * d.m_pad + i];
        if (y0 + col < ntgt) vb = pool[(int64_t)d.gtgt[y0 + col] * d.m_pad + i];
      }
      As[kc][col] = va;
      Bs[kc][col] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T ra[4], rb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { ra[a] = As[k][tx + 16 * a]; rb[a] = Bs[k][ty + 16 * a]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += ra[a] * rb[b];
    }
    __syncthreads();
    if (++since == 4) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { acc64[a][b] += (double)acc[a][b]; acc[a][b] = T(0); }
      since = 0;
    }
  }
  const int two_t = 2 * d.t;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int x = x0 + tx + 16 * a, y = y0 + ty + 16 * b;
      if (x < nnew && y < ntgt)
        d.gpart[((size_t)blockIdx.z * d.t + x) * two_t + y] = acc64[a][b] + (double)acc[a][b];
    }
}

__global__ void gram_reduce_kernel(Dev d, int nsplit) {
  const int nnew = d.meta[META_NNEW], ntgt = d.meta[META_NTGT];
  const int two_t = 2 * d.t;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= d.t * two_t) return;
  const int x = idx / two_t, y = idx % two_t;
  if (x >= nnew || y >= ntgt) return;
  double v = 0.0;
  for (int z = 0; z < nsplit; ++z) v += d.gpart[((size_t)z * d.t + x) * two_t + y];
  const int a = d.gnew[x], b = d.gtgt[y];
  const int np = d.npool;
  // a pair of two new columns is computed twice; only the one with a <= b writes it, so
  // that the stored Gram is symmetric and independent of the order of the writes
  bool b_new = false;
  for (int z = 0; z < nnew; ++z) b_new |= d.gnew[z] == b;
  if (b_new && a > b) return;
  d.Gp[a + (size_t)b * np] = v;
  d.Gp[b + (size_t)a * np] = v;
}

// ---------------------------------------------------------------- gather + factorizations
// Gather Omega A_J (scaled), the probe rows of the basis and the new-element columns for
// Algorithm 6 (sketch side), or G = A_J^T A_J and A_J^T A_Jprev from the pool Gram (Gram side);
// grid-stride, many blocks.
template <bool kSketch>
__global__ void gather_kernel(Dev d, WorkLayout w) {
  const int s = d.s, np = d.npool, hh = d.h1 + d.h2 + d.h3;
  const int na = d.meta[META_NACT], npa = d.meta[META_NPACT], nn = d.meta[META_NNEW];
  const double rs = 1.0 / sqrt((double)s);
  double* SJ = d.work + w.SJ;
  double* HJ = d.work + w.HJ;
  double* G = d.work + w.G;
  double* Gq = d.work + w.Gq;
  double* Gc = d.work + w.Gc;
  double* QR4 = d.work + w.QR4;
  double* QR6 = d.work + w.QR6;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  if (!kSketch) {
    for (int64_t idx = g0; idx < (int64_t)na * na; idx += gs) {
      const int a = (int)(idx % na), b = (int)(idx / na);
      const double g = d.Gp[d.slotC[d.act[a]] + (size_t)d.slotC[d.act[b]] * np];
      G[a + (size_t)b * na] = g;
      Gc[a + (size_t)b * na] = g;
    }
    for (int64_t idx = g0; idx < (int64_t)na * npa; idx += gs) {
      const int a = (int)(idx % na), b = (int)(idx / na);
      Gq[a + (size_t)b * na] = d.Gp[d.slotC[d.act[a]] + (size_t)d.slotC_prev[d.pact[b]] * np];
    }
    return;
  }
  for (int64_t idx = g0; idx < (int64_t)s * na; idx += gs) {
    const int i = (int)(idx % s), a = (int)(idx / s);
    const double v = d.S[(size_t)d.JC[d.act[a]] * d.rows + i] * rs;
    SJ[i + (size_t)a * s] = v;
    QR4[i + (size_t)a * s] = v;
  }
  for (int64_t idx = g0; idx < (int64_t)s * nn; idx += gs) {
    const int i = (int)(idx % s), c = (int)(idx / s);
    QR6[i + (size_t)c * s] = d.S[(size_t)d.JC[d.act[d.newpos[c]]] * d.rows + i] * rs;
  }
  for (int64_t idx = g0; idx < (int64_t)hh * na; idx += gs) {
    const int r = (int)(idx % hh), a = (int)(idx / hh);
    HJ[r + (size_t)a * hh] = d.S[(size_t)d.JC[d.act[a]] * d.rows + d.hbase + r];
  }
}

// Row sharding: the step's new-element x target block of the pool Gram, packed t x 2t (zeros past
// the counts) for the exchange, and the summed block written back to both triangles.
__global__ void gram_pack_kernel(Dev d) {
  const int t = d.t, nn = d.meta[META_NNEW], nt = d.meta[META_NTGT], np = d.npool;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < t * 2 * t; idx += gridDim.x * blockDim.x) {
    const int x = idx % t, y = idx / t;
    d.xbuf[idx] = (x < nn && y < nt) ? d.Gp[d.gnew[x] + (size_t)d.gtgt[y] * np] : 0.0;
  }
}
__global__ void gram_unpack_kernel(Dev d) {
  const int t = d.t, nn = d.meta[META_NNEW], nt = d.meta[META_NTGT], np = d.npool;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < t * 2 * t; idx += gridDim.x * blockDim.x) {
    const int x = idx % t, y = idx / t;
    if (x >= nn || y >= nt) continue;
    const double v = d.xbuf[idx];
    d.Gp[d.gnew[x] + (size_t)d.gtgt[y] * np] = v;     // a pair of two new elements: equal values
    d.Gp[d.gtgt[y] + (size_t)d.gnew[x] * np] = v;
  }
}

// Cholesky of G (t x t at most; FP64, one CTA).
constexpr size_t kCholSmemBytes = 160 * 1024;
constexpr size_t kHutchSmemBytes = 160 * 1024;

// Cholesky factor of the basis Gram (in place in Gc); staged in shared memory when it fits.
//
// Algorithms 5 and 7 go through G = A_J^T A_J, whose condition number is kappa(A_J)^2.  When
// the smallest pivot falls below rho0 x the largest diagonal entry -- the basis is so nearly
// dependent that the Gram's own rounding (rho0 is ten times its relative accuracy: FP64 sums,
// or the BF16x2 split on tensor cores) would dominate the solve -- G is factored again with the
// Tikhonov shift rho0 max_a G_aa on its diagonal: directions of A_J below the shift are damped
// instead of amplified, so the coefficients stay bounded and the residual near its minimum.
__global__ void __launch_bounds__(1024) gram_chol_kernel(Dev d, WorkLayout w, int staged, double rho0) {
  extern __shared__ double gsm[];
  __shared__ int fail;
  __shared__ double gm, pmin;
  const int na = d.meta[META_NACT];
  double* Gc = d.work + w.Gc;
  const double* G = d.work + w.G;
  const bool use_smem = staged && (size_t)na * na * sizeof(double) <= kCholSmemBytes;
  double* A = use_smem ? gsm : Gc;
  if (use_smem)
    for (int i = threadIdx.x; i < na * na; i += blockDim.x) gsm[i] = Gc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    fail = 0;
    pmin = 0.0;
    double m = 0.0;
    for (int a = 0; a < na; ++a) m = fmax(m, A[a + (size_t)a * na]);
    gm = m;
  }
  __syncthreads();
  cta_cholesky(A, na, na, 1e-13 * gm, &fail, &pmin);
  __syncthreads();
  const bool shift = na > 0 && pmin < rho0 * gm;
  if (shift) {
    for (int i = threadIdx.x; i < na * na; i += blockDim.x) {
      const int a = i % na, b = i / na;
      A[i] = G[i] + (a == b ? rho0 * gm : 0.0);
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    cta_cholesky(A, na, na, 1e-13 * gm, &fail);
  }
  if (threadIdx.x == 0) d.scal[SCAL_GSHIFT] = shift ? rho0 : 0.0;
  double* linv = d.work + w.Lcinv;
  for (int a = threadIdx.x; a < na; a += blockDim.x) {
    const double ljj = A[a + (size_t)a * na];
    linv[a] = (ljj != 0.0) ? 1.0 / ljj : 0.0;
  }
  if (use_smem)
    for (int i = threadIdx.x; i < na * na; i += blockDim.x) Gc[i] = gsm[i];
}

// Reciprocal diagonals of the two QR factors, with the rank tolerance of each:
// |R_jj| <= max(max(s, n) eps, sk_rel) max|R_ii| gives 0 (the component is dropped; sk_rel is
// the relative accuracy of a reduced-precision sketch, 0 for FP64).
__global__ void __launch_bounds__(256) qr_prep_kernel(Dev d, WorkLayout w) {
  __shared__ double sm[2][8];
  const int na = d.meta[META_NACT], nn = d.meta[META_NNEW], s = d.s;
  const double* r4 = d.work + w.r4;
  const double* r6 = d.work + w.r6;
  double m4 = 0.0, m6 = 0.0;
  for (int a = threadIdx.x; a < na; a += blockDim.x) m4 = fmax(m4, fabs(r4[a]));
  for (int c = threadIdx.x; c < nn; c += blockDim.x) m6 = fmax(m6, fabs(r6[c]));
  for (int o = 16; o > 0; o >>= 1) {
    m4 = fmax(m4, __shfl_xor_sync(0xffffffffu, m4, o));
    m6 = fmax(m6, __shfl_xor_sync(0xffffffffu, m6, o));
  }
  if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = m4; sm[1][threadIdx.x >> 5] = m6; }
  __syncthreads();
  m4 = 0.0; m6 = 0.0;
  for (int i = 0; i < 8; ++i) { m4 = fmax(m4, sm[0][i]); m6 = fmax(m6, sm[1][i]); }
  const double tol4 = fmax((double)(s > na ? s : na) * 2.220446049250313e-16, d.sk_rel) * m4;
  const double tol6 = fmax((double)(s > nn ? s : nn) * 2.220446049250313e-16, d.sk_rel) * m6;
  for (int a = threadIdx.x; a < na; a += blockDim.x)
    d.work[w.r4inv + a] = (fabs(r4[a]) > tol4) ? 1.0 / r4[a] : 0.0;
  for (int c = threadIdx.x; c < nn; c += blockDim.x)
    d.work[w.r6inv + c] = (fabs(r6[c]) > tol6) ? 1.0 / r6[c] : 0.0;
}

// T = G^{-1} Gq, one warp per column (Algorithm 7 through the Gram:
// R^+ Q^T A_Jprev = (A_J^T A_J)^{-1} A_J^T A_Jprev).
__global__ void tsolve_kernel(Dev d, WorkLayout w) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int na = d.meta[META_NACT], npa = d.meta[META_NPACT];
  const double* Gc = d.work + w.Gc;
  const double* Gq = d.work + w.Gq;
  double* T = d.work + w.T;
  for (int b = gw; b < npa; b += nwarps) {
    double* x = T + (size_t)b * na;
    for (int a = lane; a < na; a += 32) x[a] = Gq[a + (size_t)b * na];
    __syncwarp();
    warp_trsv_lower_r(Gc, d.work + w.Lcinv, na, na, x);
    warp_trsv_lower_t_r(Gc, d.work + w.Lcinv, na, na, x);
  }
}

// ---------------------------------------------------------------- Algorithms 4-7
// The Householder QR factors of Omega A_J (QR4) and of its new columns (QR6) are turned into
// explicit thin Q factors once per batch step, so that the per-column work is two small GEMMs
// over all observed columns plus triangular arithmetic:
//   Z4 = Q4^T S~, Z6 = Q6^T S~ (S~ = Omega A_obs / sqrt(s)), M6 = Q6^T (Omega A_J) / sqrt(s);
//   Algorithm 4: P4(:, j) = R4^{-1} Z4(:, j);
//   Algorithm 5: (Omega A_J)^T s~_j = R4^T Q4^T s~_j = R4^T Z4(:, j), then G^{-1} (Cholesky);
//   Algorithm 6: Q6^T (s~_j - (Omega A_J)_kept p_j) = Z6(:, j) - M6_kept p_j, then R6^{-1}.
// Equal in exact arithmetic to applying the reflectors to every column (the products carry the
// same rounding order of magnitude), with about half of the FP64 operations.

// Explicit thin Q (s x n) of a Householder factorization: column c = H_0 ... H_c e_c (the
// reflectors after c leave e_c unchanged), one warp per column; Q4 columns first, then Q6.
__global__ void __launch_bounds__(256) qform_kernel(Dev d, WorkLayout w) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int s = d.s, t = d.t;
  const int na = d.meta[META_NACT], nn = d.meta[META_NNEW];
  if (gw >= na + nn) return;
  const bool six = gw >= na;
  const int c = six ? gw - na : gw;
  const double* QR = d.work + (six ? w.QR6 : w.QR4);
  const double* beta = d.work + (six ? w.b6 : w.b4);
  const double* vhead = d.work + (six ? w.h6 : w.h4);
  double* x = d.work + w.vec + (size_t)gw * vec_stride(s, t);
  for (int i = lane; i < s; i += 32) x[i] = (i == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int j = c; j >= 0; --j) {
    const double bj = beta[j];
    if (bj == 0.0) continue;
    const double* v = QR + (size_t)j * s;
    const double vh = vhead[j];
    double dot = (lane == 0) ? vh * x[j] : 0.0;
    for (int i = j + 1 + lane; i < s; i += 32) dot += v[i] * x[i];
    dot = warp_sum(dot);
    const double f = bj * dot;
    __syncwarp();
    if (lane == 0) x[j] -= f * vh;
    for (int i = j + 1 + lane; i < s; i += 32) x[i] -= f * v[i];
    __syncwarp();
  }
  double* Q = d.work + (six ? w.Q6x : w.Q4x) + (size_t)c * s;
  for (int i = lane; i < s; i += 32) Q[i] = x[i];
}

// C(0:M, 0:N) = Q^T B over K = s rows, in 32 x 32 output tiles (256 threads, 4 outputs each):
//   mode 0: Q = Q4 (M = n_act), B = S~ (N = n_obs), C = Z4;  mode 1: Q = Q6 (M = n_new),
//   B = S~, C = Z6;  mode 2: Q = Q6, B = Omega A_J / sqrt(s) (N = n_act), C = M6.
// Each output is one dot product in row order, i = 0 .. s-1.
__global__ void __launch_bounds__(256) proj_gemm_kernel(Dev d, WorkLayout w, int mode, int64_t n_obs) {
  __shared__ double Qs[32][33];
  __shared__ double Bs[32][33];
  const int s = d.s, t = d.t;
  const int na = d.meta[META_NACT], nn = d.meta[META_NNEW];
  const int M = mode == 0 ? na : nn;
  const int64_t N = mode == 2 ? (int64_t)na : n_obs;
  const int m0 = blockIdx.x * 32;
  const int64_t n0 = (int64_t)blockIdx.y * 32;
  if (m0 >= M || n0 >= N) return;
  const double* Q = d.work + (mode == 0 ? w.Q4x : w.Q6x);
  const double rs = 1.0 / sqrt((double)s);
  double* C = mode == 0 ? d.zq : mode == 1 ? d.zq + (size_t)t * d.n_cap : d.work + w.M6;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;         // output column n0 + tx, rows m0 + ty + 8 u
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < s; k0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
      const int kk = idx & 31, cc = idx >> 5;
      const int k = k0 + kk;
      const int mq = m0 + cc;
      const int64_t nb = n0 + cc;
      Qs[cc][kk] = (k < s && mq < M) ? Q[k + (size_t)mq * s] : 0.0;
      double bv = 0.0;
      if (k < s && nb < N)
        bv = mode == 2 ? d.work[w.SJ + k + (size_t)nb * s] : d.S[(size_t)nb * d.rows + k] * rs;
      Bs[cc][kk] = bv;
    }
    __syncthreads();
    const int kmax = (s - k0) < 32 ? (s - k0) : 32;
    for (int kk = 0; kk < kmax; ++kk) {
      const double bv = Bs[tx][kk];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(Qs[ty + 8 * u][kk], bv, acc[u]);
    }
    __syncthreads();
  }
  const int64_t nb = n0 + tx;
  if (nb < N)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int mq = m0 + ty + 8 * u;
      if (mq < M) C[mq + (size_t)nb * t] = acc[u];
    }
}

__global__ void __launch_bounds__(kApplyThreads) coeff_kernel(Dev d, WorkLayout w, int64_t n_obs,
                                                              int64_t n_prev) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int s = d.s, t = d.t;
  const int na = d.meta[META_NACT], npa = d.meta[META_NPACT];
  const double* QR4 = d.work + w.QR4;
  const double* QR6 = d.work + w.QR6;
  const double* r4 = d.work + w.r4;
  const double* M6 = d.work + w.M6;
  const double* Gc = d.work + w.Gc;
  const double* T = d.work + w.T;
  double* b = d.work + w.vec + (size_t)gw * vec_stride(s, t);
  double* y = b + t;                                   // a second t-vector
  double* P4 = d.cand;
  double* P5 = d.cand + (size_t)t * d.n_cap;
  double* P6 = d.cand + 2 * (size_t)t * d.n_cap;
  double* P7 = d.cand + 3 * (size_t)t * d.n_cap;
  // reciprocal diagonals (0 below the rank tolerance) from qr_prep_kernel and gram_chol_kernel
  const double* r4inv = d.work + w.r4inv;
  const double* r6inv = d.work + w.r6inv;
  const double* lcinv = d.work + w.Lcinv;
  const int nn = d.meta[META_NNEW];
  for (int64_t j = gw; j < n_obs; j += nwarps) {
    const double* z4 = d.zq + (size_t)j * t;
    const double* z6 = d.zq + (size_t)t * d.n_cap + (size_t)j * t;
    // Algorithm 5's right-hand side (Omega A_J)^T s~_j = R4^T z4 (lane per row, four partial sums)
    for (int a = lane; a < na; a += 32) {
      double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
      int c = 0;
      for (; c + 4 <= a; c += 4) {
        p0 += QR4[c + (size_t)a * s] * z4[c];
        p1 += QR4[c + 1 + (size_t)a * s] * z4[c + 1];
        p2 += QR4[c + 2 + (size_t)a * s] * z4[c + 2];
        p3 += QR4[c + 3 + (size_t)a * s] * z4[c + 3];
      }
      for (; c < a; ++c) p0 += QR4[c + (size_t)a * s] * z4[c];
      y[a] = ((p0 + p1) + (p2 + p3)) + r4[a] * z4[a];
      b[a] = z4[a];
    }
    __syncwarp();
    // Algorithm 4 (Eq. 24): P4(:, j) = R4^{-1} Q4^T s~_j
    warp_trsv_upper_r(QR4, r4inv, na, s, b);
    for (int a = lane; a < na; a += 32) P4[a + (size_t)j * t] = b[a];
    __syncwarp();
    // Algorithm 5: P5(:, j) = G^{-1} (Omega A_J)^T s~_j
    warp_trsv_lower_r(Gc, lcinv, na, na, y);
    warp_trsv_lower_t_r(Gc, lcinv, na, na, y);
    for (int a = lane; a < na; a += 32) P5[a + (size_t)j * t] = y[a];
    __syncwarp();
    // Algorithm 6 (Eqs. 27-30): keep the rows of unchanged basis elements, refit the new
    // ones on the sketched residual, Q6^T r = z6 - M6_kept p.  Previous coefficients of
    // columns observed since the last batch step are the preliminary estimate P4.
    for (int c = lane; c < nn; c += 32) {
      double p0 = 0.0, p1 = 0.0;
      int a = 0;
      for (; a + 2 <= na; a += 2) {
        if (!d.isnew[a]) {
          const double pp = (j < n_prev) ? d.P[d.act[a] + (size_t)j * t] : P4[a + (size_t)j * t];
          p0 += M6[c + (size_t)a * t] * pp;
        }
        if (!d.isnew[a + 1]) {
          const double pp = (j < n_prev) ? d.P[d.act[a + 1] + (size_t)j * t] : P4[a + 1 + (size_t)j * t];
          p1 += M6[c + (size_t)(a + 1) * t] * pp;
        }
      }
      if (a < na && !d.isnew[a]) {
        const double pp = (j < n_prev) ? d.P[d.act[a] + (size_t)j * t] : P4[a + (size_t)j * t];
        p0 += M6[c + (size_t)a * t] * pp;
      }
      b[c] = z6[c] - (p0 + p1);
    }
    __syncwarp();
    warp_trsv_upper_r(QR6, r6inv, nn, s, b);
    if (lane == 0) {
      int c = 0;
      for (int a = 0; a < na; ++a) {
        double v;
        if (d.isnew[a]) v = b[c++];
        else v = (j < n_prev) ? d.P[d.act[a] + (size_t)j * t] : P4[a + (size_t)j * t];
        P6[a + (size_t)j * t] = v;
      }
    }
    __syncwarp();
    // Algorithm 7 (Eqs. 31-32): P7 = T P_prev on the previous columns, P4 on the new ones
    for (int a = lane; a < na; a += 32) {
      double v;
      if (j < n_prev) {
        v = 0.0;
        for (int c = 0; c < npa; ++c) v += T[a + (size_t)c * na] * d.P[d.pact[c] + (size_t)j * t];
      } else {
        v = P4[a + (size_t)j * t];
      }
      P7[a + (size_t)j * t] = v;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- NA-Hutch++ (Algorithm 8)
// grid (ceil(n_obs / kHutChunk), 4): partial Z_q = H P_q^T over a column chunk, and tr(G P P^T).
__global__ void __launch_bounds__(256) hutch_partial_kernel(Dev d, WorkLayout w, int64_t n_obs) {
  __shared__ double sh[33];
  const int q = blockIdx.y;
  const int na = d.meta[META_NACT];
  const int hh = d.h1 + d.h2 + d.h3;
  const int t = d.t;
  const double* Pq = d.cand + (size_t)q * t * d.n_cap;
  const int64_t j0 = (int64_t)blockIdx.x * kHutChunk;
  const int64_t j1 = (j0 + kHutChunk < n_obs) ? j0 + kHutChunk : n_obs;
  double* out = d.hpart + ((size_t)q * gridDim.x + blockIdx.x) * hpart_stride(hh, t);
  for (int idx = threadIdx.x; idx < hh * na; idx += blockDim.x) {
    const int r = idx % hh, a = idx / hh;
    double acc = 0.0;
    for (int64_t j = j0; j < j1; ++j) acc += d.S[(size_t)j * d.rows + d.hbase + r] * Pq[a + (size_t)j * t];
    out[idx] = acc;
  }
  const double* G = d.work + w.G;
  double part = 0.0, part_e = 0.0;
  for (int idx = threadIdx.x; idx < na * (int)(j1 - j0); idx += blockDim.x) {
    const int a = idx % na;
    const int64_t j = j0 + idx / na;
    double gp = 0.0;
    for (int c = 0; c < na; ++c) gp += G[a + (size_t)c * na] * Pq[c + (size_t)j * t];
    const double p = Pq[a + (size_t)j * t];
    part += gp * p;
    part_e += G[a + (size_t)a * na] * p * p;
  }
  const double tot = block_sum(part, sh);
  const double tot_e = block_sum(part_e, sh);
  if (threadIdx.x == 0) {
    out[(size_t)hh * t] = tot;
    out[(size_t)hh * t + 1] = tot_e;
  }
}

// sum_{c < n} a[c sa] b[c sb] with four independent partial sums: a dependent FP64 FMA chain
// costs about 64 cycles per step on this GPU.
__device__ __forceinline__ double dot4(const double* a, int64_t sa, const double* b, int64_t sb, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int c = 0;
  for (; c + 4 <= n; c += 4) {
    s0 += a[c * sa] * b[c * sb];
    s1 += a[(c + 1) * sa] * b[(c + 1) * sb];
    s2 += a[(c + 2) * sa] * b[(c + 2) * sb];
    s3 += a[(c + 3) * sa] * b[(c + 3) * sb];
  }
  for (; c < n; ++c) s0 += a[c * sa] * b[c * sb];
  return (s0 + s1) + (s2 + s3);
}

// Pseudo-inverse of the small p x q matrix X (p <= q, row-major in Y) by one-sided Jacobi on
// its rows, all warps of the CTA: each sweep visits every row pair once in p' - 1 rounds of
// disjoint pairs (round-robin order, p' = p rounded up to even; warp w rotates pair w of the
// round).  Writes Xp (q x p, row-major); J (p x p), nr2 (p) and wred (>= 33 doubles) are scratch.
// Singular values below rcond * sigma_max are dropped, as in an SVD-based pseudo-inverse.
__device__ void cta_pinv_rows(double* Y, double* J, int p, int q, double* Xp, double rcond, double* nr2,
                              double* wred) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int idx = tid; idx < p * p; idx += blockDim.x) J[idx] = (idx % (p + 1) == 0) ? 1.0 : 0.0;
  const int pe = p + (p & 1);
  const int npair = pe / 2;
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int r = 0; r < pe - 1; ++r) {
      for (int pr = wid; pr < npair; pr += nw) {
        // circle method: pair 0 is (r, pe - 1); pair i is ((r + i) mod (pe-1), (r - i) mod (pe-1))
        int a, c;
        if (pr == 0) { a = r; c = pe - 1; }
        else { a = (r + pr) % (pe - 1); c = (r - pr + (pe - 1)) % (pe - 1); }
        if (a > c) { const int tmp = a; a = c; c = tmp; }
        if (c >= p) continue;                     // the dummy row of an odd p
        double al0 = 0.0, be0 = 0.0, ga0 = 0.0, al1 = 0.0, be1 = 0.0, ga1 = 0.0;
        int k = lane;
        for (; k + 32 < q; k += 64) {
          const double ya = Y[a * q + k], yc = Y[c * q + k];
          const double yb = Y[a * q + k + 32], yd = Y[c * q + k + 32];
          al0 += ya * ya; be0 += yc * yc; ga0 += ya * yc;
          al1 += yb * yb; be1 += yd * yd; ga1 += yb * yd;
        }
        if (k < q) { const double ya = Y[a * q + k], yc = Y[c * q + k]; al0 += ya * ya; be0 += yc * yc; ga0 += ya * yc; }
        const double al = warp_sum(al0 + al1), be = warp_sum(be0 + be1), ga = warp_sum(ga0 + ga1);
        if (al == 0.0 || be == 0.0) continue;
        const double rel = fabs(ga) * rsqrt(al * be);
        off = fmax(off, rel);
        if (rel < 1e-15) continue;
        // rotation annihilating ga: t = ga / (d + sign(d) sqrt(d^2 + ga^2)), d = (be - al) / 2
        const double dd = 0.5 * (be - al);
        const double tt = ga / (dd + copysign(sqrt(dd * dd + ga * ga), dd));
        const double cs = rsqrt(1.0 + tt * tt), sn = cs * tt;
        for (int kk = lane; kk < q; kk += 32) {
          const double ya = Y[a * q + kk], yc = Y[c * q + kk];
          Y[a * q + kk] = cs * ya - sn * yc;
          Y[c * q + kk] = sn * ya + cs * yc;
        }
        for (int kk = lane; kk < p; kk += 32) {
          const double ja = J[kk * p + a], jc = J[kk * p + c];
          J[kk * p + a] = cs * ja - sn * jc;
          J[kk * p + c] = sn * ja + cs * jc;
        }
      }
      __syncthreads();
    }
    // largest off-diagonal measure of the sweep over the CTA
    if (lane == 0) wred[wid] = off;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int i = 0; i < nw; ++i) m = fmax(m, wred[i]);
      wred[32] = m;
    }
    __syncthreads();
    const bool done = wred[32] < 1e-15;
    __syncthreads();
    if (done) break;
  }
  // sigma_a^2 = ||Y_a||^2 (one warp per row); X^+ = Y^T diag(1/sigma^2) J^T over sigma > rcond sigma_max
  for (int a = wid; a < p; a += nw) {
    double v = 0.0;
    for (int k = lane; k < q; k += 32) v += Y[a * q + k] * Y[a * q + k];
    v = warp_sum(v);
    if (lane == 0) nr2[a] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int a = 0; a < p; ++a) m = fmax(m, nr2[a]);
    // nr2[a] <- 1 / sigma_a^2 for the kept rows, 0 for the dropped ones (one thread: this
    // GPU's FP64 square root and division are long instruction sequences)
    const double cut = rcond * sqrt(m);
    for (int a = 0; a < p; ++a) {
      const double sg = sqrt(nr2[a]);
      nr2[a] = (sg > cut && sg != 0.0) ? 1.0 / nr2[a] : 0.0;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < q * p; idx += blockDim.x) {
    const int k = idx / p, c = idx % p;          // Xp[k][c] = sum_a Y[a][k] / sigma_a^2 * J[c][a]
    double acc = 0.0;
    for (int a = 0; a < p; ++a) acc += Y[a * q + k] * nr2[a] * J[c * p + a];
    Xp[idx] = acc;
  }
  __syncthreads();
}


// One CTA per candidate: reduce the partials and evaluate Eqs. 36-37.
__global__ void __launch_bounds__(512) hutch_finish_kernel(Dev d, WorkLayout w, int nchunk, int staged,
                                                           int fro_slot) {
  extern __shared__ double hsm[];
  __shared__ double sh[33];
  const int q = blockIdx.x;
  const int na = d.meta[META_NACT];
  const int h1 = d.h1, h2 = d.h2, h3 = d.h3, hh = h1 + h2 + h3;
  const int t = d.t;
  double* Z = d.work + w.Z + (size_t)q * hh * t;
  const double* HJ = d.work + w.HJ;
  const double* G = d.work + w.G;
  double* hut = d.work + w.hut + (size_t)q * w.hut_stride;
  // Z and HJ are read many times below: staged in shared memory when they fit
  const bool use_smem = staged && (size_t)2 * hh * na * sizeof(double) <= kHutchSmemBytes;
  double* Zs = use_smem ? hsm : Z;
  const double* HJs = use_smem ? hsm + (size_t)hh * na : HJ;
  for (int idx = threadIdx.x; idx < hh * na; idx += blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += d.hpart[((size_t)q * nchunk + c) * hpart_stride(hh, t) + idx];
    Z[idx] = v;                                   // Z[r + a*hh] = (Omega A_obs P^T)[r][a]
    if (use_smem) Zs[idx] = v;
  }
  if (use_smem)
    for (int idx = threadIdx.x; idx < hh * na; idx += blockDim.x) hsm[(size_t)hh * na + idx] = HJ[idx];
  double trg = 0.0, ener = 0.0;
  if (threadIdx.x == 0)
    for (int c = 0; c < nchunk; ++c) {
      const double* pc = d.hpart + ((size_t)q * nchunk + c) * hpart_stride(hh, t) + (size_t)hh * t;
      trg += pc[0];
      ener += pc[1];
    }
  __syncthreads();
  // views: Zi rows [o_i, o_i + h_i) of Z and HJ
  const int o1 = 0, o2 = h1, o3 = h1 + h2;
  double* X = hut;                    // h1 x h2 row-major
  double* W = X + h1 * h2;            // h1 x h2 row-major: Z1 G Z2^T
  double* ZG = W + h1 * h2;           // h1 x na row-major
  double* Jm = ZG + (size_t)h1 * t;   // h1 x h1
  double* Xp = Jm + h1 * h1;          // h2 x h1 row-major
  double* M1 = Xp + h2 * h1;          // h1 x h3 row-major: Z1 K3^T
  double* F = M1 + h1 * h3;           // h3 x h2 row-major: K3 Z2^T
  double* E = F + h3 * h2;            // h2 x h3 row-major: Xp M1
  double term1 = 0.0, corr = 0.0;
  if (h1 > 0 && h2 > 0) {
    for (int idx = threadIdx.x; idx < h1 * h2; idx += blockDim.x) {
      const int a = idx / h2, b = idx % h2;
      X[idx] = dot4(Zs + (o1 + a), hh, HJs + (o2 + b), hh, na);
    }
    for (int idx = threadIdx.x; idx < h1 * na; idx += blockDim.x) {
      const int a = idx / na, c = idx % na;
      // G is symmetric: G[e][c] read as G[c][e], consecutive c at consecutive addresses
      ZG[idx] = dot4(Zs + (o1 + a), hh, G + c, na, na);
    }
    for (int idx = threadIdx.x; idx < h1 * h3; idx += blockDim.x) {
      const int a = idx / h3, r = idx % h3;
      M1[idx] = dot4(Zs + (o1 + a), hh, HJs + (o3 + r), hh, na);
    }
    for (int idx = threadIdx.x; idx < h3 * h2; idx += blockDim.x) {
      const int r = idx / h2, b = idx % h2;
      F[idx] = dot4(HJs + (o3 + r), hh, Zs + (o2 + b), hh, na);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < h1 * h2; idx += blockDim.x) {
      const int a = idx / h2, b = idx % h2;
      W[idx] = dot4(ZG + a * na, 1, Zs + (o2 + b), hh, na);
    }
    __syncthreads();
    {
      const int mx = (h1 > h2) ? h1 : h2;
      cta_pinv_rows(X, Jm, h1, h2, Xp, fmax((double)mx * 2.220446049250313e-16, d.sk_rel), ZG /* free after W */,
                    sh);
    }
    for (int idx = threadIdx.x; idx < h2 * h3; idx += blockDim.x) {
      const int a = idx / h3, r = idx % h3;
      double acc = 0.0;
      for (int b = 0; b < h1; ++b) acc += Xp[a * h1 + b] * M1[b * h3 + r];
      E[idx] = acc;
    }
    __syncthreads();
    double p1 = 0.0;
    for (int idx = threadIdx.x; idx < h2 * h1; idx += blockDim.x) {
      const int a = idx / h1, b = idx % h1;
      p1 += Xp[idx] * W[b * h2 + a];
    }
    term1 = block_sum(p1, sh);
    double p2 = 0.0;
    for (int idx = threadIdx.x; idx < h3 * h2; idx += blockDim.x) {
      const int r = idx / h2, a = idx % h2;
      p2 += F[idx] * E[a * h3 + r];
    }
    corr = block_sum(p2, sh);
  }
  double p3 = 0.0;
  for (int idx = threadIdx.x; idx < h3 * na; idx += blockDim.x) {
    const int r = idx % h3, c = idx / h3;
    p3 += Zs[(o3 + r) + (size_t)c * hh] * HJs[(o3 + r) + (size_t)c * hh];
  }
  const double direct = block_sum(p3, sh);
  if (threadIdx.x == 0) {
    const double cross = term1 + (direct - corr) / (double)h3;
    const double fro = d.scal[fro_slot];
    d.scal[SCAL_EST + q] = fro - 2.0 * cross + trg;
    // Every term of the estimate is a sum over the basis expansion A_J P; with reduced-
    // precision sketches and Gram (relative accuracy sk_rel) each carries a rounding error of
    // about sk_rel x sum_j sum_a G_aa P_aj^2, the energy of the expansion before cancellation.
    d.scal[SCAL_UNC + q] = fro > 0.0 ? d.sk_rel * ener / fro : 0.0;
  }
}

// ---------------------------------------------------------------- commit P = P_{q*}
// q* = argmin of the estimates (Algorithm 8), over the candidates whose estimate the rounding
// of a reduced-precision sketch cannot overturn (uncertainty <= 0.1 ||A_obs||^2): a candidate
// whose coefficients cancel far beyond that precision can have an estimate of any sign and
// size.  If no candidate qualifies, the one with the smallest uncertainty.  With FP64 sketches
// every uncertainty is 0 and this is the plain argmin.
__device__ __forceinline__ int choose_q(const double* scal) {
  const double* e = scal + SCAL_EST;
  const double* u = scal + SCAL_UNC;
  int q = -1;
  for (int i = 0; i < 4; ++i)
    if (u[i] <= 0.1 && (q < 0 || e[i] < e[q])) q = i;
  if (q >= 0) return q;
  q = 0;
  for (int i = 1; i < 4; ++i) if (u[i] < u[q]) q = i;
  return q;
}

__global__ void commit_kernel(Dev d, int64_t n_obs) {
  const int t = d.t;
  const int q = choose_q(d.scal);
  const double* Pq = d.cand + (size_t)q * t * d.n_cap;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (int64_t)t * n_obs;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % t);
    const int64_t j = idx / t;
    const int a = d.posof[i];
    d.P[i + (size_t)j * t] = (a >= 0) ? Pq[a + (size_t)j * t] : 0.0;
  }
}

// The end of a step's tail: its decision and counts go to the handle's reporting state (gmeta,
// and the basis it leaves as gjcp / gslotp, which equal the live basis once no step is in
// flight).
__global__ void finish_kernel(Dev d, int batch, int64_t n_obs, int* gmeta, int64_t* gjcp, int* gslotp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  d.meta[META_QSTAR] = 4 + choose_q(d.scal);
  d.meta[META_BATCH] = batch + 1;
  d.meta[META_NPREV] = (int)n_obs;
  for (int i = 0; i < META_LEN; ++i) gmeta[i] = d.meta[i];
  for (int i = 0; i < d.t; ++i) { gjcp[i] = d.JC[i]; gslotp[i] = d.slotC[i]; }
}

__global__ void reset_kernel(Dev d) {
  const int t = d.t;
  for (int i = threadIdx.x; i < t; i += blockDim.x) {
    d.JC[i] = -1; d.JC_prev[i] = -1; d.slotC[i] = -1; d.slotC_prev[i] = -1;
    for (int k = 0; k < d.la; ++k) d.dslot_all[(size_t)k * t + i] = k * t + i;
    d.tau_old[i] = 1.0; d.JD[i] = -1;
  }
  if (threadIdx.x == 0) {
    d.fro2[0] = 0.0; d.fro2[1] = 0.0;
    for (int i = 0; i < META_LEN; ++i) d.meta[i] = 0;
    for (int i = 0; i < SCAL_LEN; ++i) d.scal[i] = 0.0;
    *d.err = 0;
  }
}



int launch_reset_state(const Dev& d, cudaStream_t st) {
  reset_kernel<<<1, 256, 0, st>>>(d);
  cudaMemsetAsync(d.SSt, 0, sizeof(double) * (size_t)d.s * d.s, st);
  cudaMemsetAsync(d.Gp, 0, sizeof(double) * (size_t)d.npool * d.npool, st);
  return 1;
}

int launch_batch_lambda(const Dev& d, int batch, cudaStream_t st) {
  const WorkLayout w = layout(d);
  const bool odd = batch & 1;
  return launch_lambda(d, batch, d.work, odd ? w.eigA2 : w.eigA, odd ? w.eigR2 : w.eigR, odd ? w.eigD2 : w.eigD,
                       odd ? w.eigE2 : w.eigE, odd ? w.beta2 : w.beta, odd ? w.vhead2 : w.vhead,
                       odd ? w.eigP2 : w.eigP, odd ? w.mu2 : w.mu, odd ? w.ldld2 : w.ldld, odd ? w.ldll2 : w.ldll,
                       odd ? d.gbar + 8 : d.gbar, d.n_sm, st);
}

int launch_batch_select(const Dev& d, const Dev& r, int count, int64_t n_obs, int batch, cudaStream_t st,
                        cudaEvent_t ev_scores, cudaEvent_t ev_wait_rec, cudaEvent_t* tl) {
  const WorkLayout w = layout(d);
  const int64_t jd0 = n_obs - count;
  const bool odd = batch & 1;
  if (tl) cudaEventRecord(tl[TL_TAIL0], st);
  int nk = launch_scores(d, count, jd0, d.work, odd ? w.eigR2 : w.eigR, odd ? w.beta2 : w.beta,
                         odd ? w.vhead2 : w.vhead, odd ? w.ldld2 : w.ldld, odd ? w.ldll2 : w.ldll, w.svec,
                         (int)vec_stride(d.s, d.t), st);
  if (ev_scores) cudaEventRecord(ev_scores, st);
  if (tl) cudaEventRecord(tl[TL_SCORES], st);
  const int nu = d.t * (count + 2);
  uniforms_kernel<<<(nu + 255) / 256, 256, 0, st>>>(d, d.work + w.unif, count, batch);
  // the record this step writes was last read by the tail of step batch - 2
  if (ev_wait_rec) cudaStreamWaitEvent(st, ev_wait_rec, 0);
  {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
      attr = true;
    }
    const bool stage_u = select_smem_bytes(d.t, count, true, d.npool) <= 160 * 1024;
    select_kernel<<<1, 256, select_smem_bytes(d.t, count, stage_u, d.npool), st>>>(d, r, d.work + w.unif, count,
                                                                         stage_u ? 1 : 0, jd0, batch);
  }
  if (tl) cudaEventRecord(tl[TL_SELECT], st);
  return nk + 2;
}

int launch_batch_tail(const Dev& d, int count, int64_t n_obs, int64_t n_prev, int batch,
                      cudaStream_t st, cudaStream_t stg, cudaEvent_t ev_fork, cudaEvent_t ev_gram,
                      int* gmeta, int64_t* gjcp, int* gslotp, cudaEvent_t* tl) {
  (void)count;
  const WorkLayout w = layout(d);
  if (tl) cudaEventRecord(tl[TL_QR0], st);
  // Gram side on stg (basis Gram, G, its Cholesky factor, T of Algorithm 7), sketch side
  // (gather, Householder QRs) on st; they join before the coefficient kernel.
  cudaEventRecord(ev_fork, st);
  cudaStreamWaitEvent(stg, ev_fork, 0);
  if (tl) cudaEventRecord(tl[TL_GRAM0], stg);
  int ngk = 2;
  if (d.dtype == 1 && d.tc_part) {
    ngk = launch_tc_gram(d, d.tc_blocks, d.tg_part, stg);
    if (ngk < 0) return 0;
  } else {
    dim3 gg((d.t + 63) / 64, (2 * d.t + 63) / 64, d.gram_split);
    if (d.dtype == 0) basis_gram_kernel<double><<<gg, 256, 0, stg>>>(d);
    else basis_gram_kernel<float><<<gg, 256, 0, stg>>>(d);
    gram_reduce_kernel<<<(d.t * 2 * d.t + 255) / 256, 256, 0, stg>>>(d, d.gram_split);
  }
  if (d.allreduce) {
    // row shard: the partial Gram entries of this step summed over the shards
    const int nb = (2 * d.t * d.t + 255) / 256;
    gram_pack_kernel<<<nb, 256, 0, stg>>>(d);
    if (((rid_allreduce_fn)d.allreduce)(d.xbuf, 2 * (int64_t)d.t * d.t, (void*)stg, d.allreduce_user) != 0) return 0;
    gram_unpack_kernel<<<nb, 256, 0, stg>>>(d);
    ngk += 2;
  }
  gather_kernel<false><<<d.n_sm, 256, 0, stg>>>(d, w);
  {
    static int staged = -1;
    if (staged < 0)
      staged = cudaFuncSetAttribute(gram_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kCholSmemBytes) == cudaSuccess ? 1 : 0;
    gram_chol_kernel<<<1, 1024, staged ? kCholSmemBytes : 0, stg>>>(d, w, staged, d.gram_rho0);
  }
  tsolve_kernel<<<(d.t + 7) / 8, 256, 0, stg>>>(d, w);
  if (tl) cudaEventRecord(tl[TL_GRAM1], stg);
  cudaEventRecord(ev_gram, stg);
  gather_kernel<true><<<d.n_sm, 256, 0, st>>>(d, w);
  if (!launch_qr_coop(d, d.work + w.QR4, d.work + w.b4, d.work + w.h4, d.work + w.r4, d.work + w.QR6,
                      d.work + w.b6, d.work + w.h6, d.work + w.r6, d.gbar2, st))
    return 0;
  qr_prep_kernel<<<1, 256, 0, st>>>(d, w);
  qform_kernel<<<(2 * d.t + 7) / 8, 256, 0, st>>>(d, w);
  {
    const unsigned gm = (unsigned)((d.t + 31) / 32);
    proj_gemm_kernel<<<dim3(gm, (unsigned)((n_obs + 31) / 32)), 256, 0, st>>>(d, w, 0, n_obs);
    proj_gemm_kernel<<<dim3(gm, (unsigned)((n_obs + 31) / 32)), 256, 0, st>>>(d, w, 1, n_obs);
    proj_gemm_kernel<<<dim3(gm, gm), 256, 0, st>>>(d, w, 2, n_obs);
  }
  if (tl) cudaEventRecord(tl[TL_QR1], st);
  cudaStreamWaitEvent(st, ev_gram, 0);
  coeff_kernel<<<kApplyBlocks, kApplyThreads, 0, st>>>(d, w, n_obs, n_prev);
  const int nchunk = (int)((n_obs + kHutChunk - 1) / kHutChunk);
  hutch_partial_kernel<<<dim3(nchunk, 4), 256, 0, st>>>(d, w, n_obs);
  {
    static int staged = -1;
    if (staged < 0)
      staged = cudaFuncSetAttribute(hutch_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kHutchSmemBytes) == cudaSuccess ? 1 : 0;
    hutch_finish_kernel<<<4, 512, staged ? kHutchSmemBytes : 0, st>>>(d, w, nchunk, staged,
                                                                      SCAL_FRO0 + (batch & 7));
  }
  commit_kernel<<<kApplyBlocks, 256, 0, st>>>(d, n_obs);
  finish_kernel<<<1, 32, 0, st>>>(d, batch, n_obs, gmeta, gjcp, gslotp);
  if (tl) cudaEventRecord(tl[TL_TAIL1], st);
  return 16 + ngk;
}

}  // namespace rid
