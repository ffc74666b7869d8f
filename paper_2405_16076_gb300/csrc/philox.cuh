// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11)
// and the random streams of the online randomized ID (Algorithm 3).
//
// Definition: 128-bit counter (x0..x3), 64-bit key (k0, k1); each of the 10
// rounds multiplies x0 by 0xD2511F53 and x2 by 0xCD9E8D57 (32x32 -> 64 bit)
// and forms (hi(x2*M1) ^ x1 ^ k0, lo(x2*M1), hi(x0*M0) ^ x3 ^ k1, lo(x0*M0));
// before every round after the first the key is bumped by (0x9E3779B9,
// 0xBB67AE85).
//
// Stream layout (counter = (c0, c1, tag, c3), key = (seed_lo, seed_hi)):
//   Rademacher Omega[r][i]: with j = i mod 128, word w = j/32, e = j mod 32, pair p = e/2:
//                           bit 15-p (even e) or 31-p (odd e) of word w of
//                           Philox(i/128, r, RAD, 0); set bit = -1.  A pair of
//                           coordinates is then one AND/OR of a shifted word.
//   Gaussian   Omega[r][i]: Box-Muller from Philox(i/2, r, GAU, 0); even i cosine, odd i sine
//   uniform u(batch, i, r): 53-bit uniform from words 0,1 of Philox(i, r, UNI, batch)
#pragma once
#include <stdint.h>

namespace rid {

constexpr uint32_t kTagRademacher = 0x52414431u;
constexpr uint32_t kTagGauss = 0x47415531u;
constexpr uint32_t kTagUniform = 0x554E4931u;
constexpr uint32_t kTagGradRademacher = 0x47524431u;
constexpr uint32_t kTagGradGauss = 0x47524731u;

struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                         uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
    const uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
    c0 = h1 ^ c1 ^ k0;
    c1 = l1;
    c2 = h0 ^ c3 ^ k1;
    c3 = l0;
  }
  return u32x4{c0, c1, c2, c3};
}

// (w0 >> 5) * 2^26 + (w1 >> 6), times 2^-53: an exact double in [0, 1).
__host__ __device__ __forceinline__ double uniform53(uint32_t w0, uint32_t w1) {
  const double a = (double)(w0 >> 5);
  const double b = (double)(w1 >> 6);
  return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0);
}

__host__ __device__ __forceinline__ double sample_uniform(uint64_t seed, uint32_t batch,
                                                          uint32_t i, uint32_t r) {
  u32x4 w = philox4x32_10(i, r, kTagUniform, batch, (uint32_t)seed, (uint32_t)(seed >> 32));
  return uniform53(w.x, w.y);
}

// One N(0,1) entry Omega[r][i] by Box-Muller (FP64; libm log/sqrt/cos/sin).
__device__ __forceinline__ double gauss_entry(uint64_t seed, uint32_t tag, uint32_t r, uint64_t i) {
  u32x4 w = philox4x32_10((uint32_t)(i >> 1), r, tag, 0, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = uniform53(w.x, w.y) + 0.5 * (1.0 / 9007199254740992.0);
  const double u2 = uniform53(w.z, w.w);
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  return (i & 1) ? rad * sin(ang) : rad * cos(ang);
}

// One Rademacher entry (r, i) of a +-1 stream with the layout above: bit 15 - p (even e) or
// 31 - p (odd e) of word (i mod 128) / 32 of Philox(i / 128, r, tag, 0), e = i mod 32,
// p = e / 2; a set bit is -1.
__device__ __forceinline__ double rademacher_entry(uint64_t seed, uint32_t tag, uint32_t r, uint64_t i) {
  const u32x4 w = philox4x32_10((uint32_t)(i >> 7), r, tag, 0, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t j = (uint32_t)(i & 127), e = j & 31, p = e >> 1;
  const uint32_t word = (j >> 5) == 0 ? w.x : (j >> 5) == 1 ? w.y : (j >> 5) == 2 ? w.z : w.w;
  const uint32_t bit = (e & 1) ? 31 - p : 15 - p;
  return ((word >> bit) & 1u) ? -1.0 : 1.0;
}

}  // namespace rid
