// philox.cuh -- counter-based Gaussian noise for the Brownian terms of
// Sec. II.C (Eqs. 20-24).
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each
// multiplying words 0 and 2 by 0xD2511F53 and 0xCD9E8D57, swapping the
// product halves into the next counter and mixing in the key, which is
// advanced by 0x9E3779B9 / 0xBB67AE85 between rounds.  The counter is
// (k_lo, tag_i, tag_j, 2 k_hi + block) with tag_i < tag_j for a pair and
// tag_i == tag_j for the one-body terms; the key is the 64-bit seed.  So the
// noise of a pair depends only on (seed, k, i, j), whichever thread, order or
// device draws it.
#pragma once
#include <stdint.h>

namespace susp {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Two Philox blocks -> six standard normal deviates (double precision).
// u = (w + 1/2) 2^-32 lies strictly inside (0, 1).
__device__ __forceinline__ void gauss6_f64(uint32_t k0, uint32_t k1,
                                           long long k, uint32_t t1,
                                           uint32_t t2, double g[6]) {
  const uint32_t klo = (uint32_t)((unsigned long long)k & 0xffffffffull);
  const uint32_t khi = (uint32_t)((unsigned long long)k >> 32);
  const U4 a = philox4x32_10(U4{klo, t1, t2, 2u * khi}, k0, k1);
  const U4 b = philox4x32_10(U4{klo, t1, t2, 2u * khi + 1u}, k0, k1);
  const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
  const double two_pi = 6.283185307179586476925286766559;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double ua = ((double)w[2 * q] + 0.5) * 2.3283064365386962890625e-10;
    const double ub = ((double)w[2 * q + 1] + 0.5) * 2.3283064365386962890625e-10;
    const double rr = sqrt(-2.0 * log(ua));
    double s, c;
    sincos(two_pi * ub, &s, &c);
    g[2 * q] = rr * c;
    g[2 * q + 1] = rr * s;
  }
}

// Single-precision variant for the mixed path: 24-bit uniforms
// u = (w >> 8 + 1/2) 2^-24 in (0, 1), hardware log2 and sin/cos of the
// angle 2 pi u - pi in [-pi, pi) (the special-function unit is accurate to
// ~1e-6 absolute on that range; cos and sin of the shifted angle are the
// negatives of those of 2 pi u, so the deviates are negated back and follow
// the double-precision ones to single-precision accuracy).
__device__ __forceinline__ void gauss6_f32(uint32_t k0, uint32_t k1,
                                           long long k, uint32_t t1,
                                           uint32_t t2, float g[6]) {
  const uint32_t klo = (uint32_t)((unsigned long long)k & 0xffffffffull);
  const uint32_t khi = (uint32_t)((unsigned long long)k >> 32);
  const U4 a = philox4x32_10(U4{klo, t1, t2, 2u * khi}, k0, k1);
  const U4 b = philox4x32_10(U4{klo, t1, t2, 2u * khi + 1u}, k0, k1);
  const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float ua = ((float)(w[2 * q] >> 8) + 0.5f) * 5.9604644775390625e-08f;
    const float ub = ((float)(w[2 * q + 1] >> 8) + 0.5f) * 5.9604644775390625e-08f;
    const float rr = sqrtf(-2.0f * __logf(ua));
    float s, c;
    __sincosf(6.2831853071795865f * ub - 3.14159265358979f, &s, &c);
    g[2 * q] = -rr * c;
    g[2 * q + 1] = -rr * s;
  }
}

}  // namespace susp
