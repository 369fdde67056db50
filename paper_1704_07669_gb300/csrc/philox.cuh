// Device-side Philox4x32-10 and Box-Muller normals: the Gaussian test matrix
// Omega of Alg. 4, step 3 ("Omega = randn(n, l)").
//
// Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds, each
// multiplying counter words 0 and 2 by fixed odd 32-bit constants, keeping the
// high and low halves of both products, and mixing the high halves with
// counter words 1 and 3 and the key; the two key words advance by fixed Weyl
// increments between rounds. Being counter-based, any entry of Omega can be
// produced by any thread from (row j, column group q, seed) alone.
//
// Uniforms: u = (x + 1/2) 2^-32 in FP64 (exact), strictly inside (0, 1).
// Normals:  Box & Muller (1958): r = sqrt(-2 ln u0), z0 = r cos(2 pi u1),
//           z1 = r sin(2 pi u1), evaluated in FP64 with CUDA's libm.
// Layout:   Omega[j, 4q + t] from counter (j lo, j hi, q, stream) and key
//           (seed lo, seed hi); words (x0, x1) -> (z0, z1), (x2, x3) -> (z2, z3).
#pragma once

#include <stdint.h>

namespace spca {

struct U32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mul_hi_lo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  const uint64_t prod = static_cast<uint64_t>(a) * static_cast<uint64_t>(b);
  hi = static_cast<uint32_t>(prod >> 32);
  lo = static_cast<uint32_t>(prod);
}

__host__ __device__ __forceinline__ U32x4 philox4x32_10(U32x4 ctr, uint32_t key0, uint32_t key1) {
  constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi_a, lo_a, hi_b, lo_b;
    mul_hi_lo(kMul0, ctr.x, hi_a, lo_a);
    mul_hi_lo(kMul1, ctr.z, hi_b, lo_b);
    U32x4 next;
    next.x = hi_b ^ ctr.y ^ key0;
    next.y = lo_b;
    next.z = hi_a ^ ctr.w ^ key1;
    next.w = lo_a;
    ctr = next;
    key0 += kWeyl0;
    key1 += kWeyl1;
  }
  return ctr;
}

__device__ __forceinline__ U32x4 omega_words_at(uint64_t seed, int64_t j, uint32_t q, uint32_t stream) {
  U32x4 c;
  c.x = static_cast<uint32_t>(static_cast<uint64_t>(j));
  c.y = static_cast<uint32_t>(static_cast<uint64_t>(j) >> 32);
  c.z = q;
  c.w = stream;
  return philox4x32_10(c, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

__device__ __forceinline__ double unit_open(uint32_t x) {
  return (static_cast<double>(x) + 0.5) * 0x1.0p-32;
}

// Two standard normals from two words.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1) {
  const double r = sqrt(-2.0 * log(unit_open(a)));
  double s, c;
  sincospi(2.0 * unit_open(b), &s, &c);
  z0 = r * c;
  z1 = r * s;
}

}  // namespace spca
