// Philox4x32-10 counter-based generator, from the published definition of
// Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11). Usable on host and device; identical bits on both.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PQMC_HD __host__ __device__ __forceinline__
#else
#define PQMC_HD inline
#endif

namespace pqmc {

struct U4 { uint32_t x0, x1, x2, x3; };

PQMC_HD void mul_hi_lo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

// Ten Philox rounds on counter (c0..c3) with key (k0, k1); the key advances
// by the Weyl increments between rounds.
PQMC_HD U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mul_hi_lo(0xD2511F53u, c0, hi0, lo0);
    mul_hi_lo(0xCD9E8D57u, c2, hi1, lo1);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// Metropolis uniform in [0, 1) with 53 random bits, for proposal
// (site i, slice tau, sweep, chain).
PQMC_HD double metropolis_uniform(uint64_t seed, uint32_t chain, uint32_t sweep, uint32_t tau, uint32_t i) {
  const U4 x = philox4x32_10(i, tau, sweep, chain, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t m = ((uint64_t)x.x0 << 21) | (uint64_t)(x.x1 >> 11);
  return (double)m * 0x1.0p-53;
}

constexpr uint32_t kInitSweep = 0xFFFFFFFFu;

// Initial Ising field at (site i, slice tau): +1 iff bit 0 of word x2 is set.
PQMC_HD int initial_field(uint64_t seed, uint32_t chain, uint32_t tau, uint32_t i) {
  const U4 x = philox4x32_10(i, tau, kInitSweep, chain, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (x.x2 & 1u) ? 1 : -1;
}

}  // namespace pqmc
