// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11) and the Box-Muller
// transform: the generator of the RSVD test matrix Omega (Sec. 3.5, step
// S.1), shared by the single-graph and the grouped update.  The element
// layout and the uniform conventions are documented in rsvd.cu.
#pragma once
#include <stdint.h>

namespace grest {
namespace rng {

__device__ __forceinline__ void philox_round(uint64_t& x0, uint64_t& x1, uint64_t& x2, uint64_t& x3, uint64_t k0,
                                             uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t lo0 = M0 * x0, hi0 = __umul64hi(M0, x0);
  const uint64_t lo1 = M1 * x2, hi1 = __umul64hi(M1, x2);
  const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
  x0 = y0;
  x1 = lo1;
  x2 = y2;
  x3 = lo0;
}

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    philox_round(c[0], c[1], c[2], c[3], k0, k1);
  }
}

__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, double& z0, double& z1) {
  const double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)(b >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

}  // namespace rng
}  // namespace grest
