// Gaussian test matrix Omega of the RSVD step S.1 (Sec. 3.5).
//
// The paper asks for i.i.d. N(0,1) entries and names no generator.  This
// library draws them from Philox4x64-10 (Salmon, Moraes, Dror and Shaw,
// SC'11) followed by the Box-Muller transform, so a CPU implementation of the
// same published generator can reproduce Omega:
//   element (j, c) of the S x q matrix at update step t has linear index
//   e = j*q + c; block b = e / 4 is Philox4x64-10 of counter (b, t, 0, 0)
//   under key (seed, 0x47524553); words (0,1) and (2,3) of the block feed
//   Box-Muller, giving normals 0,1 and 2,3 of the block.  A uniform in (0,1]
//   is ((x >> 11) + 1) 2^-53 and one in [0,1) is (x >> 11) 2^-53; the first
//   word of a pair sets the radius sqrt(-2 ln u1), the second the angle 2 pi u2.
#include "common.cuh"

namespace grest {

namespace {

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

template <typename T>
__global__ void k_omega(T* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step) {
  const int64_t total = S * q;
  const int64_t nblk = (total + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)b, step, 0ull, 0ull};
    philox4x64_10(c, seed, 0x47524553ull);
    double z[4];
    box_muller(c[0], c[1], z[0], z[1]);
    box_muller(c[2], c[3], z[2], z[3]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int64_t e = 4 * b + t;
      if (e < total) Om[(e / q) * ld + (e % q)] = (T)z[t];
    }
  }
}

}  // namespace

template <typename T>
void gaussian_omega_t(T* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step, cudaStream_t s) {
  int64_t nblk = (S * q + 3) / 4;
  if (nblk <= 0) return;
  int64_t g = (nblk + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_omega<T><<<(unsigned)g, 256, 0, s>>>(Om, ld, S, q, seed, step);
}
void gaussian_omega(double* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step, cudaStream_t s) {
  gaussian_omega_t(Om, ld, S, q, seed, step, s);
}
void gaussian_omega(float* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step, cudaStream_t s) {
  gaussian_omega_t(Om, ld, S, q, seed, step, s);
}

}  // namespace grest
