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
#include "philox.cuh"

namespace grest {

namespace {

template <typename T>
__global__ void k_omega(T* Om, int64_t ld, int64_t S, int q, uint64_t seed, uint64_t step) {
  const int64_t total = S * q;
  const int64_t nblk = (total + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)b, step, 0ull, 0ull};
    rng::philox4x64_10(c, seed, 0x47524553ull);
    double z[4];
    rng::box_muller(c[0], c[1], z[0], z[1]);
    rng::box_muller(c[2], c[3], z[2], z[3]);
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
