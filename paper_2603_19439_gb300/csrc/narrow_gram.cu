// CUDA-core Gram C = X^T Y for FP32 blocks when one side is narrow (at most
// 64 columns): the projections X_bar^T Y of the mixed step (X_bar has K
// columns), C = X_bar^T Y1 of Sec. 3.3 and the coefficients of P_perp.  Such a
// product has a few flops per byte, so it runs on the CUDA cores, which use
// the row-major rows as they arrive (the tensor-core Gram must first
// transpose them into K-major operands).
//
// Precision: a product x_i y_j is exact inside the FMA; each thread sums
// 256-row spans of its rows in FP32 registers (the accumulation of the
// tensor-core kernel's FP32 spans) and adds every span (two-sum) into
// double-float accumulators kept in its own slots of shared memory.  Each CTA
// writes one FP64 partial; a second kernel adds the partials in FP64.
//
// Work split: a CTA holds G groups of ag x bg threads (G a power of two).
// Thread (ti, tj) of a group owns rows 8 ti + u (u < 8) and columns
// 4 tj + q (q < 4) of the result: per staged row it reads 8 values of the
// narrow block (two 16-byte loads, the same address across a warp) and 4 of
// the wide one (one conflict-free 16-byte load per lane) for 32 FMAs.  A slab
// of 16 G rows of both blocks arrives by two TMA tile loads into a ring of
// stages (zero-filled past the last row and column); group g takes rows
// 16 g .. 16 g + 15 of each slab.  At the end the groups' sums are added in
// FP64 in group order in shared memory.  The partials are summed by one warp
// per entry (fixed lane order and shuffle tree: deterministic results).
// Every mbarrier wait is bounded; on a timeout the CTA records an error,
// waits (bounded) for its copies in flight and returns.
#include "tc_util.cuh"

namespace grest {

using namespace tc;

namespace {

constexpr int kGroupRows = 16, kSpanRows = 256, kNarrowThreads = 256, kMaxStages = 8;
constexpr size_t kNarrowSmem = 112 * 1024;  // two CTAs per SM

inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t up128(size_t x) { return (x + 127) & ~(size_t)127; }

struct NarrowShape {
  int ag, bg, wa, wb, G, threads, stages, slab_rows;
  size_t acc_bytes, stage_bytes, smem;
};

// Shape of a narrow product (na <= 64 narrow columns, nw <= 256 wide ones);
// stages == 0 when it does not fit.
NarrowShape narrow_shape(int na, int nw) {
  NarrowShape s{};
  s.ag = (na + 7) / 8;
  s.bg = (nw + 3) / 4;
  s.wa = s.ag * 8;
  s.wb = s.bg * 4;
  const int gsz = s.ag * s.bg;
  for (int G = 8; G >= 1; G >>= 1) {
    if (G * gsz > kNarrowThreads) continue;
    const size_t acc = up128((size_t)64 * G * gsz * sizeof(float));
    const size_t st = up128((size_t)kGroupRows * G * (s.wa + s.wb) * sizeof(float));
    if (acc + 2 * st > kNarrowSmem) continue;
    if (G > 1 && acc + 3 * st > kNarrowSmem) continue;  // prefer more stages to more groups
    s.G = G;
    s.threads = G * gsz;
    s.slab_rows = kGroupRows * G;
    s.acc_bytes = acc;
    s.stage_bytes = st;
    s.stages = (int)((kNarrowSmem - acc) / st);
    if (s.stages > kMaxStages) s.stages = kMaxStages;
    s.smem = acc + s.stages * st;
    const size_t red = sizeof(double) * (size_t)na * nw;
    if (s.smem < red) s.smem = red;
    return s;
  }
  return s;
}

struct NarrowArgs {
  int a, b, wa, wb, stages, slab_rows;
  int64_t n, rows_per_cta;
  uint32_t acc_bytes, stage_bytes;
  double* part;
  int32_t* err;
};

// part[blockIdx.x][i][j] = sum over the CTA's rows of X[r][i] Y[r][j], i < a <= 64, j < b <= 256
template <int G>
__global__ void __launch_bounds__(kNarrowThreads, 2)
    k_gram_narrow(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY,
                  const NarrowArgs p) {
  extern __shared__ __align__(128) uint8_t nsm[];
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ int abort_flag;
  const int a = p.a, b = p.b, wa = p.wa, wb = p.wb, S = p.stages;
  const int bg = wb >> 2;
  const int gsz = (wa >> 3) * bg;
  const int tid = threadIdx.x, nt = blockDim.x;  // nt = G * gsz
  const int grp = tid / gsz, loc = tid - grp * gsz;
  const int ti = loc / bg, tj = loc - ti * bg;
  float* accs = reinterpret_cast<float*>(nsm);  // [64][nt]: hi of (u, v) at (4u + v) nt + tid, lo at (32 + 4u + v) nt + tid
  uint8_t* ring = nsm + p.acc_bytes;
  const int64_t r0 = blockIdx.x * p.rows_per_cta;
  const int64_t r1 = r0 + p.rows_per_cta < p.n ? r0 + p.rows_per_cta : p.n;
  const int nslab = r1 > r0 ? (int)((r1 - r0 + p.slab_rows - 1) / p.slab_rows) : 0;
  const uint32_t xbytes = (uint32_t)(p.slab_rows * wa * 4), txbytes = (uint32_t)(p.slab_rows * (wa + wb) * 4);
  if (tid == 0) {
    for (int q = 0; q < S; ++q) mbar_init(&full[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  for (int k = 0; k < 64; ++k) accs[k * nt + tid] = 0.f;
  __syncthreads();
  auto issue = [&](int sl) {  // thread 0: slab sl into stage sl % S
    uint8_t* dst = ring + (size_t)(sl % S) * p.stage_bytes;
    const int y = (int)(r0 + (int64_t)sl * p.slab_rows);
    mbar_expect_tx(&full[sl % S], txbytes);
    tma_load_2d(dst, &mapX, 0, y, &full[sl % S]);
    tma_load_2d(dst + xbytes, &mapY, 0, y, &full[sl % S]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < S - 1 && issued < nslab; ++issued) issue(issued);
  float acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  constexpr int kSlabsPerSpan = kSpanRows / kGroupRows;
  int consumed = 0;
  for (int sl = 0; sl < nslab; ++sl) {
    if (!mbar_wait(&full[sl % S], (uint32_t)((sl / S) & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;  // uniform: read after the barrier
    consumed = sl + 1;
    // refill the stage read in the previous iteration (every thread is past it)
    if (tid == 0 && issued < nslab && issued == sl + S - 1) issue(issued++);
    const uint8_t* st = ring + (size_t)(sl % S) * p.stage_bytes;
    const float* xs = reinterpret_cast<const float*>(st) + (grp * kGroupRows) * wa + ti * 8;
    const float* ys = reinterpret_cast<const float*>(st + xbytes) + (grp * kGroupRows) * wb + tj * 4;
#pragma unroll
    for (int q = 0; q < kGroupRows; ++q) {
      const float4 x0 = *reinterpret_cast<const float4*>(xs + q * wa);
      const float4 x1 = *reinterpret_cast<const float4*>(xs + q * wa + 4);
      const float4 y = *reinterpret_cast<const float4*>(ys + q * wb);
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
    }
    if ((sl + 1) % kSlabsPerSpan == 0 || sl + 1 == nslab) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float& hi = accs[(4 * u + v) * nt + tid];
          float& lo = accs[(32 + 4 * u + v) * nt + tid];
          const float x = acc[u][v];
          const float s = hi + x;
          const float bb = s - hi;
          lo += (hi - (s - bb)) + (x - bb);
          hi = s;
          acc[u][v] = 0.f;
        }
    }
  }
  if (abort_flag) {
    // copies issued but not consumed may still be landing: wait for them (bounded)
    if (tid == 0) {
      for (int sl = consumed; sl < issued; ++sl) mbar_wait(&full[sl % S], (uint32_t)((sl / S) & 1));
      atomicCAS(p.err, 0, DERR_TIMEOUT);
    }
    __syncthreads();
    return;
  }
  __syncthreads();
  double vals[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      vals[u][v] = (double)accs[(4 * u + v) * nt + tid] + (double)accs[(32 + 4 * u + v) * nt + tid];
  __syncthreads();
  // the groups' sums, added in group order into red[a][b] (FP64)
  double* red = reinterpret_cast<double*>(nsm);
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (grp == g) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = ti * 8 + u, j = tj * 4 + v;
          if (i < a && j < b) red[i * b + j] = g == 0 ? vals[u][v] : red[i * b + j] + vals[u][v];
        }
    }
    __syncthreads();
  }
  double* out = p.part + (int64_t)blockIdx.x * a * b;
  for (int e = tid; e < a * b; e += nt) out[e] = red[e];
}

// C[i][j] = sum over chunks of part[c][i][j] (transposed: part[c][j][i]); one
// warp per entry, lanes over chunks, then a fixed shuffle tree
__global__ void k_gram_narrow_reduce(const double* __restrict__ part, int64_t chunks, int a, int b, int transposed,
                                     double* C, int64_t ldc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)a * b) return;
  const int i = (int)(w / b), j = (int)(w % b);
  const int64_t off = transposed ? (int64_t)j * a + i : (int64_t)i * b + j;
  double s = 0.0;
  for (int64_t c = lane; c < chunks; c += 32) s += part[c * (int64_t)a * b + off];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) C[(int64_t)i * ldc + j] = s;
}

int sm_count() {
  static const int nsm = [] {
    int dev = 0, v = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
  }();
  return nsm;
}

template <int G>
int launch_narrow(const NarrowShape& sh, const CUtensorMap& mx, const CUtensorMap& my, NarrowArgs p, int64_t part_cap,
                  int64_t* ctas_out, cudaStream_t s) {
  if (!reserve_dynamic_smem(k_gram_narrow<G>, sh.smem)) return -1;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_narrow<G>, sh.threads, sh.smem);
  if (occ < 1) occ = 1;
  int64_t ctas = (int64_t)sm_count() * occ;
  if (ctas > cdiv64(p.n, kSpanRows)) ctas = cdiv64(p.n, kSpanRows);
  const int64_t cap = part_cap / ((int64_t)p.a * p.b);
  if (ctas > cap) ctas = cap;
  if (ctas < 1) return -1;
  int64_t rows = cdiv64(p.n, ctas);
  rows = cdiv64(rows, sh.slab_rows) * sh.slab_rows;
  ctas = cdiv64(p.n, rows);
  p.rows_per_cta = rows;
  k_gram_narrow<G><<<(unsigned)ctas, sh.threads, sh.smem, s>>>(mx, my, p);
  *ctas_out = ctas;
  return 0;
}

}  // namespace

bool gram_narrow_supported(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b) {
  const int na = a <= b ? a : b, nw = a <= b ? b : a;
  if (na < 1 || na > 64 || nw > 256) return false;
  if (narrow_shape(na, nw).stages == 0) return false;
  if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || (ldx & 3) || (ldy & 3)) return false;
  return encode_fn() != nullptr;
}

int gram_f32_narrow(const float* X, int64_t ldx, int a, const float* Y, int64_t ldy, int b, int64_t n, double* C,
                    int64_t ldc, double* part, int64_t part_cap, int32_t* err, cudaStream_t s) {
  if (n <= 0 || n > INT32_MAX || !gram_narrow_supported(X, ldx, a, Y, ldy, b)) return -1;
  // the narrow block goes on the left; a right-narrow product is computed
  // transposed and its partials are read transposed by the reduction
  const bool swap = a > b;
  const float* L = swap ? Y : X;
  const float* R = swap ? X : Y;
  const int64_t ldl = swap ? ldy : ldx, ldr = swap ? ldx : ldy;
  const int na = swap ? b : a, nw = swap ? a : b;
  const NarrowShape sh = narrow_shape(na, nw);
  CUtensorMap mx, my;
  if (!make_map_f32(&mx, L, n, na, ldl, sh.wa, sh.slab_rows, false) ||
      !make_map_f32(&my, R, n, nw, ldr, sh.wb, sh.slab_rows, false))
    return -1;
  NarrowArgs p;
  p.a = na;
  p.b = nw;
  p.wa = sh.wa;
  p.wb = sh.wb;
  p.stages = sh.stages;
  p.slab_rows = sh.slab_rows;
  p.n = n;
  p.rows_per_cta = 0;  // set at launch
  p.acc_bytes = (uint32_t)sh.acc_bytes;
  p.stage_bytes = (uint32_t)sh.stage_bytes;
  p.part = part;
  p.err = err;
  int64_t ctas = 0;
  int st = -1;
  switch (sh.G) {
    case 1: st = launch_narrow<1>(sh, mx, my, p, part_cap, &ctas, s); break;
    case 2: st = launch_narrow<2>(sh, mx, my, p, part_cap, &ctas, s); break;
    case 4: st = launch_narrow<4>(sh, mx, my, p, part_cap, &ctas, s); break;
    default: st = launch_narrow<8>(sh, mx, my, p, part_cap, &ctas, s); break;
  }
  if (st != 0) return -1;
  const int64_t warps = (int64_t)a * b;
  k_gram_narrow_reduce<<<(unsigned)cdiv64(warps * 32, 256), 256, 0, s>>>(part, ctas, a, b, swap ? 1 : 0, C, ldc);
  return 0;
}

}  // namespace grest
