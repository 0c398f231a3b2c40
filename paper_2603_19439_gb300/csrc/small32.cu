// FP32 projected problems of the mixed path on one SM.
//
// The mixed path solves H = Z^T M Z, the CholQR Gram matrices and the RSVD
// Gram B_s B_s^T in FP32 arithmetic (their entries come from FP32 blocks).
// In FP32 one SM retires 128 FMAs per clock, so for small m (the whole matrix
// in shared memory) a single CTA of 1024 threads beats the cluster kernels,
// whose cost there is dominated by cluster barriers; for large m the rank-1/2
// updates are bound by one SM's shared-memory bandwidth and the cluster
// kernels win.
//   k_pchol_f32 : Cholesky with diagonal pivoting and the drop rule of the
//                 orthonormalization, then T = P R^{-1} (warp per column).
//   k_tridiag_f32 : Householder reduction to tridiagonal form; reflectors
//                 and their coefficients kept in FP32 for the back-transform.
// Storage outside the kernels (G, H, T, d, e) stays FP64.
#include <float.h>

#include "common.cuh"

namespace grest {

namespace {

constexpr int kT1 = 1024;

__device__ __forceinline__ float block_sum_f(float v, float* red, float* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float s = lane < nw ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) *out = s;
  }
  __syncthreads();
  return *out;
}

// Pivot k: the largest remaining Schur-complement diagonal (lowest index on
// ties); stop at the first pivot with R_kk^2 <= drop_tol^2 max(R_00^2,
// abs_ref^2).  Rows are not swapped: row piv[k] of A keeps the Schur row of
// step k, so R_{k,t} = A[piv[k]][piv[t]] / R_kk.  Outputs as k_pchol_cl +
// k_trinv: T (c x c, ldt) = P R^{-1} with zero columns >= rank, piv, info.
__global__ void __launch_bounds__(kT1, 1) k_pchol_f32(const double* G, int64_t ld, int c, double drop_tol,
                                                     double abs_ref, const double* abs_ref_ptr, double* Tm,
                                                     int64_t ldt, int* piv_out, double* info) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* A = reinterpret_cast<float*>(smraw);  // c x c
  float* rinv = A + (size_t)c * c;             // c
  int* piv = reinterpret_cast<int*>(rinv + c); // c
  int* done = piv + c;                         // c
  float* S = reinterpret_cast<float*>(done + c);  // 32 warps x c (inverse scratch)
  __shared__ double s_ref, s_thr, s_vlast, s_vdrop;
  __shared__ float s_ri;
  __shared__ int s_p, s_stop, s_rank;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < c * c; e += blockDim.x) {
    const int i = e / c, l = e % c;
    A[e] = (float)(i <= l ? G[(int64_t)i * ld + l] : G[(int64_t)l * ld + i]);
  }
  for (int l = tid; l < c; l += blockDim.x) done[l] = 0;
  if (tid == 0) {
    s_rank = c;
    s_vlast = 0.0;
    s_vdrop = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    if (wid == 0) {
      float bv = -1.f;
      int bi = c;
      for (int i = lane; i < c; i += 32) {
        if (done[i]) continue;
        const float d = A[(size_t)i * c + i];
        if (d > bv || (d == bv && i < bi)) { bv = d; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        const double v = (double)bv;
        if (k == 0) {
          const double a = abs_ref_ptr ? fabs(*abs_ref_ptr) : abs_ref;
          s_ref = fmax(v, a * a);
          s_thr = drop_tol * drop_tol * s_ref;
        }
        if (bi >= c || !(v > 0.0) || !(v > s_thr) || !isfinite(v)) {
          s_stop = 1;
          s_rank = k;
          s_vdrop = v > 0.0 ? v : 0.0;
        } else {
          s_stop = 0;
          const float ri = 1.f / sqrtf(bv);
          s_ri = ri;
          s_vlast = v;
          s_p = bi;
          piv[k] = bi;
          rinv[k] = ri;
          done[bi] = 1;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    const float ri2 = s_ri * s_ri;
    const float* Ap = A + (size_t)p * c;
    // Schur update of the rows and columns not pivoted yet
    for (int i = wid; i < c; i += nw) {
      if (done[i]) continue;
      const float f = Ap[i] * ri2;
      float* row = A + (size_t)i * c;
      for (int l = lane; l < c; l += 32)
        if (!done[l]) row[l] = fmaf(-f, Ap[l], row[l]);
    }
    __syncthreads();
  }
  const int rk = s_rank;
  if (tid == 0) {
    int t = rk;
    for (int l = 0; l < c; ++l)
      if (!done[l]) piv[t++] = l;
  }
  __syncthreads();
  // T = P R^{-1}: warp per column j, x = R^{-1} e_j by right-looking back
  // substitution with R_{i,t} = A[piv[i]][piv[t]] rinv[i]
  float* s = S + (size_t)wid * c;
  for (int j = wid; j < c; j += nw) {
    if (j >= rk) {
      for (int i = lane; i < c; i += 32) Tm[(int64_t)i * ldt + j] = 0.0;
      continue;
    }
    for (int i = lane; i < j; i += 32) s[i] = 0.f;
    float xt = rinv[j];
    if (lane == 0) s[j] = xt;
    __syncwarp();
    for (int t = j; t >= 1; --t) {
      const int pt = piv[t];
      for (int i = lane; i < t; i += 32) s[i] = fmaf(A[(size_t)piv[i] * c + pt] * rinv[i], xt, s[i]);
      __syncwarp();
      xt = -s[t - 1] * rinv[t - 1];
      __syncwarp();
      if (lane == 0) s[t - 1] = xt;
      __syncwarp();
    }
    for (int i = lane; i < c; i += 32) Tm[(int64_t)piv[i] * ldt + j] = i <= j ? (double)s[i] : 0.0;
    __syncwarp();
  }
  for (int l = tid; l < c; l += blockDim.x) piv_out[l] = piv[l];
  if (tid == 0) {
    const double ref = s_ref;
    info[0] = rk;
    info[1] = (rk > 0 && ref > 0.0) ? sqrt(s_vlast / ref) : 0.0;
    info[2] = (ref > 0.0 && s_vdrop > 0.0) ? sqrt(s_vdrop / ref) : 0.0;
    info[3] = 0.0;
  }
}

// Householder tridiagonalization of H (m x m, upper triangle read) in FP32:
// d, e (FP64 and FP32 copies), reflector v_j (v_0 = x_0 - alpha) in vf row j
// right of the diagonal (FP32, ld m) and beta_j.
__global__ void __launch_bounds__(kT1, 1) k_tridiag_f32(const double* H, int64_t ld, int m, double* d_out,
                                                       double* e_out, double* beta_out, float* df, float* ef,
                                                       float* betaf, float* vf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* A = reinterpret_cast<float*>(smraw);  // m x m
  float* v = A + (size_t)m * m;
  float* w = v + m;
  __shared__ float red[32];
  __shared__ float bc[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, l = e % m;
    A[e] = (float)(i <= l ? H[(int64_t)i * ld + l] : H[(int64_t)l * ld + i]);
  }
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const float* x = A + (size_t)j * m;
    float s = 0.f;
    for (int l = j + 1 + tid; l < m; l += blockDim.x) {
      const float xv = x[l];
      v[l] = xv;
      s = fmaf(xv, xv, s);
    }
    const float nrm2 = block_sum_f(s, red, bc);
    if (tid == 0) {
      const float x0 = v[j + 1];
      const float alpha = nrm2 > 0.f ? -copysignf(sqrtf(nrm2), x0) : 0.f;
      const float beta = nrm2 > 0.f ? 1.f / (nrm2 - alpha * x0) : 0.f;
      v[j + 1] = x0 - alpha;
      bc[1] = alpha;
      bc[2] = beta;
      d_out[j] = (double)A[(size_t)j * m + j];
      e_out[j] = (double)alpha;
      beta_out[j] = (double)beta;
      df[j] = A[(size_t)j * m + j];
      ef[j] = alpha;
      betaf[j] = beta;
    }
    __syncthreads();
    const float beta = bc[2];
    for (int l = j + 1 + tid; l < m; l += blockDim.x) vf[(size_t)j * m + l] = v[l];
    if (beta == 0.f) {
      __syncthreads();  // v is rewritten by the next step
      continue;
    }
    // p = beta B v, warp per row of the trailing block
    for (int i = j + 1 + wid; i < m; i += nw) {
      const float* row = A + (size_t)i * m;
      float a = 0.f;
      for (int l = j + 1 + lane; l < m; l += 32) a = fmaf(row[l], v[l], a);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (lane == 0) w[i] = beta * a;
    }
    __syncthreads();
    float t = 0.f;
    for (int i = j + 1 + tid; i < m; i += blockDim.x) t = fmaf(w[i], v[i], t);
    const float K = 0.5f * beta * block_sum_f(t, red, bc);
    for (int i = j + 1 + tid; i < m; i += blockDim.x) w[i] -= K * v[i];
    __syncthreads();
    // B -= v w^T + w v^T
    for (int i = j + 1 + wid; i < m; i += nw) {
      float* row = A + (size_t)i * m;
      const float vi = v[i], wi = w[i];
      for (int l = j + 1 + lane; l < m; l += 32) row[l] -= vi * w[l] + wi * v[l];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      d_out[m - 2] = (double)A[(size_t)(m - 2) * m + m - 2];
      d_out[m - 1] = (double)A[(size_t)(m - 1) * m + m - 1];
      e_out[m - 2] = (double)A[(size_t)(m - 2) * m + m - 1];
      df[m - 2] = A[(size_t)(m - 2) * m + m - 2];
      df[m - 1] = A[(size_t)(m - 1) * m + m - 1];
      ef[m - 2] = A[(size_t)(m - 2) * m + m - 1];
    } else {
      d_out[0] = (double)A[0];
      df[0] = A[0];
    }
    e_out[m - 1] = 0.0;
    ef[m - 1] = 0.f;
  }
}

size_t pchol_f32_smem(int c) { return sizeof(float) * ((size_t)c * c + c) + sizeof(int) * 2 * c + sizeof(float) * 32 * c; }
size_t tridiag_f32_smem(int m) { return sizeof(float) * ((size_t)m * m + 2 * m); }

}  // namespace

bool pchol_f32_1cta(const double* G, int64_t ldg, int c, double drop_tol, double abs_ref, const double* abs_ref_ptr,
                    double* Tm, int64_t ldt, int* piv, double* info, cudaStream_t s) {
  if (c < 1) return false;
  const size_t smem = pchol_f32_smem(c);
  if (!reserve_dynamic_smem(k_pchol_f32, smem)) return false;
  k_pchol_f32<<<1, kT1, smem, s>>>(G, ldg, c, drop_tol, abs_ref, abs_ref_ptr, Tm, ldt, piv, info);
  return true;
}

bool tridiag_f32_1cta(const double* H, int64_t ld, int m, double* d, double* e, double* beta, float* df, float* ef,
                      float* betaf, float* vf, cudaStream_t s) {
  if (m < 1) return false;
  const size_t smem = tridiag_f32_smem(m);
  if (!reserve_dynamic_smem(k_tridiag_f32, smem)) return false;
  k_tridiag_f32<<<1, kT1, smem, s>>>(H, ld, m, d, e, beta, df, ef, betaf, vf);
  return true;
}

}  // namespace grest
