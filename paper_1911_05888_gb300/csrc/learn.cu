// Learned element-local post-smoother: kernels for features, a two-layer
// perceptron (training and inference), Adam, and the accept/reject step.
//
// Not part of the paper's method: after the post-smoothing sweeps of the
// finest level, each element's residual and the residuals of its 2d face
// neighbours (scaled by 1/||r_i||) are mapped by a small MLP to a correction
// of x_i (scaled back by ||r_i||).  Whether a correction is kept is decided
// by the outer iteration in api.cu (its residual contraction against the plain
// cycles' measured contraction).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "stk_internal.h"

namespace stk {

// ---- features --------------------------------------------------------------------
// F[i] = [r_i, r_{i-e_0}, r_{i+e_0}, ..., r_{i+e_{d-1}}] / (||r_i|| + tiny), zeros
// for missing neighbours; nrm[i] = ||r_i||.  Neighbour slots 0..2d-1 of the
// pattern are -e_0, +e_0, -e_1, ...  Rows of F are padded to ldf columns.
__global__ void features_kernel(int ne, int nb, int nface, int NO, int ldf, const int* __restrict__ nbr_nat,
                                const float* __restrict__ r, float* __restrict__ F, float* __restrict__ nrm) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (e >= ne) return;
  float ss = 0.f;
  for (int k = lane; k < nb; k += 32) {
    const float v = r[(size_t)e * nb + k];
    ss += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float n = sqrtf(ss);
  const float inv = 1.f / (n + 1e-30f);
  if (lane == 0) nrm[e] = n;
  float* row = F + (size_t)e * ldf;
  for (int k = lane; k < nb; k += 32) row[k] = r[(size_t)e * nb + k] * inv;
  for (int f = 0; f < nface; ++f) {
    const int j = nbr_nat[(size_t)e * NO + f];
    for (int k = lane; k < nb; k += 32) row[(f + 1) * nb + k] = (j >= 0) ? r[(size_t)j * nb + k] * inv : 0.f;
  }
  for (int k = (1 + nface) * nb + lane; k < ldf; k += 32) row[k] = 0.f;
}

// ---- dense layers: C = act(op(A) op(B) + bias) ---------------------------------
// A is M x K (or K x M when ta), B is K x N (or N x K when tb), row-major with
// leading dimensions lda, ldb; C is M x N with ldc.  act: 0 none, 1 tanh.
// beta accumulates into C (0 overwrites).  64 x 64 tiles, 4 x 4 per thread.
__global__ void sgemm_kernel(int M, int N, int K, int ta, int tb, const float* __restrict__ A, int lda,
                             const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                             const float* __restrict__ bias, int act, float alpha, float beta) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 256 threads
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      const int mm = i / 16, kk = i % 16;
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = va;
      const int nn = i / 16;
      const int gn = n0 + nn;
      float vb = 0.f;
      if (gn < N && gk < K) vb = tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[kk][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = alpha * acc[i][j] + (bias ? bias[gn] : 0.f);
      if (beta != 0.f) v += beta * C[(size_t)gm * ldc + gn];
      if (act == 1) v = tanhf(v);
      C[(size_t)gm * ldc + gn] = v;
    }
  }
}

// column sums of an M x N matrix (bias gradients): out[n] = alpha * sum_m A[m][n]
__global__ void colsum_kernel(int M, int N, const float* __restrict__ A, int lda, float* __restrict__ out,
                              float alpha) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += A[(size_t)m * lda + n];
  out[n] = alpha * s;
}

// dY = 2 scale (Y - T) (scale = 1 / rows); per-block partial sums of
// (Y - T)^2 in FP64 (dY may alias Y: each entry is read before it is written)
__global__ void mse_grad_kernel(int64_t n, float scale, const float* Y, const float* __restrict__ T, float* dY,
                                double* __restrict__ loss_part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * scale * d;
    acc += (double)d * (double)d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

// dZ = dH * (1 - H^2)   (tanh derivative)
__global__ void tanh_back_kernel(int64_t n, const float* __restrict__ H, float* __restrict__ dH) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dH[i] *= (1.f - H[i] * H[i]);
}

__global__ void adam_kernel(int64_t n, float lr, float b1, float b2, float c1, float c2, float eps,
                            float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// x_t = x + nrm_i * Y_i  (correction in natural element order)
__global__ void apply_correction_kernel(int ne, int nb, int ldy, const float* __restrict__ x,
                                        const float* __restrict__ nrm, const float* __restrict__ Y,
                                        float* __restrict__ xt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ne * nb) return;
  const int e = (int)(i / nb), k = (int)(i - (int64_t)e * nb);
  xt[i] = x[i] + nrm[e] * Y[(size_t)e * ldy + k];
}

// sum of squares of a float vector into out[0] (double), deterministic two-pass
__global__ void sumsq_f_partial_kernel(int64_t n, const float* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[i] * (double)x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(int n, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// Counter-based uniform(-1, 1) from (seed, index): splitmix64 finaliser.
__device__ inline float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed * 0x9E3779B97F4A7C15ULL + i + 0x632BE59BD9B4E019ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Smooth random field: mode 0 of every variable is a sum of 4 seeded plane
// waves of the element centre; higher modes carry 1e-3 white noise.
// ctr (may be NULL): element centres [ne][d] in box-relative coordinates, for
// meshes whose element index is not a grid index (cut cells).
__global__ void smooth_field_kernel(int ne, int nb, int s, int d, const int* n, const double* ctr, uint64_t seed,
                                    float* __restrict__ x) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ne * nb) return;
  const int e = (int)(i / nb), k = (int)(i - (int64_t)e * nb);
  const int v = k / s, mode = k - v * s;
  if (mode != 0) {
    x[i] = 1e-3f * hash_uniform(seed, i);
    return;
  }
  double c[3];
  if (ctr) {
    for (int a = 0; a < d; ++a) c[a] = ctr[(size_t)e * d + a];
  } else {
    const int idx[3] = {e % n[0], (e / n[0]) % n[1], d == 3 ? e / (n[0] * n[1]) : 0};
    for (int a = 0; a < d; ++a) c[a] = (idx[a] + 0.5) / n[a];
  }
  float acc = 0.f;
  for (int w = 0; w < 4; ++w) {
    const uint64_t base = ((uint64_t)v * 4 + w) * 8;
    double ph = 3.14159265358979 * hash_uniform(seed ^ 0xABCDEFULL, base);
    for (int a = 0; a < d; ++a) {
      const int kk = (int)floorf(2.5f + 2.5f * hash_uniform(seed ^ 0x1234567ULL, base + 1 + a));   // 0..5
      ph += 6.283185307179586 * kk * c[a];
    }
    const float amp = hash_uniform(seed ^ 0x55AA55ULL, base + 7) / (1.f + w);
    acc += amp * (float)sin(ph);
  }
  x[i] = acc;
}

// T[i] = (x*_i - x_i) / ||r_i||
__global__ void target_kernel(int ne, int nb, int ldt, const float* __restrict__ xs, const float* __restrict__ x,
                              const float* __restrict__ nrm, float* __restrict__ T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ne * nb) return;
  const int e = (int)(i / nb), k = (int)(i - (int64_t)e * nb);
  T[(size_t)e * ldt + k] = (xs[i] - x[i]) / (nrm[e] + 1e-30f);
}

__global__ void scale_f_kernel(int64_t n, float a, const float* __restrict__ x, float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

// g <- 2 g / ||r||^2 with ||r||^2 = sums[0]
__global__ void scale_by_norm_kernel(int64_t n, const double* __restrict__ sums, float* __restrict__ g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] = (float)(2.0 * (double)g[i] / (sums[0] + 1e-300));
}

// ---------------------------------------------------------------------------
cudaError_t launch_scale_by_norm(int64_t n, const double* sums, float* g, cudaStream_t st) {
  scale_by_norm_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, sums, g);
  return cudaGetLastError();
}

cudaError_t launch_scale_f(int64_t n, float a, const float* x, float* y, cudaStream_t st) {
  scale_f_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

cudaError_t launch_features(int ne, int nb, int nface, int NO, int ldf, const int* nbr_nat, const float* r, float* F,
                            float* nrm, cudaStream_t st) {
  features_kernel<<<(unsigned)(((int64_t)ne * 32 + 255) / 256), 256, 0, st>>>(ne, nb, nface, NO, ldf, nbr_nat, r, F, nrm);
  return cudaGetLastError();
}

cudaError_t launch_sgemm(int M, int N, int K, int ta, int tb, const float* A, int lda, const float* B, int ldb,
                         float* C, int ldc, const float* bias, int act, float alpha, float beta, cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  sgemm_kernel<<<grid, 256, 0, st>>>(M, N, K, ta, tb, A, lda, B, ldb, C, ldc, bias, act, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_colsum(int M, int N, const float* A, int lda, float* out, float alpha, cudaStream_t st) {
  colsum_kernel<<<(N + 127) / 128, 128, 0, st>>>(M, N, A, lda, out, alpha);
  return cudaGetLastError();
}

__global__ void fill_kernel(double* v, double a) { v[0] = a; }
cudaError_t launch_fill(double* v, double a, cudaStream_t st) {
  fill_kernel<<<1, 1, 0, st>>>(v, a);
  return cudaGetLastError();
}
cudaError_t launch_mse_grad(int64_t n, float scale, const float* Y, const float* T, float* dY, double* part,
                            double* out, cudaStream_t st) {
  mse_grad_kernel<<<256, 256, 0, st>>>(n, scale, Y, T, dY, part);
  sum_partials_kernel<<<1, 256, 0, st>>>(256, part, out);
  return cudaGetLastError();
}

cudaError_t launch_tanh_back(int64_t n, const float* H, float* dH, cudaStream_t st) {
  tanh_back_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, H, dH);
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float lr, float b1, float b2, float c1, float c2, float eps, float* w,
                        const float* g, float* m, float* v, cudaStream_t st) {
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, lr, b1, b2, c1, c2, eps, w, g, m, v);
  return cudaGetLastError();
}

cudaError_t launch_apply_correction(int ne, int nb, int ldy, const float* x, const float* nrm, const float* Y, float* xt,
                                    cudaStream_t st) {
  int64_t n = (int64_t)ne * nb;
  apply_correction_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ne, nb, ldy, x, nrm, Y, xt);
  return cudaGetLastError();
}


cudaError_t launch_sumsq_f(int64_t n, const float* x, double* part, double* out, cudaStream_t st) {
  sumsq_f_partial_kernel<<<512, 256, 0, st>>>(n, x, part);
  sum_partials_kernel<<<1, 256, 0, st>>>(512, part, out);
  return cudaGetLastError();
}

cudaError_t launch_smooth_field(int ne, int nb, int s, int d, const int* n_dev, const double* ctr, uint64_t seed,
                                float* x, cudaStream_t st) {
  int64_t n = (int64_t)ne * nb;
  smooth_field_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ne, nb, s, d, n_dev, ctr, seed, x);
  return cudaGetLastError();
}

cudaError_t launch_target(int ne, int nb, int ldt, const float* xs, const float* x, const float* nrm, float* T,
                          cudaStream_t st) {
  int64_t n = (int64_t)ne * nb;
  target_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ne, nb, ldt, xs, x, nrm, T);
  return cudaGetLastError();
}

}  // namespace stk
