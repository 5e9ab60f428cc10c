// linalg.cu -- the d x d step of Eq. 2 for OLS / ridge: Cholesky H = L L^T
// and x^{t+1} = x^t + L^{-T} L^{-1} g.
//
// The factor is blocked in 32 x 32 tiles, right-looking, two launches per
// tile column: a one-CTA kernel factors the diagonal tile and solves the
// panel below it, then a grid of CTAs applies the rank-32 update to every
// trailing lower tile in parallel.  Tiles are padded with the identity so
// any d works.  The factor runs in FP64 (plain form) or FP32 (mixed form:
// there the Hessian itself carries TF32/BF16 input rounding, so the
// factorisation only has to be a good preconditioner; the iterate update
// x += delta stays FP64).  A pivot that is not positive records
// DEV_NOT_SPD in the status word.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

int chol_padded(int d) { return (d + 31) / 32 * 32; }

template <typename T>
__global__ void k_chol_init(const double* __restrict__ H, int d, int dp, T* __restrict__ L) {
  const int64_t total = (int64_t)dp * dp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / dp), j = (int)(e - (int64_t)i * dp);
    T v;
    if (i < d && j < d) v = (T)H[(int64_t)i * d + j];
    else v = (i == j) ? T(1) : T(0);
    L[e] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_chol_panel(T* __restrict__ L, int dp, int k,
                                                    int* status) {
  __shared__ T D[32][33];
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;  // ty in [0, 16): rows ty, ty + 16
  const int k0 = k * 32;
  D[ty][tx] = L[(int64_t)(k0 + ty) * dp + k0 + tx];
  D[ty + 16][tx] = L[(int64_t)(k0 + ty + 16) * dp + k0 + tx];
  __syncthreads();
  for (int j = 0; j < 32; ++j) {
    if (threadIdx.x == 0) {
      T p = D[j][j];
      if (!(p > T(0))) {
        set_status(status, DEV_NOT_SPD);
        p = T(1);
      }
      D[j][j] = sqrt(p);
    }
    __syncthreads();
    if (threadIdx.x < 32 && tx > j) D[tx][j] = D[tx][j] / D[j][j];
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = ty + 16 * h;
      if (r > j && tx > j && tx <= r) D[r][tx] -= D[r][j] * D[tx][j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = ty + 16 * h;
    L[(int64_t)(k0 + r) * dp + k0 + tx] = (tx <= r) ? D[r][tx] : T(0);
  }
  __shared__ T R[32];
  if (threadIdx.x < 32) R[threadIdx.x] = T(1) / D[threadIdx.x][threadIdx.x];
  __syncthreads();
  // panel: rows below solve x L_kk^T = a
  for (int row = k0 + 32 + threadIdx.x; row < dp; row += blockDim.x) {
    T a[32];
    T* pr = L + (int64_t)row * dp + k0;
#pragma unroll
    for (int c = 0; c < 32; ++c) a[c] = pr[c];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      a[c] *= R[c];
#pragma unroll
      for (int q = c + 1; q < 32; ++q) a[q] -= a[c] * D[q][c];
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) pr[c] = a[c];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_update(T* __restrict__ L, int dp, int k, int Tt) {
  __shared__ T Pi[32][33];
  __shared__ T Pj[32][33];
  // lower tile (i, j), k < j <= i < Tt
  const int q = blockIdx.x;
  int ii = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
  while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
  while (ii * (ii + 1) / 2 > q) --ii;
  const int jj = q - ii * (ii + 1) / 2;
  const int i = k + 1 + ii, j = k + 1 + jj;
  const int k0 = k * 32;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int r = e >> 5, c = e & 31;
    Pi[r][c] = L[(int64_t)(i * 32 + r) * dp + k0 + c];
    Pj[r][c] = L[(int64_t)(j * 32 + r) * dp + k0 + c];
  }
  __syncthreads();
  const int a = threadIdx.x >> 3, b0 = (threadIdx.x & 7) * 4;
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
  for (int c = 0; c < 32; ++c) {
    const T pa = Pi[a][c];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += pa * Pj[b0 + u][c];
  }
  T* out = L + (int64_t)(i * 32 + a) * dp + j * 32 + b0;
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] -= acc[u];
}

template <typename T>
static cudaError_t chol_impl(const double* H, int d, T* L, int* status, cudaStream_t st) {
  const int dp = chol_padded(d), Tt = dp / 32;
  const int blocks = (int)std::min<int64_t>(((int64_t)dp * dp + 255) / 256, 2048);
  { k_chol_init<T><<<blocks, 256, 0, st>>>(H, d, dp, L); note_launches(1); }
  for (int k = 0; k < Tt; ++k) {
    { k_chol_panel<T><<<1, 512, 0, st>>>(L, dp, k, status); note_launches(1); }
    const int u = Tt - k - 1;
    { if (u > 0) k_chol_update<T><<<u * (u + 1) / 2, 256, 0, st>>>(L, dp, k, Tt); note_launches(1); }
  }
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const double* H, int d, int f32, void* Lbuf, int* status,
                            cudaStream_t st) {
  return f32 ? chol_impl<float>(H, d, (float*)Lbuf, status, st)
             : chol_impl<double>(H, d, (double*)Lbuf, status, st);
}

// ----------------------------------------------------------------------------
// Solve L L^T delta = v in one CTA (forward then backward substitution by 32
// tiles: one warp solves the diagonal tile, all threads update the rest).
// mode 0: x += delta, step_norm = max |delta|;  mode 1: out = delta.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_solve(const T* __restrict__ L, int d, int dp,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ x,
                                                     double* __restrict__ step_norm, int mode) {
  extern __shared__ unsigned char sm_raw[];
  T* y = reinterpret_cast<T*>(sm_raw);
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Tt = dp / 32;
  for (int i = tid; i < dp; i += blockDim.x) y[i] = (i < d) ? (T)v[i] : T(0);
  __syncthreads();
  for (int kt = 0; kt < Tt; ++kt) {
    const int k0 = kt * 32;
    if (warp == 0) {
      T yl = y[k0 + lane];
      const T* Lr = L + (int64_t)(k0 + lane) * dp + k0;
      for (int j = 0; j < 32; ++j) {
        if (lane == j) yl = yl / Lr[j];
        const T yj = __shfl_sync(0xffffffffu, yl, j);
        if (lane > j) yl -= Lr[j] * yj;
      }
      y[k0 + lane] = yl;
    }
    __syncthreads();
    for (int r = k0 + 32 + tid; r < dp; r += blockDim.x) {
      const T* Lr = L + (int64_t)r * dp + k0;
      T s = T(0);
#pragma unroll 8
      for (int c = 0; c < 32; ++c) s += Lr[c] * y[k0 + c];
      y[r] -= s;
    }
    __syncthreads();
  }
  for (int kt = Tt - 1; kt >= 0; --kt) {
    const int k0 = kt * 32;
    if (warp == 0) {
      T yl = y[k0 + lane];
      for (int j = 31; j >= 0; --j) {
        if (lane == j) yl = yl / L[(int64_t)(k0 + j) * dp + k0 + j];
        const T zj = __shfl_sync(0xffffffffu, yl, j);
        if (lane < j) yl -= L[(int64_t)(k0 + j) * dp + k0 + lane] * zj;
      }
      y[k0 + lane] = yl;
    }
    __syncthreads();
    for (int r = tid; r < k0; r += blockDim.x) {
      T s = T(0);
#pragma unroll 8
      for (int c = 0; c < 32; ++c) s += L[(int64_t)(k0 + c) * dp + r] * y[k0 + c];
      y[r] -= s;
    }
    __syncthreads();
  }
  double mx = 0.0;
  for (int i = tid; i < d; i += blockDim.x) {
    const double dl = (double)y[i];
    if (mode == 0) {
      x[i] += dl;
      mx = fmax(mx, fabs(dl));
    } else {
      x[i] = dl;
    }
  }
  if (mode == 0) {
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m2 = fmax(m2, red[w]);
      if (step_norm) *step_norm = m2;
    }
  }
}

template <typename T>
static cudaError_t solve_impl(const T* L, int d, const double* v, double* x, double* step_norm,
                              int mode, cudaStream_t st) {
  const int dp = chol_padded(d);
  { k_chol_solve<T><<<1, 1024, (size_t)dp * sizeof(T), st>>>(L, d, dp, v, x, step_norm, mode); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_chol_step(const void* Lbuf, int d, int f32, const double* g, double* x,
                             double* step_norm, cudaStream_t st) {
  return f32 ? solve_impl<float>((const float*)Lbuf, d, g, x, step_norm, 0, st)
             : solve_impl<double>((const double*)Lbuf, d, g, x, step_norm, 0, st);
}

cudaError_t launch_chol_apply(const void* Lbuf, int d, int f32, const double* v, double* out,
                              cudaStream_t st) {
  return f32 ? solve_impl<float>((const float*)Lbuf, d, v, out, nullptr, 1, st)
             : solve_impl<double>((const double*)Lbuf, d, v, out, nullptr, 1, st);
}
