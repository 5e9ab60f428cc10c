// l2ball.cu -- the step of Eq. 2 over the p = 2 ball C = {x : ||x||_2 <= R}
// (Sec. 1 lists the p-norm balls beside the l1 ball):
//     x^{t+1} = argmin_{||x|| <= R} 1/2 (x - x^t)^T H (x - x^t) - g^T (x - x^t).
// With c = H x^t + g the answer is the Newton point H^{-1} c when it lies in
// the ball; otherwise x(mu) = (H + mu I)^{-1} c with mu > 0 the root of
// ||x(mu)|| = R, found by Newton's method on phi(mu) = 1/||x(mu)|| - 1/R
// (More & Sorensen 1983: phi is concave and increasing, so Newton from
// mu = 0 climbs to the root monotonically), each iterate factoring H + mu I
// with the cooperative Cholesky.  The host drives the iteration (a few
// device-to-host reads of two scalars per Newton step).  Each x(mu) is
// refined with FP64 residuals of (H + mu I) x = c, so the root and the
// point are FP64 accurate even with the mixed form's FP32 factor.  These
// are the kernels; the loop is in capi.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

// r = c - (H + mu I) x, or (with x = x^t, mu = 0, c = g) c = H x^t + g: out_j =
// base_j + sgn * (sum_i H_ji x_i + mu x_j); one warp per row, FP64.
__global__ void k_l2_matvec(const double* __restrict__ H, int d, const double* __restrict__ x,
                            double mu, const double* __restrict__ base, double sgn,
                            double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= d) return;
  const double* row = H + (int64_t)j * d;
  double s = 0.0;
  for (int i = lane; i < d; i += 32) s = fma(row[i], x[i], s);
  s = warp_sum(s);
  if (lane == 0) out[j] = base[j] + sgn * (s + mu * x[j]);
}

// scal[0] = a^T a, scal[1] = a^T b (fixed order, one CTA)
__global__ void __launch_bounds__(1024) k_l2_dots(const double* __restrict__ a,
                                                  const double* __restrict__ b, int d,
                                                  double* __restrict__ scal) {
  __shared__ double r0[32], r1[32];
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    s0 = fma(a[i], a[i], s0);
    s1 = fma(a[i], b[i], s1);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = s0;
    r1[threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t0 += r0[w];
      t1 += r1[w];
    }
    scal[0] = t0;
    scal[1] = t1;
  }
}

// y += a (elementwise)
__global__ void k_l2_axpy(double* __restrict__ y, const double* __restrict__ a, int d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    y[i] += a[i];
}

// x <- src; step_norm = max |src - x_old| (one CTA)
__global__ void __launch_bounds__(1024) k_l2_store(const double* __restrict__ src, int d,
                                                   double* __restrict__ x,
                                                   double* __restrict__ step_norm) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    mx = fmax(mx, fabs(src[i] - x[i]));
    x[i] = src[i];
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    *step_norm = m;
  }
}

}  // namespace

cudaError_t launch_l2_matvec(const double* H, int d, const double* x, double mu, const double* base,
                             double sgn, double* out, cudaStream_t st) {
  k_l2_matvec<<<(d + 7) / 8, 256, 0, st>>>(H, d, x, mu, base, sgn, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l2_dots(const double* a, const double* b, int d, double* scal, cudaStream_t st) {
  k_l2_dots<<<1, 1024, 0, st>>>(a, b, d, scal);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l2_axpy(double* y, const double* a, int d, cudaStream_t st) {
  k_l2_axpy<<<(d + 255) / 256, 256, 0, st>>>(y, a, d);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_l2_store(const double* src, int d, double* x, double* step_norm,
                            cudaStream_t st) {
  k_l2_store<<<1, 1024, 0, st>>>(src, d, x, step_norm);
  note_launches(1);
  return cudaGetLastError();
}
