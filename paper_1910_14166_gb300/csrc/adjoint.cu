// adjoint.cu -- reverse-mode derivative of a loss L(x) of the ridge / OLS
// solution x = (A^T A + lambda I)^{-1} A^T b (not in the paper).
//
//   v = (A^T A + lambda I)^{-1} dL/dx   conjugate gradients, preconditioned
//                                        by the Cholesky factor of the last
//                                        sketched Hessian (H + lambda I)
//   dL/db = A v
//   dL/dA = r v^T - (A v) x^T,  r = b - A x
//
// The CG operator is one fused pass over A (the gradient kernel with b = 0:
// A^T(0 - A p) - lambda p = -(A^T A + lambda I) p).  The d-vector updates
// are single-CTA kernels with FP64 scalars kept on the device; the host
// reads only the residual norm to stop.  dL/dA is one more streaming pass:
// per row, both dot products A_i x and A_i v (FP64-class), then the output
// row r_i v^T - (A v)_i x^T.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kCgThreads = 1024;

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// scal[0] = r.z (current), scal[1] = r.r, scal[2] = |rhs|^2
__global__ void __launch_bounds__(kCgThreads) k_cg_init(const double* __restrict__ rhs, int d,
                                                        double* __restrict__ v,
                                                        double* __restrict__ r,
                                                        double* __restrict__ scal) {
  __shared__ double red[33];
  double a = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double q = rhs[j];
    v[j] = 0.0;
    r[j] = q;
    a += q * q;
  }
  a = block_sum_d(a, red);
  if (threadIdx.x == 0) {
    scal[1] = a;
    scal[2] = a;
  }
}

// p = z + beta p with beta = (r.z) / (r.z)_old  (first: p = z)
__global__ void __launch_bounds__(kCgThreads) k_cg_dir(const double* __restrict__ r,
                                                       const double* __restrict__ z, int d,
                                                       double* __restrict__ p,
                                                       double* __restrict__ scal, int first) {
  __shared__ double red[33];
  double a = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) a += r[j] * z[j];
  const double rz = block_sum_d(a, red);
  const double beta = first ? 0.0 : rz / scal[0];
  for (int j = threadIdx.x; j < d; j += blockDim.x) p[j] = z[j] + (first ? 0.0 : beta * p[j]);
  __syncthreads();
  if (threadIdx.x == 0) scal[0] = rz;
}

// q = -(negq) = (A^T A + lambda I) p;  alpha = rz / p.q;  v += alpha p;  r -= alpha q
__global__ void __launch_bounds__(kCgThreads) k_cg_step(const double* __restrict__ p,
                                                        const double* __restrict__ negq, int d,
                                                        double* __restrict__ v,
                                                        double* __restrict__ r,
                                                        double* __restrict__ scal) {
  __shared__ double red[33];
  double a = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) a -= p[j] * negq[j];
  const double pq = block_sum_d(a, red);
  const double alpha = scal[0] / pq;
  double rr = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    v[j] += alpha * p[j];
    const double rn = r[j] + alpha * negq[j];
    r[j] = rn;
    rr += rn * rn;
  }
  rr = block_sum_d(rr, red);
  if (threadIdx.x == 0) scal[1] = rr;
}

__global__ void k_negate(double* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = -a[i];
}

// dL/dA row i = r_i v^T - (A v)_i x^T; one warp per row, lanes over columns.
template <typename Tin>
__global__ void __launch_bounds__(256) k_adjoint_dA(const Tin* __restrict__ A, int64_t lda,
                                                    int64_t n, int d,
                                                    const double* __restrict__ b,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ v,
                                                    Tin* __restrict__ out) {
  extern __shared__ double xv_sm[];  // x[d], v[d] (double), then their float-pair splits
  double* xs = xv_sm;
  double* vs = xv_sm + d;
  float* fsp = reinterpret_cast<float*>(xv_sm + 2 * d);  // xh, xl, vh, vl: 4 d floats
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    xs[c] = x[c];
    vs[c] = v[c];
    split_double(x[c], fsp[c], fsp[d + c]);
    split_double(v[c], fsp[2 * d + c], fsp[3 * d + c]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    const Tin* row = A + i * lda;
    if constexpr (sizeof(Tin) == 4) {
      // float-pair dot products with x and v
      float sxh = 0.f, sxl = 0.f, svh = 0.f, svl = 0.f;
      for (int c = lane; c < d; c += 32) {
        const float a = __ldcs(row + c);
        dd_fma_acc(sxh, sxl, a, fsp[c], fsp[d + c]);
        dd_fma_acc(svh, svl, a, fsp[2 * d + c], fsp[3 * d + c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float ah = __shfl_xor_sync(0xffffffffu, sxh, o), al = __shfl_xor_sync(0xffffffffu, sxl, o);
        dd_add(sxh, sxl, ah, al);
        ah = __shfl_xor_sync(0xffffffffu, svh, o);
        al = __shfl_xor_sync(0xffffffffu, svl, o);
        dd_add(svh, svl, ah, al);
      }
      const double ri = b[i] - ((double)sxh + (double)sxl);
      const double avi = (double)svh + (double)svl;
      const float rf = (float)ri, af = (float)avi;
      for (int c = lane; c < d; c += 32)
        out[i * d + c] = rf * fsp[2 * d + c] - af * fsp[c];
    } else {
      double sx = 0.0, sv = 0.0;
      for (int c = lane; c < d; c += 32) {
        const double a = __ldcs(row + c);
        sx = fma(a, xs[c], sx);
        sv = fma(a, vs[c], sv);
      }
      sx = warp_sum(sx);
      sv = warp_sum(sv);
      const double ri = b[i] - sx;
      for (int c = lane; c < d; c += 32) out[i * d + c] = ri * vs[c] - sv * xs[c];
    }
  }
}

}  // namespace

cudaError_t launch_cg_init(const double* rhs, int d, double* v, double* r, double* scal,
                           cudaStream_t st) {
  k_cg_init<<<1, kCgThreads, 0, st>>>(rhs, d, v, r, scal);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cg_dir(const double* r, const double* z, int d, double* p, double* scal,
                          int first, cudaStream_t st) {
  k_cg_dir<<<1, kCgThreads, 0, st>>>(r, z, d, p, scal, first);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cg_step(const double* p, const double* negq, int d, double* v, double* r,
                           double* scal, cudaStream_t st) {
  k_cg_step<<<1, kCgThreads, 0, st>>>(p, negq, d, v, r, scal);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_negate(double* a, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_negate<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(a, n);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_adjoint_dA(const DenseA& A, const double* b, const double* x, const double* v,
                              void* out, cudaStream_t st) {
  if (A.n == 0) return cudaSuccess;
  const size_t smem = (size_t)2 * A.d * sizeof(double) + (size_t)4 * A.d * sizeof(float);
  const unsigned blocks = (unsigned)std::min<int64_t>((A.n + 7) / 8, 152 * 16);
  if (A.f32)
    k_adjoint_dA<float><<<blocks, 256, smem, st>>>((const float*)A.val, A.ld, A.n, (int)A.d, b, x,
                                                   v, (float*)out);
  else
    k_adjoint_dA<double><<<blocks, 256, smem, st>>>((const double*)A.val, A.ld, A.n, (int)A.d, b,
                                                    x, v, (double*)out);
  note_launches(1);
  return cudaGetLastError();
}
