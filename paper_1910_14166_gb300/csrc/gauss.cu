// gauss.cu -- the Gaussian sketch of Sec. 2, S = G / sqrt(m) with G_ij iid
// N(0, 1), the paper's dense comparison: the raw SA = G A (the 1/m goes to
// the Gram scale).  G is never stored whole: it is generated in column
// chunks of nc (entry (r, i) from the counter word out(key_t2, r n + i) by
// the Box-Muller transform of its two 32-bit halves, the oracle's
// definition) and each chunk is multiplied into SA with a plain library
// GEMM (cuBLAS): TF32 tensor cores with FP32 accumulation in the mixed form,
// FP64 in the plain form.  This is the one sketch whose cost is a dense
// O(m n d) product -- the point of the comparison.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace {

// G[r, c] for columns i0 .. i0 + nc of the m x n matrix, stored row-major
// with leading dimension nc.
template <typename T>
__global__ void k_gauss_fill(uint64_t key, int64_t m, int64_t n, int64_t i0, int64_t nc,
                             T* __restrict__ G) {
  const int64_t total = m * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / nc, c = e - r * nc;
    const int64_t i = i0 + c;
    T g = T(0);
    if (i < n) {
      const uint64_t w = sm64_out(key, (uint64_t)(r * n + i));
      const T u1 = ((T)(uint32_t)(w >> 32) + T(0.5)) * (T)(1.0 / 4294967296.0);
      const T u2 = ((T)(uint32_t)(w & 0xFFFFFFFFull) + T(0.5)) * (T)(1.0 / 4294967296.0);
      g = sqrt(T(-2) * log(u1)) * cos((T)6.283185307179586476925286766559 * u2);
    }
    G[e] = g;
  }
}

// rows i0 .. i0 + nc of A (Tin, leading dimension lda) into B (T, nc x d,
// leading dimension d), zero beyond n
template <typename T, typename Tin>
__global__ void k_rows_convert(const Tin* __restrict__ A, int64_t lda, int64_t n, int d, int64_t i0,
                               int64_t nc, T* __restrict__ B) {
  const int64_t total = nc * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d;
    const int j = (int)(e - r * d);
    const int64_t i = i0 + r;
    B[e] = i < n ? (T)A[i * lda + j] : T(0);
  }
}

}  // namespace

int64_t gauss_chunk(int64_t m, int64_t n) {
  // about 64 Mi entries of G per chunk, a multiple of 256 columns
  int64_t nc = std::max<int64_t>(256, ((int64_t)1 << 26) / std::max<int64_t>(m, 1));
  nc = nc / 256 * 256;
  return std::min<int64_t>(nc, (n + 255) / 256 * 256);
}

cudaError_t launch_gauss(void* cublas, const DenseA& A, const SketchKeys& K, int64_t m, int acc64,
                         void* Gbuf, void* Abuf, void* SA, cudaStream_t st) {
  cublasHandle_t h = (cublasHandle_t)cublas;
  if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const int64_t n = A.n, nc = gauss_chunk(m, n);
  const int d = (int)A.d;
  const unsigned fill_blocks = (unsigned)std::min<int64_t>((m * nc + 255) / 256, 8192);
  const unsigned conv_blocks = (unsigned)std::min<int64_t>((nc * d + 255) / 256, 8192);
  // the chunk of A goes to the GEMM in place when its type matches and the
  // whole chunk lies inside A; otherwise (type change, or the ragged last
  // chunk) it is copied, zero-padded
  const bool same = acc64 ? !A.f32 : A.f32;
  for (int64_t i0 = 0; i0 < n; i0 += nc) {
    const bool direct = same && i0 + nc <= n;
    if (acc64) {
      k_gauss_fill<double><<<fill_blocks, 256, 0, st>>>(K.key[2], m, n, i0, nc, (double*)Gbuf);
      note_launches(1);
      const double* Ap;
      int64_t lda;
      if (direct) {
        Ap = (const double*)A.val + i0 * A.ld;
        lda = A.ld;
      } else {
        if (A.f32)
          k_rows_convert<double, float><<<conv_blocks, 256, 0, st>>>((const float*)A.val, A.ld, n,
                                                                     d, i0, nc, (double*)Abuf);
        else
          k_rows_convert<double, double><<<conv_blocks, 256, 0, st>>>((const double*)A.val, A.ld,
                                                                      n, d, i0, nc, (double*)Abuf);
        note_launches(1);
        Ap = (const double*)Abuf;
        lda = d;
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      // column-major view: SA^T (d x m) += A_chunk^T (d x nc) G_chunk^T (nc x m)
      const double one = 1.0, beta = i0 == 0 ? 0.0 : 1.0;
      if (cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, d, (int)m, (int)nc, &one, Ap, (int)lda,
                      (const double*)Gbuf, (int)nc, &beta, (double*)SA, d) !=
          CUBLAS_STATUS_SUCCESS)
        return cudaErrorUnknown;
    } else {
      k_gauss_fill<float><<<fill_blocks, 256, 0, st>>>(K.key[2], m, n, i0, nc, (float*)Gbuf);
      note_launches(1);
      const float* Ap;
      int64_t lda;
      if (direct) {
        Ap = (const float*)A.val + i0 * A.ld;
        lda = A.ld;
      } else {
        if (A.f32)
          k_rows_convert<float, float><<<conv_blocks, 256, 0, st>>>((const float*)A.val, A.ld, n,
                                                                    d, i0, nc, (float*)Abuf);
        else
          k_rows_convert<float, double><<<conv_blocks, 256, 0, st>>>((const double*)A.val, A.ld,
                                                                     n, d, i0, nc, (float*)Abuf);
        note_launches(1);
        Ap = (const float*)Abuf;
        lda = d;
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      const float one = 1.f, beta = i0 == 0 ? 0.f : 1.f;
      if (cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, d, (int)m, (int)nc, &one, Ap, CUDA_R_32F,
                       (int)lda, Gbuf, CUDA_R_32F, (int)nc, &beta, SA, CUDA_R_32F, d,
                       CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
        return cudaErrorUnknown;
    }
  }
  return cudaGetLastError();
}

void* gauss_blas_create() {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
  return (void*)h;
}

void gauss_blas_destroy(void* h) {
  if (h) cublasDestroy((cublasHandle_t)h);
}
