// srht.cu -- the subsampled randomized Hadamard transform of Sec. 2,
// S = m^{-1/2} P H D, as the comparison sketch of the paper's experiments:
//   D  the sign of block 0's word of row i (the same word a CountSketch with
//      the same (seed, t) would use),
//   H  the Sylvester (recursively defined) Hadamard transform of order
//      n2 = the least power of two >= n, A padded with zero rows,
//   P  m rows sampled uniformly with replacement (block 1's words).
// The raw P H D A goes to SA; the 1/m goes to the Gram scale.
//
// The transform runs stage by stage exactly as its recursive definition
// (stage h maps the pair (u, v) at rows (i, i + h), bit h of i clear, to
// (u + v, u - v), for h = 1, 2, 4, ...), so every output is rounded in the
// same order as the plain stage loop: in FP64 the result is the oracle's
// bit for bit.  Passes of up to 10 (FP32) / 9 (FP64) stages over blocks of 2^kp rows
// (at stride 2^s0) x kCols columns: the low five stages of a block in
// registers (32 values per thread), a transpose through shared memory, the
// remaining stages in registers again.  Each pass reads and writes the n2 x
// d_pad buffer T once (the first reads A and applies D); the sampled rows
// are then gathered into SA.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kCols = 32;       // columns per block

// threads per block: 512 (FP32), 256 (FP64: 32 doubles per thread in registers)
template <typename T>
__host__ __device__ constexpr int fw_threads() { return sizeof(T) == 4 ? 512 : 256; }

template <typename T>
__host__ __device__ constexpr int pass_stages() { return sizeof(T) == 4 ? 10 : 9; }

// In-register butterflies over the low `r` bits of the index of v[0..2^r).
template <typename T, int R>
IHS_DEV void fwht_regs(T (&v)[32]) {
#pragma unroll
  for (int h = 1; h < (1 << R); h <<= 1)
#pragma unroll
    for (int i = 0; i < (1 << R); ++i)
      if (!(i & h)) {
        const T a = v[i], b = v[i + h];
        v[i] = a + b;
        v[i + h] = a - b;
      }
}

template <typename T, int R>
IHS_DEV void fwht_regs_dyn(T (&v)[32], int r) {
  // r <= R; stages h = 1 .. 2^(r-1)
#pragma unroll
  for (int hb = 0; hb < R; ++hb) {
    if (hb >= r) break;
    const int h = 1 << hb;
#pragma unroll
    for (int i = 0; i < (1 << R); ++i)
      if (!(i & h) && i + h < (1 << r)) {
        const T a = v[i], b = v[i + h];
        v[i] = a + b;
        v[i + h] = a - b;
      }
  }
}

// One pass: stages s0 .. s0 + kp - 1 (kp <= pass_stages<T>()).
// first: read A (Tin, n rows, lda) with the signs of D and zero padding;
// else read T.  Always writes T (n2 x ldt).
template <typename T, typename Tin>
__global__ void __launch_bounds__(fw_threads<T>()) k_fwht_pass(const Tin* __restrict__ A, int64_t n,
                                                        int64_t lda, int d, uint64_t key_sign,
                                                        T* __restrict__ Tbuf, int64_t ldt,
                                                        int s0, int kp, int first) {
  extern __shared__ __align__(16) unsigned char fw_smem[];
  T (*S)[kCols + 1] = reinterpret_cast<T (*)[kCols + 1]>(fw_smem);
  const int c = 1 << kp;
  const int64_t st = (int64_t)1 << s0;
  // block -> (low, high, column slab)
  const int64_t rb = blockIdx.x;
  const int64_t low = rb % st, high = rb / st;
  const int64_t row0 = high * st * c + low;
  const int col0 = blockIdx.y * kCols;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  const int col = col0 + lane;
  const int r1 = kp < 5 ? kp : 5;
  const int g1 = 1 << r1;           // rows per thread in phase A
  const int ngroups = c / g1;       // row groups
  // phase A: rows j = g * g1 + i, i < g1, stages on the low r1 bits of j
  for (int g = wq; g < ngroups; g += fw_threads<T>() / 32) {
    T v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      v[i] = T(0);
      if (i < g1) {
        const int64_t R = row0 + (int64_t)(g * g1 + i) * st;
        if (first) {
          if (R < n && col < d) {
            const T a = (T)A[R * lda + col];
            const uint64_t w = sm64_out(key_sign, (uint64_t)R);
            v[i] = (w & 1ULL) ? -a : a;
          }
        } else if (col < d) {
          v[i] = Tbuf[R * ldt + col];
        }
      }
    }
    if (r1 == 5) fwht_regs<T, 5>(v);
    else fwht_regs_dyn<T, 5>(v, r1);
    if (kp == r1) {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < g1 && col < d) Tbuf[(row0 + (int64_t)(g * g1 + i) * st) * ldt + col] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) S[g * g1 + i][lane] = v[i];
    }
  }
  if (kp == r1) return;
  __syncthreads();
  // phase B: rows j = lo + i2 * 32, stages on bits 5 .. kp-1 of j
  const int r2 = kp - 5;
  const int g2 = 1 << r2;
  for (int lo = wq; lo < 32; lo += fw_threads<T>() / 32) {
    T v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = (i < g2) ? S[lo + i * 32][lane] : T(0);
    if (r2 == 5) fwht_regs<T, 5>(v);
    else fwht_regs_dyn<T, 5>(v, r2);
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < g2 && col < d) Tbuf[(row0 + (int64_t)(lo + i * 32) * st) * ldt + col] = v[i];
  }
}

// rows[r] = floor(hi32(out(key_rows, r)) * n2 / 2^32)
__global__ void k_srht_rows(uint64_t key_rows, int64_t m, uint64_t n2, int32_t* __restrict__ rows) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = sm64_out(key_rows, (uint64_t)r);
    rows[r] = (int32_t)(((w >> 32) * n2) >> 32);
  }
}

// SA[k, :] = T[rows[k], :d]
template <typename T>
__global__ void k_srht_gather(const T* __restrict__ Tbuf, int64_t ldt, const int32_t* __restrict__ rows,
                              int64_t m, int d, T* __restrict__ SA) {
  const int64_t total = m * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / d;
    const int j = (int)(e - k * d);
    SA[e] = Tbuf[(int64_t)rows[k] * ldt + j];
  }
}

template <typename T, typename Tin>
cudaError_t srht_impl(const DenseA& A, const SketchKeys& K, int64_t m, int64_t n2, T* Tbuf,
                      int32_t* rows, T* SA, cudaStream_t st) {
  const int d = (int)A.d;
  const int64_t ldt = srht_ldt(d);
  int L = 0;
  while (((int64_t)1 << L) < n2) ++L;
  const int maxk = pass_stages<T>();
  const dim3 block(fw_threads<T>());
  int s0 = 0;
  bool first = true;
  if (L == 0) {
    // n2 = 1: H = [1]; T = D A
    const size_t smem = (size_t)1 * (kCols + 1) * sizeof(T);
    dim3 grid(1, (unsigned)((d + kCols - 1) / kCols));
    k_fwht_pass<T, Tin><<<grid, block, smem, st>>>((const Tin*)A.val, A.n, A.ld, d, K.key[0], Tbuf,
                                                   ldt, 0, 0, 1);
    note_launches(1);
  }
  while (s0 < L) {
    const int kp = std::min(maxk, L - s0);
    const size_t smem = (size_t)(1 << kp) * (kCols + 1) * sizeof(T);
    {
      cudaError_t e = ensure_smem((const void*)k_fwht_pass<T, Tin>,
                                  (int)((1 << maxk) * (kCols + 1) * sizeof(T)));
      if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(n2 >> kp), (unsigned)((d + kCols - 1) / kCols));
    k_fwht_pass<T, Tin><<<grid, block, smem, st>>>((const Tin*)A.val, A.n, A.ld, d, K.key[0], Tbuf,
                                                   ldt, s0, kp, first ? 1 : 0);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    first = false;
    s0 += kp;
  }
  { k_srht_rows<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, st>>>(
      K.key[1], m, (uint64_t)n2, rows); note_launches(1); }
  { k_srht_gather<T><<<(unsigned)std::min<int64_t>((m * d + 255) / 256, 4096), 256, 0, st>>>(
      Tbuf, ldt, rows, m, d, SA); note_launches(1); }
  return cudaGetLastError();
}

}  // namespace

int64_t srht_n2(int64_t n) {
  int64_t n2 = 1;
  while (n2 < n) n2 <<= 1;
  return n2;
}

int64_t srht_ldt(int d) { return (int64_t)((d + kCols - 1) / kCols) * kCols; }

cudaError_t launch_srht(const DenseA& A, const SketchKeys& K, int64_t m, int acc64, void* Tbuf,
                        int32_t* rows, void* SA, cudaStream_t st) {
  const int64_t n2 = srht_n2(A.n);
  if (acc64)
    return A.f32 ? srht_impl<double, float>(A, K, m, n2, (double*)Tbuf, rows, (double*)SA, st)
                 : srht_impl<double, double>(A, K, m, n2, (double*)Tbuf, rows, (double*)SA, st);
  return A.f32 ? srht_impl<float, float>(A, K, m, n2, (float*)Tbuf, rows, (float*)SA, st)
               : srht_impl<float, double>(A, K, m, n2, (float*)Tbuf, rows, (float*)SA, st);
}
