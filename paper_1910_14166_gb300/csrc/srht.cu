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
// bit for bit.  Passes of five stages: one warp per group of 32 rows (at
// stride 2^s0) and 32 columns, each lane one column in registers; the first
// pass reads A and applies D and the zero padding, the others read and write
// the n2 x d_pad buffer T, and the last transforms only the groups holding a
// sampled row and writes those rows straight into SA.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kCols = 32;  // columns per warp slab (T rows padded to a multiple)

// Register-only pass: stages s0 .. s0 + KP - 1 (KP <= 5).  One warp per
// (group of 2^KP rows at stride 2^s0, slab of 32 columns): each lane holds
// one column of the group in registers, so the pass needs no shared memory
// and no block barrier and a warp keeps 2^KP row loads in flight; many
// warps per SM overlap their loads and stores.  The stages run in the same
// order as the recursive definition (h = 2^s0, 2^(s0+1), ...), so every
// output is rounded exactly as in the plain stage loop.
template <typename T, typename Tin, bool First, int KP>
__global__ void __launch_bounds__(256) k_fwht_reg(const Tin* __restrict__ A, int64_t n,
                                                  int64_t lda, int d, uint64_t key_sign,
                                                  T* __restrict__ Tbuf, int64_t ldt, int64_t n2,
                                                  int s0) {
  constexpr int C = 1 << KP;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int slabs = (d + 31) / 32;
  const int64_t st = (int64_t)1 << s0;
  const int64_t groups = n2 >> KP;
  for (int64_t u = warp; u < groups * slabs; u += nwarps) {
    const int64_t grp = u / slabs;
    const int col = (int)(u - grp * slabs) * 32 + lane;
    const int64_t row0 = (grp >> s0) * st * C + (grp & (st - 1));
    const bool cin = col < d;
    T v[C];
    if constexpr (First) {
      // lane i draws the sign of the group's row i; the warp shares them
      const int64_t Rl = row0 + (int64_t)lane * st;
      const bool neg = lane < C && (sm64_out(key_sign, (uint64_t)Rl) & 1ULL);
      const unsigned sgn = __ballot_sync(0xffffffffu, neg);
      const Tin* q = A + row0 * lda + col;
      const int64_t step = st * lda;
#pragma unroll
      for (int i = 0; i < C; ++i) {
        const int64_t R = row0 + (int64_t)i * st;
        v[i] = T(0);
        if (R < n && cin) {
          const T a = (T)q[(int64_t)i * step];
          v[i] = ((sgn >> i) & 1u) ? -a : a;
        }
      }
    } else {
      const T* q = Tbuf + row0 * ldt + col;
      const int64_t step = st * ldt;
#pragma unroll
      for (int i = 0; i < C; ++i) v[i] = cin ? q[(int64_t)i * step] : T(0);
    }
#pragma unroll
    for (int h = 1; h < C; h <<= 1)
#pragma unroll
      for (int i = 0; i < C; ++i)
        if (!(i & h)) {
          const T a = v[i], b = v[i + h];
          v[i] = a + b;
          v[i + h] = a - b;
        }
    if (cin) {
      T* q = Tbuf + row0 * ldt + col;
      const int64_t step = st * ldt;
#pragma unroll
      for (int i = 0; i < C; ++i) q[(int64_t)i * step] = v[i];
    }
  }
}

// Last pass fused with the row sampling: for sample k (row p = rows[k] of
// H D A), the pass's group holding p (rows p mod 2^s0 + i 2^s0, i < 2^KP:
// the last pass spans the top KP bits) is loaded, transformed exactly as
// k_fwht_reg would, and only the entry of p goes to SA row k.  Only the
// groups that hold a sampled row are read (about m of n2 / 2^KP), and T is
// not written back.
template <typename T, int KP>
__global__ void __launch_bounds__(256) k_fwht_last_gather(const T* __restrict__ Tbuf, int64_t ldt,
                                                          int d, int s0,
                                                          const int32_t* __restrict__ rows,
                                                          int64_t m, T* __restrict__ SA) {
  constexpr int C = 1 << KP;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int slabs = (d + 31) / 32;
  const int64_t st = (int64_t)1 << s0;
  for (int64_t u = warp; u < m * slabs; u += nwarps) {
    const int64_t k = u / slabs;
    const int col = (int)(u - k * slabs) * 32 + lane;
    const int64_t p = rows[k];
    const int64_t low = p & (st - 1);
    const int ip = (int)(p >> s0);
    if (col >= d) continue;
    const T* q = Tbuf + low * ldt + col;
    const int64_t step = st * ldt;
    T v[C];
#pragma unroll
    for (int i = 0; i < C; ++i) v[i] = q[(int64_t)i * step];
#pragma unroll
    for (int h = 1; h < C; h <<= 1)
#pragma unroll
      for (int i = 0; i < C; ++i)
        if (!(i & h)) {
          const T a = v[i], b = v[i + h];
          v[i] = a + b;
          v[i + h] = a - b;
        }
    T out = v[0];
#pragma unroll
    for (int i = 1; i < C; ++i)
      if (i == ip) out = v[i];
    SA[k * d + col] = out;
  }
}

template <typename T, typename Tin, bool First>
cudaError_t fwht_reg_pass(const DenseA& A, uint64_t key, T* Tbuf, int64_t ldt, int64_t n2, int s0,
                          int kp, unsigned blocks, cudaStream_t st) {
  const Tin* a = (const Tin*)A.val;
  const int d = (int)A.d;
  switch (kp) {
#define FW(K) \
  case K: k_fwht_reg<T, Tin, First, K><<<blocks, 256, 0, st>>>(a, A.n, A.ld, d, key, Tbuf, ldt, n2, s0); break;
    FW(0) FW(1) FW(2) FW(3) FW(4) FW(5)
#undef FW
    default: return cudaErrorInvalidValue;
  }
  note_launches(1);
  return cudaGetLastError();
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
  // passes of five stages in registers (k_fwht_reg); n2 = 1 is the pass
  // with no stage (T = D A)
  int dev = 0, sms = 0;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int64_t slabs = (d + 31) / 32;
  { k_srht_rows<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, st>>>(
      K.key[1], m, (uint64_t)n2, rows); note_launches(1); }
  // every pass but the last writes T; the last (when there are two or more)
  // transforms only the sampled rows' groups, straight into SA
  const int npass = std::max(1, (L + 4) / 5);
  int s0 = 0;
  for (int pass = 0; pass < npass; ++pass) {
    const int kp = std::min(5, L - s0);
    if (pass == npass - 1 && pass > 0) {
      const unsigned blocks = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>((m * slabs + 7) / 8, (int64_t)sms * 8));
      switch (kp) {
#define FL(KK) \
  case KK: k_fwht_last_gather<T, KK><<<blocks, 256, 0, st>>>(Tbuf, ldt, d, s0, rows, m, SA); break;
        FL(1) FL(2) FL(3) FL(4) FL(5)
#undef FL
        default: return cudaErrorInvalidValue;
      }
      note_launches(1);
      return cudaGetLastError();
    }
    const int64_t units = (n2 >> kp) * slabs;
    const unsigned blocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((units + 7) / 8, (int64_t)sms * 8));
    cudaError_t e = pass == 0
        ? fwht_reg_pass<T, Tin, true>(A, K.key[0], Tbuf, ldt, n2, s0, kp, blocks, st)
        : fwht_reg_pass<T, Tin, false>(A, K.key[0], Tbuf, ldt, n2, s0, kp, blocks, st);
    if (e != cudaSuccess) return e;
    s0 += kp;
  }
  // one pass in all (n2 <= 32): T holds H D A; gather the sampled rows
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
