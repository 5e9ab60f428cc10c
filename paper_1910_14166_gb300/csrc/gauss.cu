// gauss.cu -- the Gaussian sketch of Sec. 2, S = G / sqrt(m) with G_ij iid
// N(0, 1), the paper's dense comparison: the raw SA = G A (the 1/m goes to
// the Gram scale).  G is never stored: each kernel generates the tile of G
// it multiplies, in shared memory, from the counter words -- entry (r, i)
// from the word out(key_t2, r n + i) by the Box-Muller transform of its two
// 32-bit halves (the oracle's definition) -- so the sketch reads A and writes
// SA and nothing else touches HBM.  This is the one sketch whose cost is a
// dense O(m n d) product: the point of the comparison.
//
// Mixed form (TF32): a tcgen05 kernel.  Each CTA owns 128 rows of G (an
// M tile), up to 512 columns of A (an N tile: the whole of d <= 512, so each
// entry of G is generated once) and a slice of the n rows (split K):
//   warps 0..7  producers: per K block of 32 rows of A, generate the 128 x 32
//               tile of G (16 entries a thread) and load the 32 x N tile of A
//               (lane = row, warp = column slab), both rounded to TF32 and
//               stored K-major with the 128-byte swizzle into a stage of a
//               shared-memory ring; fence to the async proxy; arrive on the
//               stage's full barrier.  Afterwards the epilogue: tcgen05.ld of
//               the FP32 accumulator from TMEM into an FP32 partial.
//   warp 8      allocates TMEM (the 128 x N FP32 accumulator); one elected
//               thread issues tcgen05.mma (M = 128, N <= 256 per instruction,
//               K = 8) per stage and commits the stage back to the producers.
// Partials are summed over the K splits in split order (FP64 sums, one
// rounding to FP32): deterministic.
// Plain form (FP64): a SIMT kernel of 64 x 64 output tiles, G generated in
// FP64 by the same definition into shared memory, FP64 partials summed over
// the K splits in split order.
// Every mbarrier wait is bounded; a wait that runs out records DEV_TIMEOUT
// and the kernel drains its issued MMAs and frees TMEM before returning.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "tc.cuh"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Entry of G from its counter word, in FP64: u1, u2 in (0, 1) from the two
// 32-bit halves, g = sqrt(-2 ln u1) cos(2 pi u2) (Box & Muller 1958).
IHS_DEV double gauss_from_word_f64(uint64_t w) {
  const double u1 = ((double)(uint32_t)(w >> 32) + 0.5) * (1.0 / 4294967296.0);
  const double u2 = ((double)(uint32_t)(w & 0xFFFFFFFFull) + 0.5) * (1.0 / 4294967296.0);
  return sqrt(-2.0 * log(u1)) * cos(kTwoPi * u2);
}

// The same entry in FP32 with the hardware's fast logarithm, reciprocal
// square root and cosine; u1 and u2 are the FP32 roundings of the same
// values.  The result is within a few FP32 ulps of the FP64 entry (absolute
// error below 1e-5 for |g| < 7), far below the TF32 rounding that follows.
IHS_DEV float gauss_from_word_f32(uint64_t w) {
  const float u1 = __fmaf_rn(__uint2float_rn((uint32_t)(w >> 32)), 0x1p-32f, 0x1p-33f);
  const float u2 = __fmaf_rn(__uint2float_rn((uint32_t)w), 0x1p-32f, 0x1p-33f);
  const float v = -1.3862943611198906f * __log2f(u1);  // -2 ln u1 = -2 ln 2 log2 u1
  const float rad = v > 0.f ? v * rsqrtf(v) : 0.f;
  return rad * __cosf(6.2831853071795865f * u2);
}

// ---------------------------------------------------------------------------
// Mixed form: tcgen05 kernel
// ---------------------------------------------------------------------------
constexpr int kGtProducerWarps = 16;
constexpr int kGtProducers = kGtProducerWarps * 32;
constexpr int kGtTmaWarp = kGtProducerWarps;       // issues the TMA loads of A
constexpr int kGtMmaWarp = kGtProducerWarps + 1;   // owns TMEM, issues the MMAs
constexpr int kGtThreads = kGtProducers + 64;
constexpr int kGtM = 128;                 // rows of G per CTA (M of the MMA)
constexpr int kGtKB = 32;                 // rows of A per K block (128 bytes of TF32)
constexpr int kGtGBytes = kGtM * 128;     // G stage: 128 rows x 128 bytes
constexpr int kGtMaxN = 512;              // TMEM columns of the accumulator

// A^T in TF32 (rounded to nearest, ties away), K-major: row j < dpad of At
// is column j of A, ldt >= n entries, zero beyond d and n.  Built once per
// context; the Gaussian kernel streams it by TMA.
template <typename Tin>
__global__ void k_gauss_operand(const Tin* __restrict__ A, int64_t lda, int64_t n, int d,
                                int dpad, int64_t ldt, uint32_t* __restrict__ At) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = r0 + k;
    const int c = c0 + tx;
    tile[k][tx] = (r < n && c < d) ? (float)A[r * lda + c] : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k;
    const int64_t r = r0 + tx;
    if (c < dpad && r < ldt) At[(int64_t)c * ldt + r] = tf32_rna_bits(tile[tx][k]);
  }
}

__global__ void __launch_bounds__(kGtThreads, 1) k_gauss_tc(
    const __grid_constant__ CUtensorMap amap, int64_t n, uint64_t key, int64_t m, int mtiles,
    int ntiles, int dn, int box_rows, int64_t kb_per_split, int stages, int tmem_cols,
    int64_t ldp, float* __restrict__ partial, int* status) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  const int sbytes = kGtGBytes + dn * 128;  // a multiple of 1024 (dn is a multiple of 64)
  uint64_t* full = (uint64_t*)(base + (size_t)stages * sbytes);
  uint64_t* empty = full + stages;
  uint64_t* done = empty + stages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // M tile varies fastest, so the CTAs resident together read the same rows
  // of A (from L2 after the first)
  const int mt = blockIdx.x % mtiles;
  const int nt = (blockIdx.x / mtiles) % ntiles;
  const int sp = blockIdx.x / (mtiles * ntiles);
  const int64_t kbt = (n + kGtKB - 1) / kGtKB;
  const int64_t kb0 = (int64_t)sp * kb_per_split;
  const int64_t kb1 = min(kbt, kb0 + kb_per_split);
  const int nkb = (int)max((int64_t)0, kb1 - kb0);
  const int c0 = nt * kGtMaxN;  // first column of A in this N tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full + s, kGtProducers + 1);  // the generators + the TMA thread's expect_tx
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGtMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kGtProducerWarps) {
    // ---- generators: G tile entries (R, k0 + 8 kq + q), q < 8 ----
    const int r = threadIdx.x & (kGtM - 1);  // row of the G tile
    const int kq = threadIdx.x >> 7;         // which 8 of the 32 columns of the K block
    const int64_t R = (int64_t)mt * kGtM + r;
    const bool rok = R < m;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % stages;
      const uint32_t ph = (uint32_t)((i / stages) & 1);
      if (!mbar_wait(empty + s, ph ^ 1u, abort_flag)) {
        set_status(status, DEV_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      uint8_t* gs = base + (size_t)s * sbytes;
      const int64_t i0 = (kb0 + i) * kGtKB + kq * 8;
      // eight consecutive counters, carried through each step of the
      // finaliser and the transform side by side (independent chains the
      // scheduler interleaves); every entry is computed (no branch), the ones
      // outside G (rows >= m, columns >= n) are stored as zero
      const int lim = rok ? (int)min((int64_t)8, max((int64_t)0, n - i0)) : 0;
      const uint64_t z0 = key + (uint64_t)(R * n + i0 + 1) * kSmGamma;
      uint64_t z[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = z0 + (uint64_t)q * kSmGamma;
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = sm64_finalise(z[q]);
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float g = gauss_from_word_f32(z[q]);
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(g));
        v[q] = q < lim ? t : 0u;
      }
      *reinterpret_cast<uint4*>(gs + sw128_offset(r, kq * 8)) = make_uint4(v[0], v[1], v[2], v[3]);
      *reinterpret_cast<uint4*>(gs + sw128_offset(r, kq * 8 + 4)) =
          make_uint4(v[4], v[5], v[6], v[7]);
      fence_proxy_async_smem();
      mbar_arrive(full + s);
    }
  } else if (warp == kGtTmaWarp && lane == 0) {
    // ---- TMA: the dn x 32 tile of A^T (box_rows rows per copy) ----
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % stages;
      const uint32_t ph = (uint32_t)((i / stages) & 1);
      if (!mbar_wait(empty + s, ph ^ 1u, abort_flag)) {
        set_status(status, DEV_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      uint8_t* bs = base + (size_t)s * sbytes + kGtGBytes;
      mbar_expect_tx(full + s, (uint32_t)dn * 128u);
      const int x = (int)((kb0 + i) * kGtKB);
      for (int h = 0; h * box_rows < dn; ++h)
        tma_load_2d(bs + h * box_rows * 128, &amap, x, c0 + h * box_rows, full + s);
      ++issued;
    }
    // every issued copy must land before the CTA exits: wait (bounded) for
    // the stages the MMA side may not have consumed
    for (int i = max(0, issued - stages); i < issued; ++i) {
      const int s = i % stages;
      const uint32_t ph = (uint32_t)((i / stages) & 1);
      for (long long it = 0; it < kSpinLimit && !mbar_try_wait(full + s, ph); ++it)
        if (it > 32) __nanosleep(64);
    }
  } else if (warp == kGtMmaWarp && lane == 0) {
    // ---- MMA issuer ----
    const int halves = dn > 256 ? 2 : 1;
    const int nmma = dn / halves;  // N of one instruction: a multiple of 32, <= 256
    const uint32_t idesc = make_idesc(2u, kGtM, nmma);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % stages;
      const uint32_t ph = (uint32_t)((i / stages) & 1);
      if (!mbar_wait(full + s, ph, abort_flag)) {
        set_status(status, DEV_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      uint8_t* gs = base + (size_t)s * sbytes;
      const uint64_t ad = smem_desc_sw128(smem_u32(gs));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // four 32-byte K steps per 128-byte row
        for (int h = 0; h < halves; ++h) {
          const uint64_t bd = smem_desc_sw128(smem_u32(gs + kGtGBytes + h * nmma * 128));
          tc_mma<0>(tmem + (uint32_t)(h * nmma), ad + 2 * kk, bd + 2 * kk, idesc,
                    (i > 0 || kk > 0) ? 1u : 0u);
        }
      tc_commit(empty + s);
    }
    tc_commit(done);  // arrives once every issued MMA has completed
  }
  if (warp < kGtProducerWarps) {
    // ---- epilogue: the lane quarter this warp may read, 32-column chunks ----
    bool ok = false;
    for (long long it = 0; it < kSpinLimit; ++it) {
      if (mbar_try_wait(done, 0)) {
        ok = true;
        break;
      }
      if (it > 32) __nanosleep(128);
    }
    tc_fence_after();
    // warp-uniform decisions: tcgen05.ld is a whole-warp instruction
    ok = __all_sync(0xffffffffu, ok);
    const bool skip = __any_sync(0xffffffffu, nkb == 0 || *abort_flag != 0);
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    float* out = partial + ((int64_t)sp * mtiles * kGtM + (int64_t)mt * kGtM + row) * ldp + c0;
    if (!ok) set_status(status, DEV_TIMEOUT);
#pragma unroll 1
    for (int c = (warp >> 2) * 32; c < dn; c += (kGtProducerWarps / 4) * 32) {
      if (!ok) break;
      if (skip) {
        for (int u = 0; u < 32; ++u) out[c + u] = 0.f;
        continue;
      }
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int u = 0; u < 32; u += 4)
        *reinterpret_cast<float4*>(out + c + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kGtMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// SA[R, c] (FP32) = sum over the splits, in split order, of partial[sp][R][c].
__global__ void k_gauss_reduce_f32(const float* __restrict__ partial, int splits, int64_t mrows,
                                   int64_t ldp, int64_t m, int d, float* __restrict__ SA) {
  const int64_t total = m * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t R = e / d;
    const int c = (int)(e - R * d);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += (double)partial[((int64_t)sp * mrows + R) * ldp + c];
    SA[e] = (float)s;
  }
}

// ---------------------------------------------------------------------------
// Plain form: FP64 SIMT kernel
// ---------------------------------------------------------------------------
template <typename Tin>
__global__ void __launch_bounds__(256) k_gauss_f64(const Tin* __restrict__ A, int64_t lda,
                                                   int64_t n, int d, uint64_t key, int64_t m,
                                                   int mtiles, int ntiles, int64_t kchunk,
                                                   double* __restrict__ partial) {
  __shared__ double Gs[16][64 + 1];  // [k][row of G]
  __shared__ double As[16][64 + 1];  // [k][column of A]
  const int mt = blockIdx.x % mtiles, nt = blockIdx.x / mtiles;
  const int sp = blockIdx.y;
  const int64_t k0 = (int64_t)sp * kchunk, k1 = min(n, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t kb = k0; kb < k1; kb += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e >> 6, c = e & 63;
      const int64_t i = kb + kk;
      const int64_t R = (int64_t)mt * 64 + c;
      const int col = nt * 64 + c;
      Gs[kk][c] = (i < k1 && R < m) ? gauss_from_word_f64(sm64_out(key, (uint64_t)(R * n + i)))
                                    : 0.0;
      As[kk][c] = (i < k1 && col < d) ? (double)A[i * lda + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = Gs[kk][ty * 4 + u];
        b[u] = As[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t R = (int64_t)mt * 64 + ty * 4 + u;
    if (R >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int col = nt * 64 + tx * 4 + v;
      if (col < d) partial[((int64_t)sp * m + R) * d + col] = acc[u][v];
    }
  }
}

__global__ void k_gauss_reduce_f64(const double* __restrict__ partial, int splits, int64_t m,
                                   int d, double* __restrict__ SA) {
  const int64_t total = m * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += partial[(int64_t)sp * total + e];
    SA[e] = s;
  }
}

}  // namespace

GaussPlan make_gauss_plan(int64_t m, int64_t n, int d, int acc64, int sms) {
  GaussPlan p;
  p.acc64 = acc64;
  p.m = m;
  p.n = n;
  p.d = d;
  sms = std::max(1, sms);
  if (acc64) {
    p.mtiles = (int)((m + 63) / 64);
    p.ntiles = (d + 63) / 64;
    const int64_t kblocks = std::max<int64_t>(1, (n + 15) / 16);
    const int64_t tiles = (int64_t)p.mtiles * p.ntiles;
    p.splits = (int)std::max<int64_t>(1, std::min<int64_t>(kblocks, (2 * sms) / tiles));
    p.kchunk = ((n + p.splits - 1) / p.splits + 15) / 16 * 16;
    p.splits = (int)std::max<int64_t>(1, (n + p.kchunk - 1) / p.kchunk);
    p.partial_bytes = (size_t)p.splits * m * d * sizeof(double);
    return p;
  }
  p.dpad = (d + 63) / 64 * 64;
  p.ntiles = (p.dpad + kGtMaxN - 1) / kGtMaxN;
  p.dn = std::min(p.dpad, kGtMaxN);
  p.box_rows = p.dn <= 256 ? p.dn : p.dn / 2;
  p.ldp = (int64_t)p.ntiles * p.dn;
  p.ldt = (n + kGtKB - 1) / kGtKB * kGtKB;
  p.at_bytes = (size_t)p.dpad * p.ldt * sizeof(uint32_t);
  p.mtiles = (int)((m + kGtM - 1) / kGtM);
  int tc = 32;
  while (tc < p.dn) tc *= 2;
  p.tmem_cols = tc;
  const int sbytes = kGtGBytes + p.dn * 128;
  p.stages = std::max(2, std::min(4, (200 * 1024) / sbytes));
  p.smem = 1024 + p.stages * sbytes + 256;
  // split K so that the grid fills whole waves of one CTA per SM, with at
  // least 8 K blocks a CTA
  const int64_t kbt = std::max<int64_t>(1, (n + kGtKB - 1) / kGtKB);
  const int64_t tiles = (int64_t)p.mtiles * p.ntiles;
  const int64_t smax = std::max<int64_t>(1, kbt / 8);
  int64_t best = 1;
  for (int64_t s = 1; s <= smax; ++s) {
    const int64_t ctas = tiles * s;
    const int64_t waves = (ctas + sms - 1) / sms;
    best = s;
    if ((double)ctas / (double)(waves * sms) >= 0.95 || ctas >= 8 * sms) break;
  }
  p.kb_per_split = (kbt + best - 1) / best;
  p.splits = (int)((kbt + p.kb_per_split - 1) / p.kb_per_split);
  p.partial_bytes = (size_t)p.splits * p.mtiles * kGtM * p.ldp * sizeof(float);
  return p;
}

cudaError_t launch_gauss_operand(const GaussPlan& p, const DenseA& A, void* At, cudaStream_t st) {
  if (p.acc64) return cudaSuccess;
  dim3 grid((unsigned)(p.ldt / 32), (unsigned)(p.dpad / 32));
  if (A.f32)
    k_gauss_operand<float><<<grid, 256, 0, st>>>((const float*)A.val, A.ld, A.n, (int)A.d, p.dpad,
                                                 p.ldt, (uint32_t*)At);
  else
    k_gauss_operand<double><<<grid, 256, 0, st>>>((const double*)A.val, A.ld, A.n, (int)A.d,
                                                  p.dpad, p.ldt, (uint32_t*)At);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gauss(const GaussPlan& p, const DenseA& A, const void* At, uint64_t key,
                         void* partial, void* SA, int* status, cudaStream_t st) {
  cudaError_t e;
  const int64_t total = p.m * p.d;
  const unsigned red_blocks =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8192));
  if (p.acc64) {
    dim3 grid((unsigned)(p.mtiles * p.ntiles), (unsigned)p.splits);
    if (A.f32)
      k_gauss_f64<float><<<grid, 256, 0, st>>>((const float*)A.val, A.ld, A.n, (int)A.d, key, p.m,
                                               p.mtiles, p.ntiles, p.kchunk, (double*)partial);
    else
      k_gauss_f64<double><<<grid, 256, 0, st>>>((const double*)A.val, A.ld, A.n, (int)A.d, key,
                                                p.m, p.mtiles, p.ntiles, p.kchunk,
                                                (double*)partial);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gauss_reduce_f64<<<red_blocks, 256, 0, st>>>((const double*)partial, p.splits, p.m, p.d,
                                                   (double*)SA);
    note_launches(1);
    return cudaGetLastError();
  }
  PFN_encodeTiled enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)p.ldt, (cuuint64_t)p.dpad};
  cuuint64_t gstride[1] = {(cuuint64_t)(p.ldt * 4)};
  cuuint32_t box[2] = {(cuuint32_t)kGtKB, (cuuint32_t)p.box_rows};
  cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(At), gdim, gstride, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if ((e = ensure_smem((const void*)k_gauss_tc, p.smem)) != cudaSuccess) return e;
  const unsigned grid = (unsigned)((int64_t)p.mtiles * p.ntiles * p.splits);
  k_gauss_tc<<<grid, kGtThreads, p.smem, st>>>(map, p.n, key, p.m, p.mtiles, p.ntiles, p.dn,
                                               p.box_rows, p.kb_per_split, p.stages, p.tmem_cols,
                                               p.ldp, (float*)partial, status);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gauss_reduce_f32<<<red_blocks, 256, 0, st>>>((const float*)partial, p.splits,
                                                 (int64_t)p.mtiles * kGtM, p.ldp, p.m, p.d,
                                                 (float*)SA);
  note_launches(1);
  return cudaGetLastError();
}
