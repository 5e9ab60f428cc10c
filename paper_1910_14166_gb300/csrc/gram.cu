// gram.cu -- the approximate Hessian H = scale * (SA)^T SA + shift * I
// (Sec. 1: IHS replaces A^T A by the quadratic form of SA; O(m d^2)).
//
// Plain form (FP64): SIMT FP64 tiles of 64 x 64, split over m.
// Mixed form (TF32 / BF16): a tcgen05 kernel.  SA is first transposed into
// a K-major operand Op = SA^T (d_pad x ldt, K = m contiguous) in the MMA input
// type; then each CTA owns one 128 x 128 lower-triangle tile of H and one
// slice of K:
//   warp 0      TMA producer: 128-row x 128-byte boxes, 128B swizzle, into a
//               4-stage shared-memory ring (mbarrier complete_tx)
//   warp 1      allocates 128 TMEM columns, one elected thread issues
//               tcgen05.mma (M=128, N=128, FP32 accumulator in TMEM) and
//               commits each stage back to the producer
//   warps 2..5  epilogue: tcgen05.ld 32x32b.x32 from their TMEM lane
//               quarter -> FP32 partial tile in global memory
// Split-K partials are summed in split order by a reduce kernel that also
// applies scale and shift and mirrors the lower triangle (deterministic).
// Every mbarrier wait is bounded; a wait that runs out records DEV_TIMEOUT,
// drains the copies it issued and frees TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "tc.cuh"

// ----------------------------------------------------------------------------
// Plan
// ----------------------------------------------------------------------------
GramPlan make_gram_plan(int m, int d, int prec, int num_sms) {
  GramPlan g;
  g.d = d;
  g.m = m;
  g.prec = prec;
  g.tdim = (prec == IHS_PREC_FP64) ? 64 : 128;
  const int T = (d + g.tdim - 1) / g.tdim;
  g.tiles = T * (T + 1) / 2;
  const int kunit = (prec == IHS_PREC_FP64) ? 16 : (prec == IHS_PREC_TF32 ? 32 : 64);
  const int64_t kblocks = (m + kunit - 1) / kunit;
  int target = (prec == IHS_PREC_FP64) ? 2 * num_sms : num_sms;
  int splits = std::max(1, target / g.tiles);
  splits = (int)std::min<int64_t>(splits, kblocks);
  g.splits = std::max(1, splits);
  g.ldt = kblocks * kunit;  // K padded to whole k-blocks (zeros)
  return g;
}

size_t gram_partial_bytes(const GramPlan& g) {
  const size_t el = (g.prec == IHS_PREC_FP64) ? sizeof(double) : sizeof(float);
  return (size_t)g.splits * g.tiles * g.tdim * g.tdim * el;
}

size_t gram_operand_bytes(const GramPlan& g) {
  if (g.prec == IHS_PREC_FP64) return 0;
  const int T = (g.d + g.tdim - 1) / g.tdim;
  const size_t el = (g.prec == IHS_PREC_TF32) ? 4 : 2;
  return (size_t)T * g.tdim * g.ldt * el;
}

IHS_DEV void tri_index(int q, int& ti, int& tj) {
  // q enumerates (ti, tj), ti >= tj, row by row: q = ti*(ti+1)/2 + tj
  int t = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= q) ++t;
  while (t * (t + 1) / 2 > q) --t;
  ti = t;
  tj = q - t * (t + 1) / 2;
}

// ----------------------------------------------------------------------------
// FP64 SIMT
// ----------------------------------------------------------------------------
template <typename Tin>
__global__ void __launch_bounds__(256) k_gram_f64(const Tin* __restrict__ SA, int64_t lda, int64_t m,
                                                  int d, int tiles, int64_t kchunk,
                                                  double* __restrict__ partial) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  int ti, tj;
  tri_index(blockIdx.x, ti, tj);
  const int sp = blockIdx.y;
  const int64_t r0 = sp * kchunk, r1 = min((int64_t)m, r0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t rb = r0; rb < r1; rb += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int rr = e >> 6, c = e & 63;
      int64_t r = rb + rr;
      int ca = ti * 64 + c, cb = tj * 64 + c;
      As[rr][c] = (r < r1 && ca < d) ? (double)SA[r * lda + ca] : 0.0;
      Bs[rr][c] = (r < r1 && cb < d) ? (double)SA[r * lda + cb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[rr][ty * 4 + u];
        b[u] = Bs[rr][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* out = partial + ((int64_t)sp * tiles + blockIdx.x) * 64 * 64;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(ty * 4 + u) * 64 + tx * 4 + v] = acc[u][v];
}

// Sum split partials in split order; H[i][j] = H[j][i] = scale * sum + shift * [i == j].
template <typename P>
__global__ void k_gram_reduce(const P* __restrict__ partial, int d, int tdim, int tiles,
                              int splits, double scale, double shift, double* __restrict__ H,
                              int* status) {
  const int64_t total = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e - (int64_t)i * d);
    if (j > i) continue;
    const int ti = i / tdim, tj = j / tdim;
    const int q = ti * (ti + 1) / 2 + tj;
    const int li = i - ti * tdim, lj = j - tj * tdim;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp)
      s += (double)partial[((int64_t)sp * tiles + q) * tdim * tdim + (int64_t)li * tdim + lj];
    double v = scale * s + (i == j ? shift : 0.0);
    if (!isfinite(v)) set_status(status, DEV_NONFINITE);
    H[(int64_t)i * d + j] = v;
    H[(int64_t)j * d + i] = v;
  }
}

// ----------------------------------------------------------------------------
// Transpose SA (m x d float) into the K-major MMA operand (rows d_pad, ld ldt).
// ----------------------------------------------------------------------------
template <bool BF16>
__global__ void k_gram_operand(const float* __restrict__ SA, int m, int d, int dpad, int64_t ldt,
                               void* __restrict__ op) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    int r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < m && c < d) ? SA[(int64_t)r * d + c] : 0.f;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    int c = c0 + k, r = r0 + tx;  // output row c, column r
    if (c < dpad && r < ldt) {
      float v = tile[tx][k];
      if constexpr (BF16) {
        ((__nv_bfloat16*)op)[(int64_t)c * ldt + r] = __float2bfloat16_rn(v);
      } else {
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
        ((uint32_t*)op)[(int64_t)c * ldt + r] = u;
      }
    }
  }
}

constexpr int kTcStages = 4;
constexpr int kTcTile = 128;
constexpr int kTcStageBytes = kTcTile * 128;  // one operand box: 128 rows x 128 bytes
constexpr int kTcSmem = 1024 + kTcStages * 2 * kTcStageBytes + 256;

template <int KIND>
__global__ void __launch_bounds__(192, 1) k_gram_tc(const __grid_constant__ CUtensorMap map,
                                                    int tiles, int kblocks, int splits,
                                                    float* __restrict__ partial, int* status) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  uint8_t* ring = base;  // stage s: A at ring + s*2*SB, B at + SB
  uint64_t* full = (uint64_t*)(ring + kTcStages * 2 * kTcStageBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti, tj;
  tri_index(blockIdx.x, ti, tj);
  const bool diag = (ti == tj);
  const int sp = blockIdx.y;
  const int per = (kblocks + splits - 1) / splits;
  const int kb0 = sp * per, kb1 = min(kblocks, kb0 + per);
  const int nkb = max(0, kb1 - kb0);
  constexpr int KB = (KIND == 0) ? 32 : 64;  // elements per 128-byte row
  constexpr uint32_t kIdesc = make_idesc(KIND == 0 ? 2u : 1u, kTcTile, kTcTile);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    const uint32_t bytes = diag ? kTcStageBytes : 2 * kTcStageBytes;
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kTcStages;
      const uint32_t ph = (uint32_t)((i / kTcStages) & 1);
      if (!mbar_wait(empty + s, ph ^ 1u, abort_flag)) {
        set_status(status, DEV_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      mbar_expect_tx(full + s, bytes);
      uint8_t* a = ring + s * 2 * kTcStageBytes;
      const int x = (kb0 + i) * KB;
      tma_load_2d(a, &map, x, ti * kTcTile, full + s);
      if (!diag) tma_load_2d(a + kTcStageBytes, &map, x, tj * kTcTile, full + s);
      ++issued;
    }
    // drain: every issued copy must land before the CTA can exit
    for (int i = max(0, issued - kTcStages); i < issued; ++i) {
      const int s = i % kTcStages;
      const uint32_t ph = (uint32_t)((i / kTcStages) & 1);
      volatile int never = 0;
      for (long long it = 0; it < kSpinLimit && !mbar_try_wait(full + s, ph); ++it)
        if (it > 32) __nanosleep(64);
      (void)never;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kTcStages;
      const uint32_t ph = (uint32_t)((i / kTcStages) & 1);
      if (!mbar_wait(full + s, ph, abort_flag)) {
        set_status(status, DEV_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      uint8_t* a = ring + s * 2 * kTcStageBytes;
      const uint64_t ad = smem_desc_sw128(smem_u32(a));
      const uint64_t bd = diag ? ad : smem_desc_sw128(smem_u32(a + kTcStageBytes));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // four 32-byte K steps per 128-byte row
        tc_mma<KIND>(tmem, ad + 2 * kk, bd + 2 * kk, kIdesc, (i > 0 || kk > 0) ? 1u : 0u);
      tc_commit(empty + s);
    }
    tc_commit(done);  // arrives once all issued MMAs have completed
  } else if (warp >= 2) {
    // ---- epilogue ----
    bool ok = false;
    for (long long it = 0; it < kSpinLimit; ++it) {
      if (mbar_try_wait(done, 0)) { ok = true; break; }
      if (it > 32) __nanosleep(128);
    }
    tc_fence_after();
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    float* out = partial + ((int64_t)sp * tiles + blockIdx.x) * kTcTile * kTcTile +
                 (int64_t)row * kTcTile;
    if (!ok) {
      set_status(status, DEV_TIMEOUT);
    } else if (nkb == 0 || *abort_flag) {
      for (int c = 0; c < kTcTile; ++c) out[c] = 0.f;
    } else {
#pragma unroll 1
      for (int c = 0; c < kTcTile; c += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int u = 0; u < 32; u += 4)
          *reinterpret_cast<float4*>(out + c + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                 : "memory");
  }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
cudaError_t launch_gram(const GramPlan& g, const void* SA, void* operand, float* partial_f,
                        double* partial_d, double scale, double shift, double* H, int* status,
                        cudaStream_t st) {
  cudaError_t e;
  const int red_blocks = (int)std::min<int64_t>(((int64_t)g.d * g.d + 255) / 256, 4096);
  if (g.prec == IHS_PREC_FP64) {
    const int64_t kchunk = ((g.m + g.splits - 1) / g.splits + 15) / 16 * 16;
    dim3 grid(g.tiles, g.splits);
    { k_gram_f64<double><<<grid, 256, 0, st>>>((const double*)SA, (int64_t)g.d, (int64_t)g.m, g.d,
                                                g.tiles, kchunk, partial_d); note_launches(1); }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    { k_gram_reduce<double><<<red_blocks, 256, 0, st>>>(partial_d, g.d, g.tdim, g.tiles, g.splits,
                                                      scale, shift, H, status); note_launches(1); }
    return cudaGetLastError();
  }
  const int T = (g.d + g.tdim - 1) / g.tdim;
  const int dpad = T * g.tdim;
  const bool bf16 = (g.prec == IHS_PREC_BF16);
  dim3 tg((unsigned)((g.ldt + 31) / 32), (unsigned)((dpad + 31) / 32));
  if (bf16)
    { k_gram_operand<true><<<tg, 256, 0, st>>>((const float*)SA, g.m, g.d, dpad, g.ldt, operand); note_launches(1); }
  else
    { k_gram_operand<false><<<tg, 256, 0, st>>>((const float*)SA, g.m, g.d, dpad, g.ldt, operand); note_launches(1); }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  PFN_encodeTiled enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const size_t el = bf16 ? 2 : 4;
  cuuint64_t gdim[2] = {(cuuint64_t)g.ldt, (cuuint64_t)dpad};
  cuuint64_t gstride[1] = {(cuuint64_t)(g.ldt * el)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / el), (cuuint32_t)kTcTile};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, operand, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int kblocks = (int)(g.ldt / (128 / el));
  dim3 grid(g.tiles, g.splits);
  if (bf16) {
    if ((e = ensure_smem((const void*)k_gram_tc<1>, kTcSmem)) != cudaSuccess) return e;
    { k_gram_tc<1><<<grid, 192, kTcSmem, st>>>(map, g.tiles, kblocks, g.splits, partial_f, status); note_launches(1); }
  } else {
    if ((e = ensure_smem((const void*)k_gram_tc<0>, kTcSmem)) != cudaSuccess) return e;
    { k_gram_tc<0><<<grid, 192, kTcSmem, st>>>(map, g.tiles, kblocks, g.splits, partial_f, status); note_launches(1); }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  { k_gram_reduce<float><<<red_blocks, 256, 0, st>>>(partial_f, g.d, g.tdim, g.tiles, g.splits,
                                                   scale, shift, H, status); note_launches(1); }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Exact Gram A^T A in FP64 (the reference of the sketch-quality experiment,
// App. B).  Dense: the FP64 SIMT Gram over the n rows of A (FP32 entries are
// promoted exactly), split-K partials reduced in split order.  CSR: each row
// adds its outer product a_i a_i^T to the lower triangle with FP64 atomics
// (rounding depends on the order of the atomics), then the upper triangle is
// mirrored.
// ----------------------------------------------------------------------------
__global__ void k_gram_csr_rows(int64_t n, const void* __restrict__ rowptr, int rowptr_i64,
                                const int32_t* __restrict__ col, const void* __restrict__ val,
                                int f32, int d, double* __restrict__ G) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = rowptr_i64 ? ((const int64_t*)rowptr)[i] : ((const int32_t*)rowptr)[i];
    const int64_t b = rowptr_i64 ? ((const int64_t*)rowptr)[i + 1] : ((const int32_t*)rowptr)[i + 1];
    for (int64_t p = a; p < b; ++p) {
      const int cp = col[p];
      const double vp = f32 ? (double)((const float*)val)[p] : ((const double*)val)[p];
      for (int64_t q = a; q < b; ++q) {
        const int cq = col[q];
        if (cq > cp) continue;
        const double vq = f32 ? (double)((const float*)val)[q] : ((const double*)val)[q];
        atomicAdd(G + (int64_t)cp * d + cq, vp * vq);
      }
    }
  }
}

__global__ void k_mirror_lower(double* __restrict__ G, int d) {
  const int64_t total = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e - (int64_t)i * d);
    if (j > i) G[e] = G[(int64_t)j * d + i];
  }
}

cudaError_t launch_exact_gram_dense(const void* A, int f32, int64_t n, int d, int64_t lda,
                                    int num_sms, double* partial, size_t partial_bytes, double* G,
                                    int* status, cudaStream_t st) {
  GramPlan g = make_gram_plan((int)std::min<int64_t>(n, 0x7fffffff), d, IHS_PREC_FP64, num_sms);
  // keep the partials within the buffer given
  while (g.splits > 1 && gram_partial_bytes(g) > partial_bytes) --g.splits;
  if (gram_partial_bytes(g) > partial_bytes) return cudaErrorInvalidValue;
  const int64_t kchunk = ((n + g.splits - 1) / g.splits + 15) / 16 * 16;
  dim3 grid(g.tiles, g.splits);
  if (f32)
    { k_gram_f64<float><<<grid, 256, 0, st>>>((const float*)A, lda, n, d, g.tiles, kchunk, partial); note_launches(1); }
  else
    { k_gram_f64<double><<<grid, 256, 0, st>>>((const double*)A, lda, n, d, g.tiles, kchunk, partial); note_launches(1); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int red_blocks = (int)std::min<int64_t>(((int64_t)d * d + 255) / 256, 4096);
  { k_gram_reduce<double><<<red_blocks, 256, 0, st>>>(partial, d, g.tdim, g.tiles, g.splits, 1.0,
                                                    0.0, G, status); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_exact_gram_csr(int64_t n, int d, const void* rowptr, int rowptr_i64,
                                  const int32_t* col, const void* val, int f32, double* G,
                                  cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(G, 0, (size_t)d * d * sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (n > 0)
    { k_gram_csr_rows<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(
        n, rowptr, rowptr_i64, col, val, f32, d, G); note_launches(1); }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  { k_mirror_lower<<<(unsigned)std::min<int64_t>(((int64_t)d * d + 255) / 256, 4096), 256, 0, st>>>(
      G, d); note_launches(1); }
  return cudaGetLastError();
}

// err = ||H - G||_F / ||G||_F, one CTA, sums in a fixed order (FP64).
__global__ void __launch_bounds__(1024) k_fro_ratio(const double* __restrict__ H,
                                                    const double* __restrict__ G, int64_t count,
                                                    double* __restrict__ out) {
  __shared__ double r1[32], r2[32];
  double a = 0.0, b = 0.0;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
    const double dh = H[e] - G[e];
    a = fma(dh, dh, a);
    b = fma(G[e], G[e], b);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = a;
    r2[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += r1[w];
      sb += r2[w];
    }
    out[0] = sb > 0.0 ? sqrt(sa / sb) : 0.0;
  }
}

cudaError_t launch_fro_ratio(const double* H, const double* G, int64_t count, double* out,
                             cudaStream_t st) {
  k_fro_ratio<<<1, 1024, 0, st>>>(H, G, count, out);
  note_launches(1);
  return cudaGetLastError();
}
