// fused.cu -- one pass over a dense FP32 A per iteration that forms both
// halves of Eq. 2's subproblem: the sketch SA of the next Hessian and the
// exact gradient g = A^T (b - A x^t).
//
// Rows arrive in bucket order (the sorted CountSketch pairs, split into equal
// chunks, one warp per chunk, exactly as k_sketch_dense walks them), so each
// row read from HBM is used three times while it sits in registers:
//   SA[h(i)] += sign(i) A_i                      (FP32, bucket order)
//   r_i = b_i - A_i x                            (float-pair, exact products)
//   g  += A_i r_i                                (float-pair, per lane/column)
// The sketch part is the same arithmetic in the same order as k_sketch_dense
// (so SA is identical); the gradient is summed in bucket order, then per CTA
// in a fixed warp order, then over CTAs in a fixed order.
//
// Used for CountSketch (s = 1) with d <= 512; other shapes take the two
// separate passes.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kFuThreads = 256;
constexpr int kFuWarps = kFuThreads / 32;

template <int NV>
__global__ void __launch_bounds__(kFuThreads) k_sketch_grad_fused(
    const float* __restrict__ A, int64_t lda, int d, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ seg_start, const int32_t* __restrict__ chunk_first, int m,
    int64_t P, int64_t CH, int nchunks, const float2* __restrict__ bs,
    const double* __restrict__ x, float* __restrict__ SA, float* __restrict__ partial,
    double* __restrict__ gcta) {
  constexpr int DP = NV * 128;
  __shared__ float xh[DP], xl[DP];
  __shared__ float2 red[kFuWarps][DP];
  for (int c = threadIdx.x; c < DP; c += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (c < d) split_double(x[c], h, l);
    xh[c] = h;
    xl[c] = l;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kFuWarps + wib;
  int colq[NV];
  bool ok[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    colq[q] = (q * 32 + lane) * 4;
    ok[q] = colq[q] < d;
  }
  float gh[NV][4], gl[NV][4];
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t) gh[q][t] = gl[q][t] = 0.f;

  if (w < nchunks) {
    const int64_t c0 = (int64_t)w * CH;
    const int64_t c1 = min(P, c0 + CH);
    for (int b = chunk_first[w]; b < m; ++b) {
      const int64_t sb = seg_start[b], eb = seg_start[b + 1];
      if (sb >= c1) break;
      const int64_t lo = max(sb, c0), hi = min(eb, c1);
      if (lo >= hi) continue;
      float acc[NV][4];
#pragma unroll
      for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[q][t] = 0.f;
      for (int64_t base = lo; base < hi; base += 32) {
        const int cnt = (int)min((int64_t)32, hi - base);
        const uint32_t my = (lane < cnt) ? __ldg(perm + base + lane) : 0u;
        // this lane's row of the batch: its b split, fetched once for the warp
        const float2 bmy = (lane < cnt) ? __ldg(bs + (my & 0x7fffffffu)) : make_float2(0.f, 0.f);
        for (int j = 0; j < cnt; ++j) {
          const uint32_t e = __shfl_sync(0xffffffffu, my, j);
          const float* row = A + (int64_t)(e & 0x7fffffffu) * lda;
          const bool neg = (e >> 31) != 0;
          float a[NV][4];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            if (ok[q]) {
              const float4 v = __ldcs(reinterpret_cast<const float4*>(row + colq[q]));
              a[q][0] = v.x; a[q][1] = v.y; a[q][2] = v.z; a[q][3] = v.w;
            } else {
              a[q][0] = a[q][1] = a[q][2] = a[q][3] = 0.f;
            }
          }
          // sketch
#pragma unroll
          for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[q][t] = neg ? acc[q][t] - a[q][t] : acc[q][t] + a[q][t];
          // residual: four independent float-pair chains, then a warp reduction
          float s0h = 0.f, s0l = 0.f, s1h = 0.f, s1l = 0.f;
          float s2h = 0.f, s2l = 0.f, s3h = 0.f, s3l = 0.f;
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const float4 vh = *reinterpret_cast<const float4*>(xh + colq[q]);
            const float4 vl = *reinterpret_cast<const float4*>(xl + colq[q]);
            dd_fma_acc(s0h, s0l, a[q][0], vh.x, vl.x);
            dd_fma_acc(s1h, s1l, a[q][1], vh.y, vl.y);
            dd_fma_acc(s2h, s2l, a[q][2], vh.z, vl.z);
            dd_fma_acc(s3h, s3l, a[q][3], vh.w, vl.w);
          }
          dd_add(s0h, s0l, s1h, s1l);
          dd_add(s2h, s2l, s3h, s3l);
          dd_add(s0h, s0l, s2h, s2l);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, s0h, o);
            const float ol = __shfl_xor_sync(0xffffffffu, s0l, o);
            dd_add(s0h, s0l, oh, ol);
          }
          float rh = __shfl_sync(0xffffffffu, bmy.x, j), rl = __shfl_sync(0xffffffffu, bmy.y, j);
          dd_add(rh, rl, -s0h, -s0l);
          // gradient
#pragma unroll
          for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t) dd_fma_acc(gh[q][t], gl[q][t], a[q][t], rh, rl);
        }
      }
      const bool split = (sb / CH) != ((eb - 1) / CH);
      float* dst;
      if (!split) {
        dst = SA + (int64_t)b * d;
      } else {
        const int slot = ((sb / CH) == w && sb != c0) ? 1 : 0;
        dst = partial + ((int64_t)w * 2 + slot) * d;
      }
#pragma unroll
      for (int q = 0; q < NV; ++q)
        if (ok[q]) *reinterpret_cast<float4*>(dst + colq[q]) =
            make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
  }
  // CTA reduction of the gradient partials in a fixed warp order (float pairs)
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t) red[wib][colq[q] + t] = make_float2(gh[q][t], gl[q][t]);
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    float h = red[0][c].x, l = red[0][c].y;
    for (int k = 1; k < kFuWarps; ++k) dd_add(h, l, red[k][c].x, red[k][c].y);
    gcta[(int64_t)blockIdx.x * d + c] = (double)h + (double)l;
  }
}

}  // namespace

bool fused_supported(const DenseA& A, int s) {
  return A.f32 && s == 1 && A.d <= 512 && (A.ld % 4 == 0) && (A.d % 4 == 0) &&
         ((uintptr_t)A.val % 16 == 0);
}

int fused_ctas(const SortPlan& p) { return (p.nchunks + kFuWarps - 1) / kFuWarps; }

cudaError_t launch_sketch_grad_fused(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                                     const int32_t* seg, const int32_t* cf, const float2* bsplit,
                                     const double* x, float* SA, float* partial, double* gcta,
                                     double* g, double lam, cudaStream_t st, void* prof) {
  const int blocks = fused_ctas(p);
  const int nv = (int)((A.d + 127) / 128);
#define FU(NV)                                                                              \
  k_sketch_grad_fused<NV><<<blocks, kFuThreads, 0, st>>>((const float*)A.val, A.ld, (int)A.d, \
                                                         perm, seg, cf, p.m, p.P, p.chunk,     \
                                                         p.nchunks, bsplit, x, SA, partial, gcta)
  switch (nv) {
    case 1: FU(1); break;
    case 2: FU(2); break;
    case 3: FU(3); break;
    case 4: FU(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef FU
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_stage_end(prof);
  prof_stage_begin(prof, IHS_ST_SKETCH_FIX);
  e = launch_sketch_fixup_f32(p, seg, (int)A.d, partial, SA, st);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(gcta, blocks, (int)A.d, x, lam, g, st);
}
