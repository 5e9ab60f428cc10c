// fused.cu -- one pass over a dense FP32 A per iteration that forms both
// halves of Eq. 2's subproblem: the sketch SA of the next Hessian and the
// exact gradient g = A^T (b - A x^t).
//
// Rows arrive in bucket order (the sorted CountSketch pairs, split into equal
// chunks, one warp per chunk, exactly as k_sketch_dense walks them), two rows
// at a time, so each row read from HBM is used three times while it sits in
// registers:
//   SA[h(i)] += sign(i) A_i                      (FP32, bucket order)
//   r_i = b_i - A_i x                            (float-pair, exact products)
//   g  += A_i r_i                                (float-pair, per lane/column)
// The sketch part is the same arithmetic in the same order as k_sketch_dense
// (so SA is identical); the gradient is summed in bucket order, then per CTA
// in a fixed warp order, then over CTAs in a fixed order.
//
// Used for CountSketch (s = 1) with d <= 512; other shapes take the two
// separate passes.  With form_sa = 0 the pass forms the gradient only (the
// rows still walked in the given bucket order).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kFuThreads = 256;
constexpr int kFuWarps = kFuThreads / 32;

template <int NV>
__global__ void __launch_bounds__(kFuThreads, 2) k_sketch_grad_fused(
    const float* __restrict__ A, int64_t lda, int d, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ seg_start, const int32_t* __restrict__ chunk_first, int m,
    int64_t P, int64_t CH, int nchunks, const float2* __restrict__ bs,
    const double* __restrict__ x, float* __restrict__ SA, float* __restrict__ partial,
    double* __restrict__ gcta, int form_sa) {
  constexpr int DP = NV * 128;
  __shared__ __align__(16) float xh[DP], xl[DP], nxh[DP];
  __shared__ float2 red[kFuWarps][DP];
  for (int c = threadIdx.x; c < DP; c += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (c < d) split_double(x[c], h, l);
    xh[c] = h;
    xl[c] = l;
    nxh[c] = -h;
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
  f2t gh[NV][2], gl[NV][2];  // pairs of columns (0,1) and (2,3) of each float4
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t) gh[q][t] = gl[q][t] = f2_zero();

  if (w < nchunks) {
    const int64_t c0 = (int64_t)w * CH;
    const int64_t c1 = min(P, c0 + CH);
    for (int b = chunk_first[w]; b < m; ++b) {
      const int64_t sb = seg_start[b], eb = seg_start[b + 1];
      if (sb >= c1) break;
      const int64_t lo = max(sb, c0), hi = min(eb, c1);
      if (lo >= hi) continue;
      f2t acc[NV][2];
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q][0] = acc[q][1] = f2_zero();
      for (int64_t base = lo; base < hi; base += 32) {
        const int cnt = (int)min((int64_t)32, hi - base);
        const uint32_t my = (lane < cnt) ? __ldg(perm + base + lane) : 0u;
        // this lane's row of the batch: its b split, fetched once for the warp
        const float2 bmy = (lane < cnt) ? __ldg(bs + (my & 0x7fffffffu)) : make_float2(0.f, 0.f);
        // rows two at a time: both rows' loads in flight together, and one
        // butterfly reduces both dot products (the first level exchanges the
        // rows between half-warps, so lanes 0-15 end with row j, 16-31 with j+1)
        for (int j = 0; j < cnt; j += 2) {
          const bool two = (j + 1) < cnt;
          const uint32_t e0 = __shfl_sync(0xffffffffu, my, j);
          const uint32_t e1 = __shfl_sync(0xffffffffu, my, two ? j + 1 : j);
          const float* row0 = A + (int64_t)(e0 & 0x7fffffffu) * lda;
          const float* row1 = A + (int64_t)(e1 & 0x7fffffffu) * lda;
          f2t a0[NV][2], a1[NV][2];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            a0[q][0] = a0[q][1] = a1[q][0] = a1[q][1] = f2_zero();
            if (ok[q]) {
              const float4 v0 = __ldcs(reinterpret_cast<const float4*>(row0 + colq[q]));
              a0[q][0] = f2_pack(v0.x, v0.y);
              a0[q][1] = f2_pack(v0.z, v0.w);
              if (two) {
                const float4 v1 = __ldcs(reinterpret_cast<const float4*>(row1 + colq[q]));
                a1[q][0] = f2_pack(v1.x, v1.y);
                a1[q][1] = f2_pack(v1.z, v1.w);
              }
            }
          }
          // sketch: SA[h(i)] += sign(i) A_i, rows in order
          const float sg0 = (e0 >> 31) ? -1.f : 1.f, sg1 = (e1 >> 31) ? -1.f : 1.f;
          const f2t s0 = f2_pack(sg0, sg0), s1 = f2_pack(sg1, sg1);
#pragma unroll
          for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int t = 0; t < 2; ++t) acc[q][t] = f2_fma(s0, a0[q][t], acc[q][t]);
          if (two) {
#pragma unroll
            for (int q = 0; q < NV; ++q)
#pragma unroll
              for (int t = 0; t < 2; ++t) acc[q][t] = f2_fma(s1, a1[q][t], acc[q][t]);
          }
          // residual partials: two float-pair chains per row, (p, q) packed:
          // p takes columns 0 and 2 of each float4, q columns 1 and 3
          f2t c0h = f2_zero(), c0l = f2_zero(), c1h = f2_zero(), c1l = f2_zero();
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const f2t* vh = reinterpret_cast<const f2t*>(xh + colq[q]);
            const f2t* vn = reinterpret_cast<const f2t*>(nxh + colq[q]);
            const f2t* vl = reinterpret_cast<const f2t*>(xl + colq[q]);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              dd2_fma_acc(c0h, c0l, a0[q][t], vh[t], vn[t], vl[t]);
              dd2_fma_acc(c1h, c1l, a1[q][t], vh[t], vn[t], vl[t]);
            }
          }
          float p0h, q0h, p0l, q0l, p1h, q1h, p1l, q1l;
          f2_unpack(c0h, p0h, q0h);
          f2_unpack(c0l, p0l, q0l);
          f2_unpack(c1h, p1h, q1h);
          f2_unpack(c1l, p1l, q1l);
          dd_add(p0h, p0l, q0h, q0l);
          dd_add(p1h, p1l, q1h, q1l);
          // level 16: keep my half's row, send the other row's partial
          const bool hi_half = lane >= 16;
          float kh = hi_half ? p1h : p0h, kl = hi_half ? p1l : p0l;
          const float sh_ = hi_half ? p0h : p1h, sl_ = hi_half ? p0l : p1l;
          dd_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh_, 16), __shfl_xor_sync(0xffffffffu, sl_, 16));
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, kh, o);
            const float ol = __shfl_xor_sync(0xffffffffu, kl, o);
            dd_add(kh, kl, oh, ol);
          }
          // r = b - dot for both rows (lane 0 holds row j, lane 16 row j+1)
          float r0h = __shfl_sync(0xffffffffu, bmy.x, j), r0l = __shfl_sync(0xffffffffu, bmy.y, j);
          float r1h = __shfl_sync(0xffffffffu, bmy.x, two ? j + 1 : j);
          float r1l = __shfl_sync(0xffffffffu, bmy.y, two ? j + 1 : j);
          const float d0h = __shfl_sync(0xffffffffu, kh, 0), d0l = __shfl_sync(0xffffffffu, kl, 0);
          const float d1h = __shfl_sync(0xffffffffu, kh, 16), d1l = __shfl_sync(0xffffffffu, kl, 16);
          dd_add(r0h, r0l, -d0h, -d0l);
          dd_add(r1h, r1l, -d1h, -d1l);
          if (!two) r1h = r1l = 0.f;
          // gradient
          const f2t r0h2 = f2_pack(r0h, r0h), r0n2 = f2_pack(-r0h, -r0h), r0l2 = f2_pack(r0l, r0l);
          const f2t r1h2 = f2_pack(r1h, r1h), r1n2 = f2_pack(-r1h, -r1h), r1l2 = f2_pack(r1l, r1l);
#pragma unroll
          for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              dd2_fma_acc(gh[q][t], gl[q][t], a0[q][t], r0h2, r0n2, r0l2);
              dd2_fma_acc(gh[q][t], gl[q][t], a1[q][t], r1h2, r1n2, r1l2);
            }
        }
      }
      if (!form_sa) continue;
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
        if (ok[q]) {
          float4 o;
          f2_unpack(acc[q][0], o.x, o.y);
          f2_unpack(acc[q][1], o.z, o.w);
          *reinterpret_cast<float4*>(dst + colq[q]) = o;
        }
    }
  }
  // CTA reduction of the gradient partials in a fixed warp order (float pairs)
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      float h0, h1, l0, l1;
      f2_unpack(gh[q][t], h0, h1);
      f2_unpack(gl[q][t], l0, l1);
      red[wib][colq[q] + 2 * t] = make_float2(h0, l0);
      red[wib][colq[q] + 2 * t + 1] = make_float2(h1, l1);
    }
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
                                     double* g, double lam, cudaStream_t st, void* prof,
                                     bool form_sa) {
  const int blocks = fused_ctas(p);
  const int nv = (int)((A.d + 127) / 128);
#define FU(NV)                                                                              \
  k_sketch_grad_fused<NV><<<blocks, kFuThreads, 0, st>>>((const float*)A.val, A.ld, (int)A.d, \
                                                         perm, seg, cf, p.m, p.P, p.chunk,     \
                                                         p.nchunks, bsplit, x, SA, partial, gcta, \
                                                         form_sa ? 1 : 0)
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
  if (form_sa) {
    prof_stage_end(prof);
    prof_stage_begin(prof, IHS_ST_SKETCH_FIX);
    e = launch_sketch_fixup_f32(p, seg, (int)A.d, partial, SA, st);
    if (e != cudaSuccess) return e;
  }
  return launch_reduce_partials(gcta, blocks, (int)A.d, x, lam, g, st);
}
