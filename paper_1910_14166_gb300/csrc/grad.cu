// grad.cu -- r = b - A x and g = A^T r (Eq. 2's linear term), FP64-class.
//
// FP64 data: plain FP64 fused multiply-adds.
// FP32 data: GB300 issues FP64 at 1/62 of the FP32 rate (1.2 vs 75 TFLOP/s
// measured), so one FP64 operation per element would leave the pass far
// below the memory roofline.  Instead every product A_ij * y of an FP32 entry
// with an FP64 factor y = yh + yl (two floats) is formed exactly as a float
// pair (TwoProd by FMA) and summed with TwoSum (Dekker 1971; Ogita, Rump &
// Oishi 2005): about 48 significant bits per accumulator, with the FP64
// conversion only once per warp at the end.
//
// Dense layout: one warp per equal row chunk; lanes own interleaved 4-float
// column groups, so each row is one coalesced read.  Per row the warp forms
// the dot product, reduces it across lanes, and every lane then adds r_i
// times its own columns into register accumulators (a single pass over A).
// Per-warp partial gradients are summed in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

constexpr int kRgThreads = 256;

int rg_dense_warps(int64_t n) {
  int64_t w = 152 * 16;  // 16 warps per SM, enough loads in flight for HBM
  w = std::min<int64_t>(w, (n + 3) / 4);
  return (int)std::max<int64_t>(1, w);
}

// ---------------------------------------------------------------- FP32 data --
template <int NV, bool VEC4>
__global__ void __launch_bounds__(kRgThreads) k_rg_dense_f32(
    const float* __restrict__ A, int64_t lda, int64_t n, int d, const float2* __restrict__ bs,
    const double* __restrict__ x, double* __restrict__ r_out, double* __restrict__ gpart,
    int nwarps) {
  extern __shared__ float xs[];  // xh[dpad], xl[dpad]
  const int dpad = NV * 128;
  float* xh = xs;
  float* xl = xs + dpad;
  for (int c = threadIdx.x; c < dpad; c += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (c < d) split_double(x[c], h, l);
    xh[c] = h;
    xl[c] = l;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int64_t per = (n + nwarps - 1) / nwarps;
  const int64_t r0 = (int64_t)w * per, r1 = min(n, r0 + per);

  constexpr int V = VEC4 ? 4 : 1;
  constexpr int NQ = VEC4 ? NV : NV * 4;  // vector groups per lane
  float gh[NQ][V], gl[NQ][V], ah[NQ][V], al[NQ][V];
  int colq[NQ];
  bool ok[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    colq[q] = (q * 32 + lane) * V;
    ok[q] = colq[q] < d;
#pragma unroll
    for (int t = 0; t < V; ++t) {
      gh[q][t] = 0.f;
      gl[q][t] = 0.f;
      ah[q][t] = xh[colq[q] + t];
      al[q][t] = xl[colq[q] + t];
    }
  }
  for (int64_t i = r0; i < r1; ++i) {
    const float* row = A + i * lda;
    float a[NQ][V];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (ok[q]) {
        if constexpr (VEC4) {
          float4 v = __ldcs(reinterpret_cast<const float4*>(row + colq[q]));
          a[q][0] = v.x; a[q][1] = v.y; a[q][2] = v.z; a[q][3] = v.w;
        } else {
          a[q][0] = __ldcs(row + colq[q]);
        }
      } else {
#pragma unroll
        for (int t = 0; t < V; ++t) a[q][t] = 0.f;
      }
    }
    // dot product A_i . x as a float pair
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int t = 0; t < V; ++t) dd_fma_acc(sh, sl, a[q][t], ah[q][t], al[q][t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float oh = __shfl_xor_sync(0xffffffffu, sh, o);
      float ol = __shfl_xor_sync(0xffffffffu, sl, o);
      dd_add(sh, sl, oh, ol);
    }
    // r_i = b_i - dot, as a float pair
    const float2 b2 = bs ? __ldg(bs + i) : make_float2(0.f, 0.f);  // no b: r = -A x
    float rh = b2.x, rl = b2.y;
    dd_add(rh, rl, -sh, -sl);
    if (r_out && lane == 0) r_out[i] = (double)rh + (double)rl;
    // g += A_i^T r_i
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int t = 0; t < V; ++t) dd_fma_acc(gh[q][t], gl[q][t], a[q][t], rh, rl);
  }
  double* gp = gpart + (int64_t)w * d;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int t = 0; t < V; ++t) {
      int c = colq[q] + t;
      if (c < d) gp[c] = (double)gh[q][t] + (double)gl[q][t];
    }
}

// The same pass for 16-byte-aligned rows with packed FP32 pair arithmetic
// and two rows per step (the fused pass's arithmetic without the sketch):
// both rows' loads are in flight together, one butterfly reduces both dot
// products (its first level exchanges the rows between half-warps), and the
// float-pair steps run on pairs of columns.  Rows are taken in order, so
// each column's gradient is summed in the same row order as above.
template <int NV>
__global__ void __launch_bounds__(kRgThreads, 2) k_rg_dense_f32x2(
    const float* __restrict__ A, int64_t lda, int64_t n, int d, const float2* __restrict__ bs,
    const double* __restrict__ x, double* __restrict__ r_out, double* __restrict__ gpart,
    int nwarps) {
  constexpr int DP = NV * 128;
  __shared__ __align__(16) float xh[DP], xl[DP], nxh[DP];
  for (int c = threadIdx.x; c < DP; c += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (c < d) split_double(x[c], h, l);
    xh[c] = h;
    xl[c] = l;
    nxh[c] = -h;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int64_t per = (n + nwarps - 1) / nwarps;
  const int64_t r0 = (int64_t)w * per, r1 = min(n, r0 + per);
  int colq[NV];
  bool ok[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    colq[q] = (q * 32 + lane) * 4;
    ok[q] = colq[q] < d;
  }
  f2t gh[NV][2], gl[NV][2];
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int t = 0; t < 2; ++t) gh[q][t] = gl[q][t] = f2_zero();
  for (int64_t i = r0; i < r1; i += 2) {
    const bool two = i + 1 < r1;
    const float* row0 = A + i * lda;
    const float* row1 = row0 + lda;
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
    const float2 b0 = bs ? __ldg(bs + i) : make_float2(0.f, 0.f);  // no b: r = -A x
    const float2 b1 = (bs && two) ? __ldg(bs + i + 1) : make_float2(0.f, 0.f);
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
    float r0h = b0.x, r0l = b0.y, r1h = b1.x, r1l = b1.y;
    const float d0h = __shfl_sync(0xffffffffu, kh, 0), d0l = __shfl_sync(0xffffffffu, kl, 0);
    const float d1h = __shfl_sync(0xffffffffu, kh, 16), d1l = __shfl_sync(0xffffffffu, kl, 16);
    dd_add(r0h, r0l, -d0h, -d0l);
    dd_add(r1h, r1l, -d1h, -d1l);
    if (!two) r1h = r1l = 0.f;
    if (r_out) {
      if (lane == 0) r_out[i] = (double)r0h + (double)r0l;
      if (lane == 1 && two) r_out[i + 1] = (double)r1h + (double)r1l;
    }
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
  double* gp = gpart + (int64_t)w * d;
#pragma unroll
  for (int q = 0; q < NV; ++q)
    if (ok[q])
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        float h0, h1, l0, l1;
        f2_unpack(gh[q][t], h0, h1);
        f2_unpack(gl[q][t], l0, l1);
        gp[colq[q] + 2 * t] = (double)h0 + (double)l0;
        gp[colq[q] + 2 * t + 1] = (double)h1 + (double)l1;
      }
}

// ---------------------------------------------------------------- FP64 data --
template <int NQ>
__global__ void __launch_bounds__(kRgThreads) k_rg_dense_f64(
    const double* __restrict__ A, int64_t lda, int64_t n, int d, const double* __restrict__ b,
    const double* __restrict__ x, double* __restrict__ r_out, double* __restrict__ gpart,
    int nwarps) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int64_t per = (n + nwarps - 1) / nwarps;
  const int64_t r0 = (int64_t)w * per, r1 = min(n, r0 + per);
  double g[NQ], xv[NQ];
  int colq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    colq[q] = q * 32 + lane;
    g[q] = 0.0;
    xv[q] = colq[q] < d ? x[colq[q]] : 0.0;
  }
  for (int64_t i = r0; i < r1; ++i) {
    const double* row = A + i * lda;
    double a[NQ];
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      a[q] = colq[q] < d ? __ldcs(row + colq[q]) : 0.0;
      s = fma(a[q], xv[q], s);
    }
    s = warp_sum(s);
    const double ri = (b ? b[i] : 0.0) - s;
    if (r_out && lane == 0) r_out[i] = ri;
#pragma unroll
    for (int q = 0; q < NQ; ++q) g[q] = fma(a[q], ri, g[q]);
  }
  double* gp = gpart + (int64_t)w * d;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (colq[q] < d) gp[colq[q]] = g[q];
}

// g[c] = sum_w gpart[w][c] - lam * x[c], in two levels when there are many
// warp partials: CTA (column block, part p) sums the partials of its slice
// [p W / P, (p + 1) W / P) (eight interleaved warps, then a fixed combine)
// into g2[p][c], and a second kernel adds the P slice sums in order.  One
// level (P = 1) writes g directly.  Either way the order is fixed, so the
// gradient is reproducible.  The split puts the FP64 additions (about two
// lanes a clock an SM on GB300) on P times more SMs.
int rg_reduce_split(int nwarps) { return std::min(32, std::max(1, nwarps / 64)); }

size_t rg_partial_bytes(int nwarps, int64_t d) {
  const int P = rg_reduce_split(nwarps);
  return (size_t)(nwarps + (P > 1 ? P : 0)) * (size_t)d * sizeof(double);
}

__global__ void k_reduce_gpart(const double* __restrict__ gpart, int nwarps, int d, int P,
                               const double* __restrict__ x, double lam, double* __restrict__ g,
                               double* __restrict__ g2) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int p = blockIdx.y;
  const int w0 = (int)((int64_t)p * nwarps / P), w1 = (int)((int64_t)(p + 1) * nwarps / P);
  double acc = 0.0;
  if (c < d)
    for (int w = w0 + wi; w < w1; w += 8) acc += gpart[(int64_t)w * d + c];
  part[wi][lane] = acc;
  __syncthreads();
  if (wi == 0 && c < d) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += part[k][lane];
    if (P > 1) {
      g2[(int64_t)p * d + c] = s;
    } else {
      if (lam != 0.0) s -= lam * x[c];
      g[c] = s;
    }
  }
}

__global__ void k_reduce_gpart2(const double* __restrict__ g2, int P, int d,
                                const double* __restrict__ x, double lam, double* __restrict__ g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  double s = 0.0;
  for (int p = 0; p < P; ++p) s += g2[(int64_t)p * d + c];
  if (lam != 0.0) s -= lam * x[c];
  g[c] = s;
}

cudaError_t launch_resid_grad_dense(const DenseA& A, const double* b, const float2* bsplit,
                                    const double* x, double* r, double* gpart, int nwarps,
                                    double* g, double lam, cudaStream_t st) {
  const int d = (int)A.d;
  const int blocks = (nwarps * 32 + kRgThreads - 1) / kRgThreads;
  if (A.n > 0) {
    if (A.f32) {
      const bool v4 = (A.ld % 4 == 0) && (A.d % 4 == 0) && ((uintptr_t)A.val % 16 == 0);
      const int nv = (d + 127) / 128;  // 4-float groups of 32 lanes
      const size_t smem = (size_t)2 * nv * 128 * sizeof(float);
#define RG32(NV)                                                                              \
  (v4 ? (k_rg_dense_f32<NV, true><<<blocks, kRgThreads, smem, st>>>(                         \
             (const float*)A.val, A.ld, A.n, d, bsplit, x, r, gpart, nwarps), 0)              \
      : (k_rg_dense_f32<NV, false><<<blocks, kRgThreads, smem, st>>>(                        \
             (const float*)A.val, A.ld, A.n, d, bsplit, x, r, gpart, nwarps), 0))
#define RGX2(NV)                                                                              \
  k_rg_dense_f32x2<NV><<<blocks, kRgThreads, 0, st>>>((const float*)A.val, A.ld, A.n, d, bsplit, \
                                                      x, r, gpart, nwarps)
      if (v4 && nv <= 4) {
        switch (nv) {
          case 1: RGX2(1); break;
          case 2: RGX2(2); break;
          case 3: RGX2(3); break;
          default: RGX2(4); break;
        }
      } else switch (nv) {
        case 1: RG32(1); break;
        case 2: RG32(2); break;
        case 3: RG32(3); break;
        case 4: RG32(4); break;
        case 5: RG32(5); break;
        case 6: RG32(6); break;
        case 7: RG32(7); break;
        case 8: RG32(8); break;
        default: return cudaErrorInvalidValue;
      }
#undef RG32
#undef RGX2
      note_launches(1);
    } else {
      const int nq = (d + 31) / 32;
#define RG64(NQ)                                                                              \
  k_rg_dense_f64<NQ><<<blocks, kRgThreads, 0, st>>>((const double*)A.val, A.ld, A.n, d, b, x, \
                                                    r, gpart, nwarps)
      if (nq <= 2) RG64(2);
      else if (nq <= 4) RG64(4);
      else if (nq <= 8) RG64(8);
      else if (nq <= 16) RG64(16);
      else if (nq <= 32) RG64(32);
      else return cudaErrorInvalidValue;
#undef RG64
      note_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    cudaMemsetAsync(gpart, 0, (size_t)nwarps * d * sizeof(double), st);
  }
  const int P = rg_reduce_split(nwarps);
  double* g2 = gpart + (int64_t)nwarps * d;  // P x d slice sums (P > 1)
  { k_reduce_gpart<<<dim3((d + 31) / 32, P), 256, 0, st>>>(gpart, nwarps, d, P, x, lam, g, g2); note_launches(1); }
  if (P > 1) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    { k_reduce_gpart2<<<(d + 127) / 128, 128, 0, st>>>(g2, P, d, x, lam, g); note_launches(1); }
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------- CSR ----
// r_i = b_i - sum_p val_p x[col_p], one thread per row.  FP32 values: float
// pair accumulation with x split in shared memory; r stored as (hi, lo).
template <typename RP>
__global__ void k_resid_csr_f32(int64_t n, int d, const RP* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const float* __restrict__ val,
                                const float2* __restrict__ bs, const double* __restrict__ x,
                                float2* __restrict__ r2, double* __restrict__ r_out) {
  extern __shared__ float xs2[];
  float* xh = xs2;
  float* xl = xs2 + d;
  for (int c = threadIdx.x; c < d; c += blockDim.x) split_double(x[c], xh[c], xl[c]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float sh = 0.f, sl = 0.f;
    const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int64_t p = p0; p < p1; ++p) {
      const int c = __ldg(col + p);
      dd_fma_acc(sh, sl, __ldg(val + p), xh[c], xl[c]);
    }
    const float2 b2 = bs ? __ldg(bs + i) : make_float2(0.f, 0.f);
    float bh = b2.x, bl = b2.y;
    dd_add(bh, bl, -sh, -sl);
    r2[i] = make_float2(bh, bl);
    if (r_out) r_out[i] = (double)bh + (double)bl;
  }
}

template <typename RP>
__global__ void k_resid_csr_f64(int64_t n, const RP* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                const double* __restrict__ b, const double* __restrict__ x,
                                double* __restrict__ r, double* __restrict__ r_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    const int64_t p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int64_t p = p0; p < p1; ++p) s = fma(__ldg(val + p), __ldg(x + __ldg(col + p)), s);
    const double ri = (b ? b[i] : 0.0) - s;
    r[i] = ri;
    if (r_out) r_out[i] = ri;
  }
}

cudaError_t launch_resid_csr(int64_t n, int64_t d, const void* rowptr, int rowptr_i64,
                             const int32_t* col, const void* val, int f32, const double* b,
                             const float2* bsplit, const double* x, void* rbuf, double* r_out,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (f32) {
    const size_t smem = (size_t)2 * d * sizeof(float);
    if (rowptr_i64)
      { k_resid_csr_f32<int64_t><<<blocks, 256, smem, st>>>(n, (int)d, (const int64_t*)rowptr, col,
                                                          (const float*)val, bsplit, x, (float2*)rbuf,
                                                          r_out); note_launches(1); }
    else
      { k_resid_csr_f32<int32_t><<<blocks, 256, smem, st>>>(n, (int)d, (const int32_t*)rowptr, col,
                                                          (const float*)val, bsplit, x, (float2*)rbuf,
                                                          r_out); note_launches(1); }
  } else {
    if (rowptr_i64)
      { k_resid_csr_f64<int64_t><<<blocks, 256, 0, st>>>(n, (const int64_t*)rowptr, col,
                                                       (const double*)val, b, x, (double*)rbuf,
                                                       r_out); note_launches(1); }
    else
      { k_resid_csr_f64<int32_t><<<blocks, 256, 0, st>>>(n, (const int32_t*)rowptr, col,
                                                       (const double*)val, b, x, (double*)rbuf,
                                                       r_out); note_launches(1); }
  }
  return cudaGetLastError();
}

// g_j = sum over column j's entries of val * r[row]: one warp per column item,
// then the items of a column summed in item order.
template <bool F32>
__global__ void k_grad_csc_items(const int32_t* __restrict__ rowidx, const void* __restrict__ val,
                                 int nitems, const int64_t* __restrict__ ib,
                                 const int64_t* __restrict__ ie, const void* __restrict__ rbuf,
                                 double* __restrict__ item_part) {
  const int lane = threadIdx.x & 31;
  const int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (it >= nitems) return;
  const int64_t e0 = ib[it], e1 = ie[it];
  if constexpr (F32) {
    const float* v = (const float*)val;
    const float2* r2 = (const float2*)rbuf;
    float h = 0.f, l = 0.f;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      float2 rr = __ldg(r2 + __ldg(rowidx + e));
      dd_fma_acc(h, l, __ldg(v + e), rr.x, rr.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float oh = __shfl_xor_sync(0xffffffffu, h, o);
      float ol = __shfl_xor_sync(0xffffffffu, l, o);
      dd_add(h, l, oh, ol);
    }
    if (lane == 0) item_part[it] = (double)h + (double)l;
  } else {
    const double* v = (const double*)val;
    const double* r = (const double*)rbuf;
    double s = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) s = fma(__ldg(v + e), __ldg(r + __ldg(rowidx + e)), s);
    s = warp_sum(s);
    if (lane == 0) item_part[it] = s;
  }
}

__global__ void k_grad_csc_cols(const int32_t* __restrict__ col_first_item, int d,
                                const double* __restrict__ item_part,
                                const double* __restrict__ x, double lam,
                                double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int it = col_first_item[j]; it < col_first_item[j + 1]; ++it) s += item_part[it];
  if (lam != 0.0) s -= lam * x[j];
  g[j] = s;
}

cudaError_t launch_grad_csc(const CscA& A, const void* rbuf, double* item_part, const double* x,
                            double lam, double* g, cudaStream_t st) {
  if (A.nitems > 0) {
    const unsigned blocks = (unsigned)((A.nitems + 7) / 8);
    if (A.f32)
      { k_grad_csc_items<true><<<blocks, 256, 0, st>>>(A.rowidx, A.val, A.nitems, A.item_begin,
                                                     A.item_end, rbuf, item_part); note_launches(1); }
    else
      { k_grad_csc_items<false><<<blocks, 256, 0, st>>>(A.rowidx, A.val, A.nitems, A.item_begin,
                                                      A.item_end, rbuf, item_part); note_launches(1); }
  }
  { k_grad_csc_cols<<<(unsigned)((A.d + 127) / 128), 128, 0, st>>>(A.col_first_item, (int)A.d,
                                                                 item_part, x, lam, g); note_launches(1); }
  return cudaGetLastError();
}

__global__ void k_split_b(const double* __restrict__ b, int64_t n, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float h, l;
    split_double(b[i], h, l);
    out[i] = make_float2(h, l);
  }
}

cudaError_t launch_split_b(const double* b, int64_t n, float2* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  { k_split_b<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(b, n, out); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* part, int nparts, int d, const double* x,
                                   double lam, double* g, cudaStream_t st) {
  k_reduce_gpart<<<(d + 31) / 32, 256, 0, st>>>(part, nparts, d, 1, x, lam, g, nullptr);
  note_launches(1);
  return cudaGetLastError();
}
