// common.cuh -- device utilities shared by the IHS kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ihs.h"

#define IHS_DEV __device__ __forceinline__

// Device status word codes (written by kernels, read at synchronisation).
enum : int {
  DEV_OK = 0,
  DEV_NOT_SPD = IHS_ERR_NOT_SPD,
  DEV_NOT_CONVERGED = IHS_ERR_NOT_CONVERGED,
  DEV_NONFINITE = IHS_ERR_NONFINITE,
  DEV_TIMEOUT = IHS_ERR_TIMEOUT,
};

IHS_DEV void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014), counter style: output j of the
// generator started at `state` is the finaliser of state + (j+1)*gamma.
// ---------------------------------------------------------------------------
constexpr uint64_t kSmGamma = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t sm64_finalise(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_out(uint64_t state, uint64_t j) {
  return sm64_finalise(state + (j + 1) * kSmGamma);
}

// Keys of one sketch draw: key[p] for the block pair (2p, 2p + 1) of
// iteration t (at most 64 blocks; the first ceil(s / 2) keys are used).
constexpr int kMaxBlocks = 64;
struct SketchKeys {
  uint64_t key[kMaxBlocks];
  int s;
  int mb;  // rows per block, m / s
};

// The draw of Sec. 2's CountSketch / SJLT for row i (the paper names no
// generator): one SplitMix64 output w = out(key[p], i) per row and block pair
// (2p, 2p + 1).  Block 2p takes the high 32 bits of w, block 2p + 1 the low
// 32 bits; a block's bucket is the multiply-shift range reduction of its
// half, floor(h32 * mb / 2^32), and its sign is -1 when bit 0 of the other
// half is set.  With s = 1 only block 0 exists.
IHS_DEV int draw_bucket(uint32_t h32, int mb) {
  return (int)(((uint64_t)h32 * (uint64_t)(uint32_t)mb) >> 32);
}
// Global row of S and sign for (block k, row i).
IHS_DEV void sketch_draw(const SketchKeys& K, int k, uint64_t i, int& row, int& neg) {
  const uint64_t w = sm64_out(K.key[k >> 1], i);
  const uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w;
  row = k * K.mb + draw_bucket((k & 1) ? lo : hi, K.mb);
  neg = (int)(((k & 1) ? hi : lo) & 1u);
}

// ---------------------------------------------------------------------------
// Double-float ("float-float") arithmetic from error-free transformations:
// TwoProd via FMA and Knuth's TwoSum (Dekker 1971; Ogita, Rump & Oishi 2005).
// A pair (hi, lo) carries about 48 significant bits; every product of an
// FP32 value with the hi part of a pair is exact.
// ---------------------------------------------------------------------------
IHS_DEV void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
IHS_DEV void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (hi, lo) += a * (yh + yl), yh/yl the split of an FP64 factor.
IHS_DEV void dd_fma_acc(float& hi, float& lo, float a, float yh, float yl) {
  float p = __fmul_rn(a, yh);
  float pe = __fmaf_rn(a, yh, -p);  // exact low part of a*yh
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
  lo = __fmaf_rn(a, yl, lo);
}
// (ah, al) + (bh, bl), renormalised.
IHS_DEV void dd_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, ah, al);
}
// Packed FP32 pairs (the sm_100 family's two-wide FP32 instructions, through
// the __fadd2_rn / __fmul2_rn / __ffma2_rn intrinsics): each applies the
// scalar round-to-nearest operation to both halves, so the results are
// those of the scalar code, with half the instructions issued.
typedef float2 f2t;
__device__ __forceinline__ f2t f2_pack(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ void f2_unpack(f2t v, float& lo, float& hi) {
  lo = v.x;
  hi = v.y;
}
__device__ __forceinline__ f2t f2_neg(f2t a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2t f2_add(f2t a, f2t b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2t f2_sub(f2t a, f2t b) { return __fadd2_rn(a, f2_neg(b)); }
__device__ __forceinline__ f2t f2_mul(f2t a, f2t b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2t f2_fma(f2t a, f2t b, f2t c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2t f2_zero() { return make_float2(0.f, 0.f); }
// (hi, lo) += a * (yh + yl) on both halves, given nyh = -yh: the same steps
// as dd_fma_acc (exact product a*yh by FMA, TwoSum into hi, low parts and
// a*yl into lo).  p = a*yh is carried as np = -p, which changes no rounding.
__device__ __forceinline__ void dd2_fma_acc(f2t& hi, f2t& lo, f2t a, f2t yh, f2t nyh, f2t yl) {
  const f2t np = f2_mul(a, nyh);
  const f2t pe = f2_fma(a, yh, np);
  const f2t s = f2_sub(hi, np);
  const f2t bb = f2_sub(s, hi);
  const f2t e = f2_sub(f2_sub(hi, f2_sub(s, bb)), f2_add(np, bb));
  hi = s;
  lo = f2_fma(a, yl, f2_add(lo, f2_add(e, pe)));
}

IHS_DEV void split_double(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

// ---------------------------------------------------------------------------
// Warp helpers.
// ---------------------------------------------------------------------------
IHS_DEV unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
template <typename T>
IHS_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1/sqrt(p) in FP64 with a short dependency chain, for the Cholesky pivots
// (each column of a sweep waits on one).  Newton-Raphson for f(y) = 1/y^2 - p:
// y <- y + (y/2)(1 - p y^2), which squares the relative error each step.  The
// seed is the FP32 reciprocal square root of p truncated to FP32 (relative
// error about 2^-21); two steps bring it to about 2^-84 before rounding, so
// the result is within about an ulp of 1/sqrt(p).  Each step is three
// dependent FP64 operations, six in all, where the FP64 library routine's
// chain is several times longer (GB300 issues one FP64 warp instruction per
// 64 cycles a sub-partition, so chain length sets a sweep's time).  The
// conversions between FP64 and FP32 go through the bit patterns (integer
// operations).  p outside FP32's normal exponent range takes rsqrt().
IHS_DEV double rsqrt_nr(double p) {
  const int hi = __double2hiint(p);
  const int E = (hi >> 20) & 0x7ff;
  if (hi < 0 || E < 1023 - 126 || E > 1023 + 127) return rsqrt(p);
  // p truncated to FP32: exponent rebased from 1023 to 127, top 23 mantissa bits
  const unsigned fb = ((unsigned)(hi - ((1023 - 127) << 20)) << 3) |
                      ((unsigned)__double2loint(p) >> 29);
  const float yf = rsqrtf(__uint_as_float(fb));
  // yf widened to FP64 exactly (a positive normal FP32 value)
  const unsigned yb = __float_as_uint(yf);
  double y = __hiloint2double((int)((yb >> 3) + ((1023 - 127) << 20)), (int)(yb << 29));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double h = 0.5 * y;
    const double e = fma(-(p * y), y, 1.0);  // 1 - p y^2
    y = fma(h, e, y);
  }
  return y;
}

// Load / store helpers with a compile-time vector width.
template <typename T, int V> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<double, 2> { using type = double2; };
template <> struct VecT<double, 1> { using type = double; };

template <typename T, int V>
IHS_DEV void load_vec(const T* p, T (&out)[V]) {
  if constexpr (V == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (V == 2) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = v.x; out[1] = v.y;
  } else {
    out[0] = __ldg(p);
  }
}
// Streaming (evict-first) variant for data read once per pass.
template <typename T, int V>
IHS_DEV void load_vec_stream(const T* p, T (&out)[V]) {
  if constexpr (V == 4) {
    float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (V == 2) {
    double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    out[0] = v.x; out[1] = v.y;
  } else {
    out[0] = __ldcs(p);
  }
}

// Bounded spin budget for every device-side wait (about a second at 2 GHz
// with the back-off below); on expiry the waiter records DEV_TIMEOUT.
constexpr long long kSpinLimit = 1ll << 26;

IHS_DEV uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// mbarrier primitives (shared memory, CTA scope): init with an arrival
// count, arrive (release), and one test of a phase's completion (acquire).
IHS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
IHS_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
IHS_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
IHS_DEV void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
