// sketch.cu -- SA = S A for the CountSketch / SJLT of Sec. 2.
//
// Dense A: the (block, row) pairs sorted by bucket (hash_sort.cu) are split
// into equal chunks, one warp per chunk, so every warp streams the same
// number of rows whatever the bucket sizes.  A warp walks the buckets that
// meet its chunk; lanes own interleaved VEC-wide column groups and read each
// row of A with coalesced vector loads (a 2 KB row of a 500-column FP32
// matrix is one 512-byte line per lane group).  Rows of a bucket are added
// in ascending row order -- the order of the streaming definition -- so the
// FP64 result equals a plain sequential loop.  A bucket that straddles
// chunks leaves per-chunk partial rows that a fix-up kernel adds in chunk
// order (deterministic); it also writes the zero rows of empty buckets.
// That split is used for FP32 accumulation (the mixed form); FP64
// accumulation keeps whole buckets per warp (k_sketch_dense_units) so the
// result is bit-identical to the sequential definition.
//
// CSR A: a column-major (CSC) copy is built once at create.  For 2 <= s <= 8
// one CTA of s warps owns a column chunk: each thread loads one entry and
// draws its row once per SJLT block pair (two blocks per SplitMix64 output),
// and warp k keeps block k's m/s accumulators in shared memory
// (k_sketch_csc_cta).  Otherwise one warp owns (column chunk, block k)
// (k_sketch_csc).  Entries arrive in ascending row order.  FP64 accumulators
// add lanes that hit the same bucket in lane (= row) order, so the sums have
// the sequential order; FP32 accumulators use shared-memory atomic adds, in
// a warp-private accumulator (see warp_bucket_add).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>

#include "internal.h"

// ----------------------------------------------------------------------------
// Dense
// ----------------------------------------------------------------------------
template <typename Tin, typename Tacc, int VEC, int NV>
__global__ void __launch_bounds__(256) k_sketch_dense(
    const Tin* __restrict__ A, int64_t lda, int d, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ seg_start, const int32_t* __restrict__ chunk_first, int m,
    int64_t P, int64_t CH, int nchunks, Tacc* __restrict__ SA, Tacc* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nchunks) return;
  const int slab = blockIdx.y;
  const int col_base = slab * (32 * NV * VEC) + lane * VEC;
  const int64_t c0 = (int64_t)w * CH;
  const int64_t c1 = min(P, c0 + CH);

  bool colok[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) colok[q] = (col_base + q * 32 * VEC) < d;

  for (int b = chunk_first[w]; b < m; ++b) {
    const int64_t sb = seg_start[b], eb = seg_start[b + 1];
    if (sb >= c1) break;
    const int64_t lo = max(sb, c0), hi = min(eb, c1);
    if (lo >= hi) continue;
    Tacc acc[NV][VEC];
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[q][v] = Tacc(0);

    for (int64_t base = lo; base < hi; base += 32) {
      const int cnt = (int)min((int64_t)32, hi - base);
      uint32_t my = (lane < cnt) ? __ldg(perm + base + lane) : 0u;
      int j = 0;
      // four rows in flight per step
      for (; j + 4 <= cnt; j += 4) {
        Tin v[4][NV][VEC];
        uint32_t e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          e[u] = __shfl_sync(0xffffffffu, my, j + u);
          const Tin* row = A + (int64_t)(e[u] & 0x7fffffffu) * lda + col_base;
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            if (colok[q]) load_vec_stream<Tin, VEC>(row + q * 32 * VEC, v[u][q]);
            else {
#pragma unroll
              for (int t = 0; t < VEC; ++t) v[u][q][t] = Tin(0);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool neg = (e[u] >> 31) != 0;
#pragma unroll
          for (int q = 0; q < NV; ++q)
#pragma unroll
            for (int t = 0; t < VEC; ++t) {
              Tacc x = (Tacc)v[u][q][t];
              acc[q][t] = neg ? acc[q][t] - x : acc[q][t] + x;
            }
        }
      }
      for (; j < cnt; ++j) {
        uint32_t e = __shfl_sync(0xffffffffu, my, j);
        const Tin* row = A + (int64_t)(e & 0x7fffffffu) * lda + col_base;
        const bool neg = (e >> 31) != 0;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          if (!colok[q]) continue;
          Tin v[VEC];
          load_vec_stream<Tin, VEC>(row + q * 32 * VEC, v);
#pragma unroll
          for (int t = 0; t < VEC; ++t) {
            Tacc x = (Tacc)v[t];
            acc[q][t] = neg ? acc[q][t] - x : acc[q][t] + x;
          }
        }
      }
    }
    // write: whole bucket -> SA row; straddling bucket -> this chunk's slot
    const bool split = (sb / CH) != ((eb - 1) / CH);
    Tacc* dst;
    if (!split) {
      dst = SA + (int64_t)b * d;
    } else {
      const int slot = ((sb / CH) == w && sb != c0) ? 1 : 0;
      dst = partial + ((int64_t)w * 2 + slot) * d;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      if (!colok[q]) continue;
#pragma unroll
      for (int t = 0; t < VEC; ++t) {
        int c = col_base + q * 32 * VEC + t;
        if (c < d) dst[c] = acc[q][t];
      }
    }
  }
}

// One warp per bucket: zero rows for empty buckets, chunk-ordered sums for
// buckets that straddle chunks.
template <typename Tacc>
__global__ void k_sketch_fixup(const int32_t* __restrict__ seg_start, int m, int d, int64_t CH,
                               const Tacc* __restrict__ partial, Tacc* __restrict__ SA) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= m) return;
  const int64_t sb = seg_start[b], eb = seg_start[b + 1];
  Tacc* out = SA + (int64_t)b * d;
  if (sb == eb) {
    for (int c = lane; c < d; c += 32) out[c] = Tacc(0);
    return;
  }
  const int64_t cf = sb / CH, cl = (eb - 1) / CH;
  if (cf == cl) return;
  for (int c = lane; c < d; c += 32) {
    Tacc acc = Tacc(0);
    for (int64_t w = cf; w <= cl; ++w) {
      int slot = (w == cf && sb != w * CH) ? 1 : 0;
      acc += partial[(w * 2 + slot) * d + c];
    }
    out[c] = acc;
  }
}

// FP64 accumulation: work units are (bucket, column slab), handed out by an
// atomic counter, so every bucket is summed by one warp in ascending row
// order -- the exact order of the streaming definition, hence bit-identical
// FP64 results -- while column slabs keep units small enough to balance.
template <typename Tin, int VEC>
__global__ void __launch_bounds__(256) k_sketch_dense_units(
    const Tin* __restrict__ A, int64_t lda, int d, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ seg_start, int m, int nslabs, int* __restrict__ counter,
    double* __restrict__ SA) {
  const int lane = threadIdx.x & 31;
  const int64_t units = (int64_t)m * nslabs;
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= units) break;
    const int b = u / nslabs, slab = u - (u / nslabs) * nslabs;
    const int col = slab * 32 * VEC + lane * VEC;
    const bool ok = col < d;
    double acc[VEC];
#pragma unroll
    for (int t = 0; t < VEC; ++t) acc[t] = 0.0;
    const int64_t lo = seg_start[b], hi = seg_start[b + 1];
    for (int64_t base = lo; base < hi; base += 32) {
      const int cnt = (int)min((int64_t)32, hi - base);
      const uint32_t my = (lane < cnt) ? __ldg(perm + base + lane) : 0u;
      int j = 0;
      for (; j + 4 <= cnt; j += 4) {
        Tin v[4][VEC];
        uint32_t e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          e[q] = __shfl_sync(0xffffffffu, my, j + q);
          if (ok) load_vec_stream<Tin, VEC>(A + (int64_t)(e[q] & 0x7fffffffu) * lda + col, v[q]);
          else {
#pragma unroll
            for (int t = 0; t < VEC; ++t) v[q][t] = Tin(0);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool neg = (e[q] >> 31) != 0;
#pragma unroll
          for (int t = 0; t < VEC; ++t) {
            const double x = (double)v[q][t];
            acc[t] = neg ? acc[t] - x : acc[t] + x;
          }
        }
      }
      for (; j < cnt; ++j) {
        const uint32_t e = __shfl_sync(0xffffffffu, my, j);
        if (!ok) continue;
        Tin v[VEC];
        load_vec_stream<Tin, VEC>(A + (int64_t)(e & 0x7fffffffu) * lda + col, v);
        const bool neg = (e >> 31) != 0;
#pragma unroll
        for (int t = 0; t < VEC; ++t) {
          const double x = (double)v[t];
          acc[t] = neg ? acc[t] - x : acc[t] + x;
        }
      }
    }
    if (ok) {
      double* dst = SA + (int64_t)b * d + col;
#pragma unroll
      for (int t = 0; t < VEC; ++t)
        if (col + t < d) dst[t] = acc[t];
    }
  }
}

template <typename Tin, int VEC>
static cudaError_t run_dense_units(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                                   const int32_t* seg, int* counter, void* SA, int sms,
                                   cudaStream_t st) {
  const int nslabs = (int)((A.d + 32 * VEC - 1) / (32 * VEC));
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  { k_sketch_dense_units<Tin, VEC><<<sms * 8, 256, 0, st>>>((const Tin*)A.val, A.ld, (int)A.d,
                                                          perm, seg, p.m, nslabs, counter,
                                                          (double*)SA); note_launches(1); }
  return cudaGetLastError();
}

template <typename Tin, typename Tacc, int VEC, int NV>
static cudaError_t run_dense(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                             const int32_t* seg, const int32_t* cf, void* SA, void* partial,
                             cudaStream_t st, void* prof) {
  const int per_slab = 32 * NV * VEC;
  dim3 grid((p.nchunks + 7) / 8, (unsigned)((A.d + per_slab - 1) / per_slab));
  { k_sketch_dense<Tin, Tacc, VEC, NV><<<grid, 256, 0, st>>>(
      (const Tin*)A.val, A.ld, (int)A.d, perm, seg, cf, p.m, p.P, p.chunk, p.nchunks,
      (Tacc*)SA, (Tacc*)partial); note_launches(1); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_stage_end(prof);
  prof_stage_begin(prof, IHS_ST_SKETCH_FIX);
  { k_sketch_fixup<Tacc><<<(p.m + 7) / 8, 256, 0, st>>>(seg, p.m, (int)A.d, p.chunk,
                                                      (const Tacc*)partial, (Tacc*)SA); note_launches(1); }
  return cudaGetLastError();
}

template <typename Tin, typename Tacc, int VEC>
static cudaError_t dense_nv(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                            const int32_t* seg, const int32_t* cf, void* SA, void* partial,
                            cudaStream_t st, void* prof) {
  const int64_t groups = (A.d + VEC - 1) / VEC;  // vector groups per row
  if (groups <= 32) return run_dense<Tin, Tacc, VEC, 1>(A, p, perm, seg, cf, SA, partial, st, prof);
  if (groups <= 64) return run_dense<Tin, Tacc, VEC, 2>(A, p, perm, seg, cf, SA, partial, st, prof);
  return run_dense<Tin, Tacc, VEC, 4>(A, p, perm, seg, cf, SA, partial, st, prof);  // + slabs
}

cudaError_t launch_sketch_dense(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                                const int32_t* seg, const int32_t* cf, int acc64, void* SA,
                                void* partial, int* counter, int sms, cudaStream_t st,
                                void* prof) {
  const uintptr_t base = (uintptr_t)A.val;
  if (acc64) {
    if (A.f32) {
      const bool v4 = (A.ld % 4 == 0) && (A.d % 4 == 0) && (base % 16 == 0);
      return v4 ? run_dense_units<float, 4>(A, p, perm, seg, counter, SA, sms, st)
                : run_dense_units<float, 1>(A, p, perm, seg, counter, SA, sms, st);
    }
    const bool v2 = (A.ld % 2 == 0) && (A.d % 2 == 0) && (base % 16 == 0);
    return v2 ? run_dense_units<double, 2>(A, p, perm, seg, counter, SA, sms, st)
              : run_dense_units<double, 1>(A, p, perm, seg, counter, SA, sms, st);
  }
  if (A.f32) {
    const bool v4 = (A.ld % 4 == 0) && (A.d % 4 == 0) && (base % 16 == 0);
    return v4 ? dense_nv<float, float, 4>(A, p, perm, seg, cf, SA, partial, st, prof)
              : dense_nv<float, float, 1>(A, p, perm, seg, cf, SA, partial, st, prof);
  }
  const bool v2 = (A.ld % 2 == 0) && (A.d % 2 == 0) && (base % 16 == 0);
  return v2 ? dense_nv<double, float, 2>(A, p, perm, seg, cf, SA, partial, st, prof)
            : dense_nv<double, float, 1>(A, p, perm, seg, cf, SA, partial, st, prof);
}

// ----------------------------------------------------------------------------
// CSR through the CSC copy
// ----------------------------------------------------------------------------
// Adds v into bucket `key` of a warp-private shared-memory accumulator for
// every valid lane.  Invalid lanes pass a key distinct from every valid key
// (-1 - lane) and touch nothing.  Three modes:
// 2 (FP32 accumulators): one shared-memory atomic add a lane.  Lanes of one
//   batch that share a bucket add in the order the hardware serialises them
//   (within the FP32 summation bound, which holds for any order); batches
//   still add in entry order, and the accumulator is private to the warp.
// Modes 1 and 0 (FP64, whose sums follow the entries' order exactly, as the
// oracle's do) add lanes that share a bucket in lane order:
// 1: one 32-bit claim word a bucket (32 = free).  In rounds, each pending
//   lane claims its bucket with a shared-memory atomicMin of its index; the
//   lowest pending lane of each bucket wins, adds, frees the word and leaves.
//   A batch without collision takes one round; each extra entry in one
//   bucket, one more.
// 0: byte tags.  Every valid lane writes its index at its bucket's tag byte and
//   reads it back; a lane that reads another index shares its bucket.
//   Whichever write survives, the test is exact.  Without a collision the
//   lanes add at once; otherwise the warp matches keys (a narrow pipe, so
//   only for batches that collide) and adds one rank per round.
template <typename Tacc, int MODE>
IHS_DEV void warp_bucket_add(Tacc* acc, uint8_t* tag, uint32_t* tag32, int key, Tacc v,
                             bool valid, int lane, unsigned lt) {
  if constexpr (MODE == 2) {
    if (valid) atomicAdd(acc + key, v);
  } else if constexpr (MODE == 1) {
    bool pending = valid;
    while (__any_sync(0xffffffffu, pending)) {
      if (pending) atomicMin(tag32 + key, (uint32_t)lane);
      __syncwarp();
      const bool win = pending && tag32[key] == (uint32_t)lane;
      __syncwarp();
      if (win) {
        acc[key] += v;
        tag32[key] = 32u;
        pending = false;
      }
      __syncwarp();
    }
  } else {
    if (valid) tag[key] = (uint8_t)lane;
    __syncwarp();
    const bool clash = valid && tag[key] != (uint8_t)lane;
    if (!__any_sync(0xffffffffu, clash)) {
      if (valid) acc[key] += v;
    } else {
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int rank = __popc(peers & lt);
      const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(peers));
      for (int r = 0; r < rounds; ++r) {
        if (valid && rank == r) acc[key] += v;
        __syncwarp();
      }
    }
    __syncwarp();
  }
}

template <typename Tin, typename Tacc, int MODE>
__global__ void __launch_bounds__(256) k_sketch_csc(
    const int32_t* __restrict__ rowidx, const Tin* __restrict__ val, int nitems,
    const int32_t* __restrict__ item_col, const int64_t* __restrict__ item_begin,
    const int64_t* __restrict__ item_end, const int32_t* __restrict__ item_slot,
    const SketchKeys K, int d, Tacc* __restrict__ SA, Tacc* __restrict__ partial) {
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int mb = K.mb;
  Tacc* acc = reinterpret_cast<Tacc*>(smem_raw) + (size_t)wib * mb;
  // after the nw accumulators: one byte per bucket to detect colliding lanes
  // (mode 0), or one 32-bit word per bucket holding the lowest lane that
  // claimed it (mode 1; 32: none); none in mode 2
  uint8_t* tag = reinterpret_cast<uint8_t*>(reinterpret_cast<Tacc*>(smem_raw) + (size_t)nw * mb) +
                 (size_t)wib * mb;
  uint32_t* tag32 = reinterpret_cast<uint32_t*>(reinterpret_cast<Tacc*>(smem_raw) + (size_t)nw * mb) +
                    (size_t)wib * mb;
  // work unit = (item, block k)
  const int64_t unit = (int64_t)blockIdx.x * nw + wib;
  if (unit >= (int64_t)nitems * K.s) return;
  const int it = (int)(unit / K.s);
  const int k = (int)(unit - (int64_t)it * K.s);
  for (int b = lane; b < mb; b += 32) {
    acc[b] = Tacc(0);
    if constexpr (MODE == 1) tag32[b] = 32u;
  }
  __syncwarp();
  const int64_t e0 = item_begin[it], e1 = item_end[it];
  const unsigned lt = lanemask_lt();
  // four batches of 32 entries per pass: all eight loads are issued before
  // the first hash, so each warp keeps several L2 round trips in flight.
  // Batches are still accumulated in entry order, and colliding lanes of a
  // batch in lane order.
  constexpr int kU = 4;
  for (int64_t base = e0; base < e1; base += 32 * kU) {
    uint32_t rq[kU];
    Tin xq[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int64_t e = base + q * 32 + lane;
      rq[q] = 0u;
      xq[q] = Tin(0);
      if (e < e1) {
        rq[q] = (uint32_t)__ldg(rowidx + e);
        xq[q] = __ldg(val + e);
      }
    }
    // the draws of all kU batches first: independent hash chains the
    // scheduler interleaves, before the scatters, which synchronise the warp
    int keyq[kU];
    Tacc vq[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      int row, neg;
      sketch_draw(K, k, (uint64_t)rq[q], row, neg);
      keyq[q] = row - k * mb;
      vq[q] = neg ? -(Tacc)xq[q] : (Tacc)xq[q];
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const bool valid = base + q * 32 + lane < e1;
      warp_bucket_add<Tacc, MODE>(acc, tag, tag32, valid ? keyq[q] : -1 - lane,
                                    valid ? vq[q] : Tacc(0), valid, lane, lt);
    }
  }
  // write block k's rows of column item_col[it]
  const int j = item_col[it];
  const int slot = item_slot[it];
  if (slot < 0) {
    for (int b = lane; b < mb; b += 32) SA[(int64_t)(k * mb + b) * d + j] = acc[b];
  } else {
    Tacc* dst = partial + ((int64_t)slot * K.s + k) * mb;
    for (int b = lane; b < mb; b += 32) dst[b] = acc[b];
  }
}

// Columns with several items: sum the items' partial columns in item order.
template <typename Tacc>
__global__ void k_sketch_csc_merge(const int32_t* __restrict__ col_first_item,
                                   const int32_t* __restrict__ item_slot, int d, int m, int s,
                                   int mb, const Tacc* __restrict__ partial,
                                   Tacc* __restrict__ SA) {
  const int j = blockIdx.y;
  const int i0 = col_first_item[j], i1 = col_first_item[j + 1];
  if (i1 - i0 <= 1) return;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const int k = r / mb, b = r - k * mb;
    Tacc acc = Tacc(0);
    for (int it = i0; it < i1; ++it) acc += partial[((int64_t)item_slot[it] * s + k) * mb + b];
    SA[(int64_t)r * d + j] = acc;
  }
}

template <typename Tacc>
static cudaError_t merge_csc(const CscA& A, const SketchKeys& K, int64_t m, void* SA,
                             const void* partial, cudaStream_t st) {
  if (A.nsplit_slots == 0) return cudaSuccess;
  dim3 g((unsigned)std::min<int64_t>((m + 255) / 256, 64), (unsigned)A.d);
  { k_sketch_csc_merge<Tacc><<<g, 256, 0, st>>>(A.col_first_item, A.item_slot, (int)A.d, (int)m,
                                              K.s, K.mb, (const Tacc*)partial, (Tacc*)SA); note_launches(1); }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// CSC sketch, one CTA per column chunk (2 <= s <= 8, m / s <= 32768).
// A CTA of s warps takes one column chunk.  Per batch of 32 s entries every
// thread loads one entry (row id and value, read once rather than once per
// block), makes its row's ceil(s / 2) pair draws (two blocks per SplitMix64
// output, see sketch_draw) and stages the value and the s codes (bucket
// within block k | sign << 15) in shared memory.  Warp k then adds the batch
// into block k's accumulator in entry order, lanes that share a bucket as
// warp_bucket_add describes, so each bucket's sum has the same order as in
// the one-warp-per-block kernel.  The next batch's row ids and values are
// loaded before the current batch is added.
// ----------------------------------------------------------------------------
// Shared-memory layout: s accumulators of mb buckets, the batch's values,
// s tag arrays, the batch's codes ([s][32 s]).
struct CscCtaLayout {
  int off_val, off_tag, off_code, bytes;
};
static CscCtaLayout csc_cta_layout(int s, int mb, int accb, int inb, int tagb) {
  auto up = [](int64_t v) { return (int)((v + 15) & ~int64_t(15)); };
  CscCtaLayout L;
  L.off_val = up((int64_t)s * mb * accb);
  L.off_tag = L.off_val + up((int64_t)32 * s * inb);
  L.off_code = L.off_tag + up((int64_t)s * mb * tagb);
  L.bytes = L.off_code + up((int64_t)32 * s * s * 2);
  return L;
}

template <typename Tin, typename Tacc, int MODE>
__global__ void __launch_bounds__(256) k_sketch_csc_cta(
    const int32_t* __restrict__ rowidx, const Tin* __restrict__ val,
    const int32_t* __restrict__ item_col, const int64_t* __restrict__ item_begin,
    const int64_t* __restrict__ item_end, const int32_t* __restrict__ item_slot,
    const SketchKeys K, int d, CscCtaLayout L, Tacc* __restrict__ SA,
    Tacc* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = K.s, mb = K.mb;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int k = tid >> 5;    // this warp's block
  const int B = blockDim.x;  // entries a batch: one per thread
  const int it = blockIdx.x;
  Tacc* acc = reinterpret_cast<Tacc*>(smem_raw) + (size_t)k * mb;
  Tin* vals = reinterpret_cast<Tin*>(smem_raw + L.off_val);
  uint8_t* tag = smem_raw + L.off_tag + (size_t)k * mb;
  uint32_t* tag32 = reinterpret_cast<uint32_t*>(smem_raw + L.off_tag) + (size_t)k * mb;
  uint16_t* codes = reinterpret_cast<uint16_t*>(smem_raw + L.off_code);
  for (int b = lane; b < mb; b += 32) {
    acc[b] = Tacc(0);
    if constexpr (MODE == 1) tag32[b] = 32u;
  }
  const int64_t e0 = item_begin[it], e1 = item_end[it];
  const unsigned lt = lanemask_lt();
  uint32_t r = 0u;
  Tin x = Tin(0);
  if (e0 + tid < e1) {
    r = (uint32_t)__ldg(rowidx + e0 + tid);
    x = __ldg(val + e0 + tid);
  }
  for (int64_t base = e0; base < e1; base += B) {
    vals[tid] = x;
#pragma unroll
    {
      // out(key_p, r) = mix(key_p + (r + 1) gamma): the counter term once
      const uint64_t ig = ((uint64_t)r + 1) * kSmGamma;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        if (2 * p < s) {
          const uint64_t w = sm64_finalise(K.key[p] + ig);
          const uint32_t hi = (uint32_t)(w >> 32), lo = (uint32_t)w;
          codes[(2 * p) * B + tid] = (uint16_t)((uint32_t)draw_bucket(hi, mb) | ((lo & 1u) << 15));
          if (2 * p + 1 < s)
            codes[(2 * p + 1) * B + tid] =
                (uint16_t)((uint32_t)draw_bucket(lo, mb) | ((hi & 1u) << 15));
        }
      }
    }
    __syncthreads();
    {  // the next batch's row ids and values
      const int64_t e = base + B + tid;
      if (e < e1) {
        r = (uint32_t)__ldg(rowidx + e);
        x = __ldg(val + e);
      }
    }
    // block k over this batch, 32 entries at a time in entry order
    const int nbt = (int)((e1 - base < (int64_t)B) ? (e1 - base) : (int64_t)B);
    const uint16_t* ck = codes + k * B;
    if constexpr (MODE == 2 && sizeof(Tin) == 4) {
      if (nbt == B) {  // a full batch: every lane valid, sign as a sign-bit flip
        for (int q = lane; q < B; q += 32) {
          const uint32_t c = ck[q];
          const float v = __uint_as_float(__float_as_uint((float)vals[q]) ^ ((c & 0x8000u) << 16));
          atomicAdd(reinterpret_cast<float*>(acc) + (c & 0x7fffu), v);
        }
        __syncthreads();
        continue;
      }
    }
    for (int q = 0; q < nbt; q += 32) {
      const int idx = q + lane;
      const bool valid = idx < nbt;
      const uint32_t c = valid ? (uint32_t)ck[idx] : 0u;
      const Tin xv = valid ? vals[idx] : Tin(0);
      const Tacc v = (c & 0x8000u) ? -(Tacc)xv : (Tacc)xv;
      warp_bucket_add<Tacc, MODE>(acc, tag, tag32, valid ? (int)(c & 0x7fffu) : -1 - lane, v,
                                  valid, lane, lt);
    }
    __syncthreads();
  }
  __syncwarp();
  const int j = item_col[it];
  const int slot = item_slot[it];
  if (slot < 0) {
    for (int b = lane; b < mb; b += 32) SA[(int64_t)(k * mb + b) * d + j] = acc[b];
  } else {
    Tacc* dst = partial + ((int64_t)slot * s + k) * mb;
    for (int b = lane; b < mb; b += 32) dst[b] = acc[b];
  }
}

template <typename Tin, typename Tacc, int MODE>
static cudaError_t launch_csc_cta(const CscA& A, const SketchKeys& K, const CscCtaLayout& L,
                                  cudaStream_t st, void* SA, void* partial) {
  cudaError_t e = cudaSuccess;
  if (L.bytes > 48 * 1024 &&
      (e = ensure_smem((const void*)k_sketch_csc_cta<Tin, Tacc, MODE>, L.bytes)) != cudaSuccess)
    return e;
  if (A.nitems == 0) return cudaSuccess;
  k_sketch_csc_cta<Tin, Tacc, MODE><<<A.nitems, 32 * K.s, L.bytes, st>>>(
      A.rowidx, (const Tin*)A.val, A.item_col, A.item_begin, A.item_end, A.item_slot, K, (int)A.d,
      L, (Tacc*)SA, (Tacc*)partial);
  note_launches(1);
  return cudaGetLastError();
}

template <typename Tin, typename Tacc, int MODE>
static cudaError_t launch_csc_warp(const CscA& A, const SketchKeys& K, int nw, size_t smem,
                                   cudaStream_t st, void* SA, void* partial) {
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024 &&
      (e = ensure_smem((const void*)k_sketch_csc<Tin, Tacc, MODE>, (int)smem)) != cudaSuccess)
    return e;
  const int64_t units = (int64_t)A.nitems * K.s;
  const unsigned grid = (unsigned)((units + nw - 1) / nw);
  k_sketch_csc<Tin, Tacc, MODE><<<grid, nw * 32, smem, st>>>(
      A.rowidx, (const Tin*)A.val, A.nitems, A.item_col, A.item_begin, A.item_end, A.item_slot, K,
      (int)A.d, (Tacc*)SA, (Tacc*)partial);
  note_launches(1);
  return cudaGetLastError();
}

template <typename Tin, typename Tacc>
static cudaError_t run_csc(const CscA& A, const SketchKeys& K, int64_t m, void* SA, void* partial,
                           cudaStream_t st) {
  // Scatter mode.  FP32 accumulators: shared-memory atomic adds (measured on
  // 1250 FP32 buckets a block: 1.03 ms against 1.38 ms with byte tags).
  // FP64 (whose sums must follow the entries' order): 32-bit claim words
  // when a CTA of eight warps' accumulators and words stays within 56 KB
  // (four CTAs an SM), the byte tags otherwise, where the claim words would
  // cost occupancy (500 FP64 buckets a block: 0.118 ms with claim words
  // against 0.152 ms with byte tags).
  auto tagb = [](int mode) { return mode == 1 ? 4 : (mode == 0 ? 1 : 0); };
  // 2 <= s <= 8: one CTA per column chunk (each entry read once and its row
  // drawn once per block pair; measured on 10,000,000 x 1000 with s = 8 and
  // 1250 FP32 buckets a block: 0.90 ms against 1.17 ms for one warp per
  // block, which draws a whole pair per entry and block)
  if (K.s >= 2 && K.s <= 8 && K.mb <= 32768) {
    const int accb = (int)sizeof(Tacc), inb = (int)sizeof(Tin);
    const int cmode = std::is_same<Tacc, float>::value
                          ? 2
                          : (csc_cta_layout(K.s, K.mb, accb, inb, 4).bytes <= 56 * 1024 ? 1 : 0);
    const CscCtaLayout L = csc_cta_layout(K.s, K.mb, accb, inb, tagb(cmode));
    if (L.bytes <= 200 * 1024) {
      cudaError_t e = cudaSuccess;
      if constexpr (std::is_same<Tacc, float>::value) {
        e = launch_csc_cta<Tin, Tacc, 2>(A, K, L, st, SA, partial);
      } else {
        e = cmode == 1 ? launch_csc_cta<Tin, Tacc, 1>(A, K, L, st, SA, partial)
                       : launch_csc_cta<Tin, Tacc, 0>(A, K, L, st, SA, partial);
      }
      if (e != cudaSuccess) return e;
      return merge_csc<Tacc>(A, K, m, SA, partial, st);
    }
  }
  const int mode = std::is_same<Tacc, float>::value
                       ? 2
                       : ((size_t)K.mb * (sizeof(Tacc) + 4) * 8 <= 56 * 1024 ? 1 : 0);
  const size_t per_warp = (size_t)K.mb * (sizeof(Tacc) + tagb(mode));
  const int nw = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
  if (nw < 1) return cudaErrorInvalidValue;
  const size_t smem = per_warp * nw;
  cudaError_t e = cudaSuccess;
  if constexpr (std::is_same<Tacc, float>::value) {
    e = launch_csc_warp<Tin, Tacc, 2>(A, K, nw, smem, st, SA, partial);
  } else {
    e = mode == 1 ? launch_csc_warp<Tin, Tacc, 1>(A, K, nw, smem, st, SA, partial)
                  : launch_csc_warp<Tin, Tacc, 0>(A, K, nw, smem, st, SA, partial);
  }
  if (e != cudaSuccess) return e;
  return merge_csc<Tacc>(A, K, m, SA, partial, st);
}

cudaError_t launch_sketch_csc(const CscA& A, const SketchKeys& K, int64_t m, int acc64, void* SA,
                              void* partial, cudaStream_t st) {
  if (A.f32) {
    return acc64 ? run_csc<float, double>(A, K, m, SA, partial, st)
                 : run_csc<float, float>(A, K, m, SA, partial, st);
  }
  return acc64 ? run_csc<double, double>(A, K, m, SA, partial, st)
               : run_csc<double, float>(A, K, m, SA, partial, st);
}

// ----------------------------------------------------------------------------
// Adjoint: (S^T G)_i = sum_k sign_k(i) G[bucket_k(i), :] / sqrt(s); one warp per row.
// ----------------------------------------------------------------------------
__global__ void k_sketch_adjoint(const SketchKeys K, int64_t n, int d, double inv_sqrt_s,
                                 const double* __restrict__ G, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  int rows[kMaxBlocks];
  double sg[kMaxBlocks];
  for (int k = 0; k < K.s; ++k) {
    int neg;
    sketch_draw(K, k, (uint64_t)i, rows[k], neg);
    sg[k] = neg ? -inv_sqrt_s : inv_sqrt_s;
  }
  for (int c = lane; c < d; c += 32) {
    double acc = 0.0;
    for (int k = 0; k < K.s; ++k) acc += sg[k] * __ldg(G + (int64_t)rows[k] * d + c);
    out[i * d + c] = acc;
  }
}

cudaError_t launch_sketch_adjoint(const SketchKeys& K, int64_t n, int64_t d, const double* G,
                                  double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  { k_sketch_adjoint<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(K, n, (int)d,
                                                           1.0 / std::sqrt((double)K.s), G,
                                                           out); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_sketch_fixup_f32(const SortPlan& p, const int32_t* seg, int d,
                                    const float* partial, float* SA, cudaStream_t st) {
  k_sketch_fixup<float><<<(p.m + 7) / 8, 256, 0, st>>>(seg, p.m, d, p.chunk, partial, SA);
  note_launches(1);
  return cudaGetLastError();
}
