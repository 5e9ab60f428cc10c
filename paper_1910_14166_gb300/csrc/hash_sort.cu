// hash_sort.cu -- the sketch draw (Sec. 2: bucket h(i) and sign per column of
// S, s independent blocks for an SJLT) and a deterministic, stable counting
// sort of the (block, row) pairs by global bucket.  The sort lets the sketch
// kernel reduce every bucket's rows in ascending row order, the order of the
// streaming definition, with no atomics.
//
// Sort structure (items p in [0, P), keys in [0, m)):
//   count   one CTA per tile of `tile` items: shared-memory histogram -> cnt[tile][m]
//   scan    per bucket, exclusive prefix over tiles (in place) and totals[m]
//   offsets one CTA: exclusive scan of totals -> seg_start[m+1]; chunk_first
//   scatter one warp per tile: ranks among equal keys by __match_any_sync in
//           item order -> perm[seg_start[key] + cnt[tile][key] + rank] = payload
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

SketchKeys make_keys(uint64_t seed, int64_t t, int s, int64_t m) {
  SketchKeys K{};
  uint64_t key_seed = sm64_out(seed, 0);
  uint64_t key_t = sm64_out(key_seed, (uint64_t)t);
  for (int k = 0; k < s && k < kMaxBlocks; ++k) K.key[k] = sm64_out(key_t, (uint64_t)k);
  K.s = s;
  K.mb = (int)(m / s);
  return K;
}

__global__ void k_hash(const SketchKeys K, int64_t n, int32_t* __restrict__ bucket,
                       int8_t* __restrict__ sign) {
  int64_t P = n * K.s;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(p / n);
    int64_t i = p - (int64_t)k * n;
    int row, neg;
    sketch_draw(K, k, (uint64_t)i, row, neg);
    bucket[p] = row;
    sign[p] = neg ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_hash(const SketchKeys& K, int64_t n, int32_t* bucket, int8_t* sign,
                        cudaStream_t st) {
  int64_t P = n * K.s;
  if (P == 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((P + 255) / 256, 152 * 16);
  { k_hash<<<blocks, 256, 0, st>>>(K, n, bucket, sign); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Key sources.
// ---------------------------------------------------------------------------
struct SketchKeySrc {
  SketchKeys K;
  uint32_t n;
  IHS_DEV void get(uint32_t p, int& key, uint32_t& payload) const {
    int k = (int)(p / n);
    uint32_t i = p - (uint32_t)k * n;
    int neg;
    sketch_draw(K, k, i, key, neg);
    payload = i | ((uint32_t)neg << 31);
  }
};
struct ArrayKeySrc {
  const int32_t* keys;
  IHS_DEV void get(uint32_t p, int& key, uint32_t& payload) const {
    key = __ldg(keys + p);
    payload = p;
  }
};

template <class Src>
__global__ void k_sort_count(Src src, uint32_t P, int tile, int m, int32_t* __restrict__ cnt) {
  extern __shared__ int32_t hist[];
  for (int b = threadIdx.x; b < m; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  uint32_t p0 = (uint32_t)blockIdx.x * tile;
  uint32_t p1 = min(P, p0 + (uint32_t)tile);
  for (uint32_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    int key;
    uint32_t pay;
    src.get(p, key, pay);
    atomicAdd(&hist[key], 1);
  }
  __syncthreads();
  int32_t* out = cnt + (int64_t)blockIdx.x * m;
  for (int b = threadIdx.x; b < m; b += blockDim.x) out[b] = hist[b];
}

// Per bucket: exclusive prefix over tiles (in place), totals[b] = sum.
__global__ void k_sort_scan_tiles(int32_t* __restrict__ cnt, int ntiles, int m,
                                  int32_t* __restrict__ totals) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= m) return;
  int32_t run = 0;
  int t = 0;
  for (; t + 4 <= ntiles; t += 4) {
    int32_t c0 = cnt[(int64_t)(t + 0) * m + b];
    int32_t c1 = cnt[(int64_t)(t + 1) * m + b];
    int32_t c2 = cnt[(int64_t)(t + 2) * m + b];
    int32_t c3 = cnt[(int64_t)(t + 3) * m + b];
    cnt[(int64_t)(t + 0) * m + b] = run; run += c0;
    cnt[(int64_t)(t + 1) * m + b] = run; run += c1;
    cnt[(int64_t)(t + 2) * m + b] = run; run += c2;
    cnt[(int64_t)(t + 3) * m + b] = run; run += c3;
  }
  for (; t < ntiles; ++t) {
    int32_t c = cnt[(int64_t)t * m + b];
    cnt[(int64_t)t * m + b] = run;
    run += c;
  }
  totals[b] = run;
}

// One CTA of 1024 threads: seg_start = exclusive scan of totals; then the
// first bucket of every reduce chunk.
__global__ void k_sort_offsets(const int32_t* __restrict__ totals, int m,
                               int32_t* __restrict__ seg_start, int64_t chunk, int nchunks,
                               int32_t* __restrict__ chunk_first) {
  __shared__ int32_t part[1024];
  int per = (m + blockDim.x - 1) / blockDim.x;
  int b0 = threadIdx.x * per, b1 = min(m, b0 + per);
  int32_t s = 0;
  for (int b = b0; b < b1; ++b) s += totals[b];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 partial sums.
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    int32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int b = b0; b < b1; ++b) {
    seg_start[b] = run;
    run += totals[b];
  }
  if (threadIdx.x == blockDim.x - 1) seg_start[m] = part[blockDim.x - 1];
  __syncthreads();
  if (chunk_first == nullptr) return;
  // chunk c starts at item c*chunk; it lies in the bucket b with
  // seg_start[b] <= c*chunk < seg_start[b+1].
  for (int b = b0; b < b1; ++b) {
    int64_t lo = seg_start[b], hi = (b + 1 < b1) ? seg_start[b + 1] : (b + 1 == m ? seg_start[m] : seg_start[b + 1]);
    if (hi <= lo) continue;
    int64_t c0 = (lo + chunk - 1) / chunk, c1 = (hi + chunk - 1) / chunk;
    for (int64_t c = c0; c < c1 && c < nchunks; ++c) chunk_first[c] = b;
  }
}

// One warp per tile: stable ranks among equal keys, in item order.
template <class Src>
__global__ void __launch_bounds__(32) k_sort_scatter(Src src, uint32_t P, int tile, int m,
                                                     const int32_t* __restrict__ cnt,
                                                     const int32_t* __restrict__ seg_start,
                                                     uint32_t* __restrict__ perm) {
  extern __shared__ int32_t run[];
  const int lane = threadIdx.x;
  const int32_t* c = cnt + (int64_t)blockIdx.x * m;
  for (int b = lane; b < m; b += 32) run[b] = seg_start[b] + c[b];
  __syncwarp();
  uint32_t p0 = (uint32_t)blockIdx.x * tile;
  uint32_t p1 = min(P, p0 + (uint32_t)tile);
  const unsigned lt = lanemask_lt();
  for (uint32_t base = p0; base < p1; base += 32) {
    uint32_t p = base + lane;
    bool valid = p < p1;
    int key = -1 - lane;  // unique, never equal to a real key
    uint32_t pay = 0;
    if (valid) src.get(p, key, pay);
    unsigned peers = __match_any_sync(0xffffffffu, key);
    if (valid) {
      int rank = __popc(peers & lt);
      perm[run[key] + rank] = pay;
    }
    __syncwarp();
    if (valid && (peers >> lane) == 1u) run[key] += __popc(peers);  // highest peer updates
    __syncwarp();
  }
}

SortPlan make_sort_plan(int64_t P, int m, int nchunks_target) {
  SortPlan p;
  p.P = P;
  p.m = m;
  // tiles of 4096 items; a small problem (under 152 such tiles) takes tiles
  // of P / 152 rounded up to 256, at least 1024, so that its count and
  // scatter kernels spread over the SMs instead of running a few long warps
  int64_t tile = 4096;
  if (P < 4096 * 152) tile = std::max<int64_t>(1024, (P / 152 + 255) / 256 * 256);
  // keep the tile-count matrix under 16M entries
  while ((P + tile - 1) / tile * (int64_t)m > (16ll << 20)) tile *= 2;
  p.tile = (int)tile;
  p.ntiles = (int)((P + tile - 1) / tile);
  if (p.ntiles < 1) p.ntiles = 1;
  int64_t nc = std::max<int64_t>(1, std::min<int64_t>(nchunks_target, (P + 31) / 32));
  p.chunk = std::max<int64_t>(1, (P + nc - 1) / nc);
  p.nchunks = (int)((P + p.chunk - 1) / p.chunk);
  if (p.nchunks < 1) p.nchunks = 1;
  return p;
}

size_t sort_workspace_bytes(const SortPlan& p) {
  return ((size_t)p.ntiles * p.m + (size_t)p.m + 64) * sizeof(int32_t);
}

template <class Src>
static cudaError_t sort_impl(const SortPlan& p, Src src, void* ws, uint32_t* perm,
                             int32_t* seg_start, int32_t* chunk_first, cudaStream_t st) {
  int32_t* cnt = (int32_t*)ws;
  int32_t* totals = cnt + (size_t)p.ntiles * p.m;
  size_t smem = (size_t)p.m * sizeof(int32_t);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_sort_count<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sort_scatter<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (p.P > 0) {
    { k_sort_count<Src><<<p.ntiles, 256, smem, st>>>(src, (uint32_t)p.P, p.tile, p.m, cnt); note_launches(1); }
    { k_sort_scan_tiles<<<(p.m + 255) / 256, 256, 0, st>>>(cnt, p.ntiles, p.m, totals); note_launches(1); }
  } else {
    cudaMemsetAsync(totals, 0, (size_t)p.m * sizeof(int32_t), st);
  }
  { k_sort_offsets<<<1, 1024, 0, st>>>(totals, p.m, seg_start, p.chunk, p.nchunks, chunk_first); note_launches(1); }
  if (p.P > 0)
    { k_sort_scatter<Src><<<p.ntiles, 32, smem, st>>>(src, (uint32_t)p.P, p.tile, p.m, cnt,
                                                    seg_start, perm); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_sort_sketch(const SortPlan& p, const SketchKeys& K, int64_t n, void* ws,
                               uint32_t* perm, int32_t* seg_start, int32_t* chunk_first,
                               cudaStream_t st) {
  SketchKeySrc src{K, (uint32_t)n};
  return sort_impl(p, src, ws, perm, seg_start, chunk_first, st);
}

cudaError_t launch_sort_keys(const SortPlan& p, const int32_t* keys, void* ws, uint32_t* perm,
                             int32_t* seg_start, cudaStream_t st) {
  ArrayKeySrc src{keys};
  return sort_impl(p, src, ws, perm, seg_start, nullptr, st);
}
