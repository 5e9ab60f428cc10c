// linalg.cu -- the d x d step of Eq. 2 for OLS / ridge: Cholesky H = L L^T
// and x^{t+1} = x^t + L^{-T} L^{-1} g.
//
// Factor: one cooperative, persistent launch (all CTAs co-resident) doing a
// blocked Cholesky on 32 x 32 tiles with a look-ahead schedule: between grid
// barriers k-1 and k the CTAs share out, as one list of independent items,
//   panel(k)   tile rows k..Tt-1 of column k.  Each such item first applies
//              the rank-32 update of step k-1 to its own tiles, factors the
//              32 x 32 diagonal tile itself (redundantly, which saves a
//              barrier) and solves x L_kk^T = a for its tile in the same
//              register sweep; the result also goes, transposed, into
//              the unused upper triangle, tile (k, i);
//   update(k-1) every trailing lower tile (i, j), k < j <= i:
//              A_ij -= L_{i,k-1} L_{j,k-1}^T,
// so a step costs one grid barrier (FP32; in FP64, where a tile update is
// slow, k_chol_coop2 takes two barriers a step and spreads the updates over
// the grid).  The item that owns the diagonal tile
// sweeps the identity alongside it, which yields D_k = L_kk^{-1} for the
// solve in the same 32 steps; L_kk itself is never written back (every panel
// item of step k reads the diagonal tile while the step runs, and the solve
// uses D_k only), so the diagonal tiles of L keep the updated H.  Tiles are
// padded with the identity so any d works.  The factor runs in FP64 (plain
// form) or FP32 (mixed form: there the Hessian already carries TF32/BF16
// input rounding, so the factor only has to be a good preconditioner; the
// iterate update x += delta stays FP64).  A pivot that is not positive
// records DEV_NOT_SPD; a barrier wait that exceeds its spin budget records
// DEV_TIMEOUT and every CTA returns.
//
// Solve: one CTA, left-looking by tiles.  Forward: warp w forms row k0+w of
// L times the solved part of y with coalesced row reads, then y_k = D_k t_k.
// Backward: the same on the stored transpose, z_k = D_k^T t_k.
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "internal.h"

int chol_padded(int d) { return (d + 31) / 32 * 32; }
size_t chol_dinv_bytes(int d, int f32) {
  return (size_t)(chol_padded(d) / 32) * 1024 * (f32 ? 4 : 8);
}

template <typename T>
__global__ void k_chol_init(const double* __restrict__ H, int d, int dp, double shift,
                            T* __restrict__ L) {
  const int64_t total = (int64_t)dp * dp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / dp), j = (int)(e - (int64_t)i * dp);
    T v;
    if (i < d && j < d) v = (T)(H[(int64_t)i * d + j] + (i == j ? shift : 0.0));
    else v = (i == j) ? T(1) : T(0);
    L[e] = v;
  }
}

// Grid-wide barrier (generation counter), bounded spin.  bar[0] = arrivals,
// bar[1] = generation, bar[2] = abort flag; all zero before the launch.
IHS_DEV bool grid_barrier(unsigned* bar, unsigned nblocks, int* status,
                          long long limit = kSpinLimit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    volatile unsigned* abort_flag = bar + 2;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      *(volatile unsigned*)bar = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > limit || *abort_flag) {
          set_status(status, DEV_TIMEOUT);
          *abort_flag = 1u;
          ok = 0;
          break;
        }
        if (it > 2048) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Self-test of the bounded wait: a barrier that expects one CTA more than
// are launched can never complete, so every CTA must give up after `limit`
// polls, record DEV_TIMEOUT and return.
__global__ void k_barrier_selftest(unsigned* bar, int* status, long long limit) {
  grid_barrier(bar, gridDim.x + 1, status, limit);
}

cudaError_t launch_barrier_selftest(unsigned* bar, int* status, cudaStream_t st) {
  k_barrier_selftest<<<2, 32, 0, st>>>(bar, status, 4096);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void k_selftest_rsqrt(const double* __restrict__ p, double* __restrict__ out,
                                 double* __restrict__ ref, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = rsqrt_nr(p[i]);
    ref[i] = rsqrt(p[i]);
  }
}

cudaError_t launch_selftest_rsqrt(const double* p, double* out, double* ref, int64_t n,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  { k_selftest_rsqrt<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(p, out, ref, n); note_launches(1); }
  return cudaGetLastError();
}

// Reciprocal square root of a pivot: FP32 through the hardware's rsqrtf,
// FP64 through rsqrt_nr (six dependent FP64 operations on the pivot chain).
IHS_DEV float pivot_rsqrt(float p) { return rsqrtf(p); }
IHS_DEV double pivot_rsqrt(double p) { return rsqrt_nr(p); }

// Panel sweep with warp 0 over the tall block [Dk; Ta] (Ta optional): lane r
// holds row r of the diagonal tile and row r of the panel tile in registers.
// Column j: the pivot comes from lane j by a shuffle, the diagonal rows below
// and every panel row are scaled by 1/L_jj, and the trailing columns of both
// are updated with L_cj fetched from lane c.  This factors Dk = L_kk L_kk^T
// and solves Ta <- Ta L_kk^{-T} in the same 32 steps, with no block-wide
// barrier inside.  Only the first ncols columns are swept: in the last tile
// the columns past d are identity padding (pivot 1, and every L entry that
// would update them is 0), so they end as they start.  All threads of the
// CTA must call.
template <typename T>
__device__ void panel_sweep(T (*Dk)[33], T (*Ta)[33], bool tall, int* spd, int ncols) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    T a[32], bb[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      a[c] = (c <= lane) ? Dk[lane][c] : T(0);
      bb[c] = tall ? Ta[lane][c] : T(0);
    }
    bool good = true;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= ncols) break;  // identity padding past d: nothing to do
      T pj = __shfl_sync(0xffffffffu, a[j], j);
      if (!(pj > T(0))) {
        good = false;
        pj = T(1);
      }
      const T rinv = pivot_rsqrt(pj);
      const T lrj = (lane > j) ? a[j] * rinv : (lane == j ? pj * rinv : T(0));
      a[j] = lrj;
      const T bj = bb[j] * rinv;
      bb[j] = bj;
#pragma unroll
      for (int c = 1; c < 32; ++c) {
        if (c > j) {
          const T lcj = __shfl_sync(0xffffffffu, lrj, c);
          if (lane >= c) a[c] -= lrj * lcj;
          bb[c] -= bj * lcj;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      Dk[lane][c] = a[c];
      if (tall) Ta[lane][c] = bb[c];
    }
    if (lane == 0) *spd = good ? 1 : 0;
  }
  __syncthreads();
}

// The same sweep spread over warps 0-3 (128 threads), for FP64, where the
// per-column updates dominate: GB300 issues about one FP64 warp instruction
// per 64 cycles on each sub-partition, so a one-warp sweep of a 32-column
// tile (about a thousand DFMA instructions) takes tens of microseconds.
// Lane r still owns row r; warp w owns the columns c = w (mod 4), eight of
// the diagonal block and eight of the panel block, so the four sub-partitions
// share the updates.  Column j is published by its owner warp (j mod 4): the
// scaled column L_rj and the scaled panel entries go to shared-memory slot j
// and each lane arrives on mbarrier j (32 arrivals complete it); a warp that
// needs column j waits on that mbarrier alone, so it is never held up by
// another warp's unfinished updates.  Each warp copies column j to registers,
// then the owner of column j + 1 applies column j's update to column j + 1
// first and publishes column j + 1 at once, before its other updates: the
// pivot chain runs from one column to the next without waiting for the rest
// of the rank-1 update.  Waits are bounded (kSpinLimit polls); one that runs
// out marks the sweep as timed out and the warp goes on, so no wait can hang
// the CTA.  Every entry goes through the same operations in the same order
// as in panel_sweep, so both give the same factor; columns from ncols on are
// skipped as there.  *spd: 1, 0 if a pivot was not positive, -1 if a wait
// timed out.  All threads must call.
template <typename T>
__device__ void panel_sweep4(T (*Dk)[33], T (*Ta)[33], bool tall, int* spd, int ncols) {
  __shared__ T colL[32][32], colB[32][32];
  __shared__ __align__(8) uint64_t ready[32];
  __shared__ int bad, late;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    bad = 0;
    late = 0;
    for (int j = 0; j < 32; ++j) mbar_init(&ready[j], 32);
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    T a[8], bb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = w + 4 * u;
      a[u] = (c <= lane) ? Dk[lane][c] : T(0);
      bb[u] = tall ? Ta[lane][c] : T(0);
    }
    // the owner's publication of column j (a[j >> 2], bb[j >> 2] final)
    auto publish = [&](const int j) {
      const int uj = j >> 2;
      T pj = __shfl_sync(0xffffffffu, a[uj], j);
      if (!(pj > T(0))) {
        if (lane == 0) bad = 1;
        pj = T(1);
      }
      const T rinv = pivot_rsqrt(pj);
      const T lrj = (lane > j) ? a[uj] * rinv : (lane == j ? pj * rinv : T(0));
      a[uj] = lrj;
      const T bj = bb[uj] * rinv;
      bb[uj] = bj;
      colL[j][lane] = lrj;
      colB[j][lane] = bj;
      __syncwarp();
      mbar_arrive(&ready[j]);
    };
    if (w == 0) publish(0);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= ncols) break;  // identity padding past d: nothing to do
      if (w != (j & 3)) {
        long long it = 0;
        while (!mbar_try_wait(&ready[j], 0)) {
          if (++it > kSpinLimit) {
            late = 1;
            break;
          }
        }
      }
      const T lrj = colL[j][lane], bj = colB[j][lane];
      T lc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) lc[u] = colL[j][w + 4 * u];
      const int jn = j + 1;
      const bool next = jn < ncols && w == (jn & 3);
      if (next) {
        const int un = jn >> 2;
        if (lane >= jn) a[un] -= lrj * lc[un];
        bb[un] -= bj * lc[un];
        publish(jn);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = w + 4 * u;
        if (c > j && !(next && c == jn)) {
          if (lane >= c) a[u] -= lrj * lc[u];
          bb[u] -= bj * lc[u];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = w + 4 * u;
      Dk[lane][c] = a[u];
      if (tall) Ta[lane][c] = bb[u];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *spd = late ? -1 : (bad ? 0 : 1);
    for (int j = 0; j < 32; ++j) mbar_inval(&ready[j]);
  }
  __syncthreads();
}

// Records a sweep's outcome: a pivot that was not positive (reported by the
// item of the diagonal tile) or a wait that ran out (any item).
IHS_DEV void note_sweep(int spd, bool diag, int* status) {
  if (threadIdx.x == 0) {
    if (spd < 0) set_status(status, DEV_TIMEOUT);
    else if (spd == 0 && diag) set_status(status, DEV_NOT_SPD);
  }
}

// The factor's panel sweep: four warps in FP64, one warp (no barriers) in
// FP32, whose FMA rate makes the one-warp sweep short.
template <typename T>
__device__ void panel_factor(T (*Dk)[33], T (*Ta)[33], bool tall, int* spd, int ncols) {
  if constexpr (sizeof(T) == 8) panel_sweep4<T>(Dk, Ta, tall, spd, ncols);
  else panel_sweep<T>(Dk, Ta, tall, spd, ncols);
}

// C (32 x 32 in smem) -= P Q^T, P, Q 32 x 32 in smem; 256 threads.
template <typename T>
__device__ void tile_sub_pqt(T (*C)[33], T (*P)[33], T (*Q)[33]) {
  const int tid = threadIdx.x;
  const int a = tid >> 3, b0 = (tid & 7) * 4;
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
  for (int cc = 0; cc < 32; ++cc) {
    const T pa = P[a][cc];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] += pa * Q[b0 + v][cc];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) C[a][b0 + v] -= acc[v];
  __syncthreads();
}

// Look-ahead schedule: between barriers k-1 and k the grid does, as one
// list of independent items,
//   panel(k)        tile rows k..Tt-1 of column k, each first applying the
//                   rank-32 update of step k-1 to its own tiles, and
//   update(k-1)     every trailing tile (i, j) with k < j <= i,
// so a step costs one grid barrier.  The diagonal factor and the panel tile's
// solve x L_kk^T = a share one register sweep (panel_sweep).  The FP32 kernel
// is held to 128 registers a thread, so one of its CTAs fits on an SM beside
// a CTA of the fused pass (256 threads x 128 registers): the look-ahead
// pipeline runs the two together.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_chol_coop(T* __restrict__ L, T* __restrict__ Dinv, int d, int dp,
                                                   int Tt, unsigned* bar, int* status) {
  __shared__ T Dk[32][33];
  __shared__ T Ta[32][33];
  __shared__ T Tb[32][33];
  __shared__ T Tc[32][33];
  __shared__ int spd;
  const int tid = threadIdx.x;
  const unsigned nb = gridDim.x;
  for (int k = 0; k < Tt; ++k) {
    const int k0 = k * 32, kp = (k - 1) * 32;
    const int npanel = Tt - k;
    const int u = Tt - k - 1;
    const int nupd = (k >= 1) ? u * (u + 1) / 2 : 0;
    for (int item = blockIdx.x; item < npanel + nupd; item += gridDim.x) {
      if (item < npanel) {
        const int c = item;
        const int i0 = (k + c) * 32;
        // all tile loads of the item at once
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int r = e >> 5, q = e & 31;
          Dk[r][q] = __ldcg(L + (int64_t)(k0 + r) * dp + k0 + q);
          if (k >= 1) Tb[r][q] = __ldcg(L + (int64_t)(k0 + r) * dp + kp + q);  // L_{k,k-1}
          if (c > 0) {
            Ta[r][q] = __ldcg(L + (int64_t)(i0 + r) * dp + k0 + q);
            if (k >= 1) Tc[r][q] = __ldcg(L + (int64_t)(i0 + r) * dp + kp + q);  // L_{i,k-1}
          }
        }
        __syncthreads();
        if (k >= 1) {
          tile_sub_pqt(Dk, Tb, Tb);
          if (c > 0) tile_sub_pqt(Ta, Tc, Tb);
        }
        if (c == 0) {
          // sweeping the identity alongside gives L_kk^{-T} in the same steps
          for (int e = tid; e < 1024; e += blockDim.x) Ta[e >> 5][e & 31] = ((e >> 5) == (e & 31)) ? T(1) : T(0);
          __syncthreads();
        }
        panel_factor<T>(Dk, Ta, true, &spd, min(32, d - k0));
        note_sweep(spd, c == 0, status);
        if (c == 0) {
          // L_kk itself is not stored: the other panel items of this step
          // read the diagonal tile of L concurrently (it must keep the
          // updated Hessian tile until the next barrier), and the solve
          // only needs D_k = L_kk^{-1}.
          for (int e = tid; e < 1024; e += blockDim.x) {
            const int r = e >> 5, q = e & 31;
            Dinv[(int64_t)k * 1024 + e] = (q <= r) ? Ta[q][r] : T(0);  // (L_kk^{-T})^T
          }
        } else {
          for (int e = tid; e < 1024; e += blockDim.x) {
            const int a = e >> 5, b = e & 31;
            L[(int64_t)(i0 + a) * dp + k0 + b] = Ta[a][b];
            L[(int64_t)(k0 + a) * dp + i0 + b] = Ta[b][a];  // transpose into tile (k, i)
          }
        }
        __syncthreads();
      } else {
        // update(k-1) of tile (i, j), k < j <= i
        const int q = item - npanel;
        int ii = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
        while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
        while (ii * (ii + 1) / 2 > q) --ii;
        const int jj = q - ii * (ii + 1) / 2;
        const int i0 = (k + 1 + ii) * 32, j0 = (k + 1 + jj) * 32;
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int r = e >> 5, cc = e & 31;
          Ta[r][cc] = __ldcg(L + (int64_t)(i0 + r) * dp + kp + cc);
          Tb[r][cc] = __ldcg(L + (int64_t)(j0 + r) * dp + kp + cc);
        }
        __syncthreads();
        const int a = tid >> 3, b0 = (tid & 7) * 4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
        for (int cc = 0; cc < 32; ++cc) {
          const T pa = Ta[a][cc];
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[v] += pa * Tb[b0 + v][cc];
        }
        T* out = L + (int64_t)(i0 + a) * dp + j0 + b0;
#pragma unroll
        for (int v = 0; v < 4; ++v) __stcg(out + v, __ldcg(out + v) - acc[v]);
        __syncthreads();
      }
    }
    if (k + 1 < Tt && !grid_barrier(bar, nb, status)) return;
  }
}

// FP64 schedule: two phases a step, each ended by a grid barrier.
//   P(k)  panel(k) items, tile rows k..Tt-1 of column k: the tiles already
//         carry every update of steps < k, so an item only sweeps;
//   U(k)  the rank-32 update of step k on every trailing lower tile (i, j),
//         k < j <= i, split into four items of eight rows each.
// At GB300's FP64 rate (about two FMA lanes a clock an SM) a 32 x 32 rank-32
// tile update takes about 8 us on one SM; in k_chol_coop's one-barrier
// schedule each panel item applied two of them (its diagonal and its own
// tile) before its sweep, on the critical path of every step.  Here the
// update is spread over the grid as 2 us items and the step's critical path
// is sweep + barrier + quarter update + barrier.  Every entry goes through
// the same operations in the same order as in k_chol_coop (the same 32-term
// product sums, subtracted once a step), so the factor is the same bit for
// bit.  The updated diagonal tiles are written back to L (nothing reads
// them: the solve and the inverse use D_k).
template <typename T>
__global__ void __launch_bounds__(256, 1) k_chol_coop2(T* __restrict__ L, T* __restrict__ Dinv,
                                                       int d, int dp, int Tt, unsigned* bar,
                                                       int* status) {
  __shared__ T Dk[32][33];
  __shared__ T Ta[32][33];
  __shared__ T Pq[8][33];
  __shared__ int spd;
  const int tid = threadIdx.x;
  const unsigned nb = gridDim.x;
  for (int k = 0; k < Tt; ++k) {
    const int k0 = k * 32;
    const int npanel = Tt - k;
    for (int c = blockIdx.x; c < npanel; c += gridDim.x) {
      const int i0 = (k + c) * 32;
      for (int e = tid; e < 1024; e += blockDim.x) {
        const int r = e >> 5, q = e & 31;
        Dk[r][q] = __ldcg(L + (int64_t)(k0 + r) * dp + k0 + q);
        // sweeping the identity alongside the diagonal item gives L_kk^{-T}
        Ta[r][q] = (c > 0) ? __ldcg(L + (int64_t)(i0 + r) * dp + k0 + q) : (r == q ? T(1) : T(0));
      }
      __syncthreads();
      panel_factor<T>(Dk, Ta, true, &spd, min(32, d - k0));
      note_sweep(spd, c == 0, status);
      if (c == 0) {
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int r = e >> 5, q = e & 31;
          Dinv[(int64_t)k * 1024 + e] = (q <= r) ? Ta[q][r] : T(0);  // (L_kk^{-T})^T
        }
      } else {
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int a = e >> 5, b = e & 31;
          L[(int64_t)(i0 + a) * dp + k0 + b] = Ta[a][b];
          L[(int64_t)(k0 + a) * dp + i0 + b] = Ta[b][a];  // transpose into tile (k, i)
        }
      }
      __syncthreads();
    }
    if (k + 1 == Tt) break;
    if (!grid_barrier(bar, nb, status)) return;
    // U(k): tile (i, j) = (k + 1 + ii, k + 1 + jj), rows 8 qr .. 8 qr + 7
    const int u = Tt - k - 1;
    const int nitems = 4 * (u * (u + 1) / 2);
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      const int q = item >> 2, qr = item & 3;
      int ii = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
      while (ii * (ii + 1) / 2 > q) --ii;
      const int jj = q - ii * (ii + 1) / 2;
      const int i0 = (k + 1 + ii) * 32 + qr * 8, j0 = (k + 1 + jj) * 32;
      for (int e = tid; e < 1024; e += blockDim.x) {
        const int r = e >> 5, cc = e & 31;
        Ta[r][cc] = __ldcg(L + (int64_t)(j0 + r) * dp + k0 + cc);  // L_{j,k}
        if (r < 8) Pq[r][cc] = __ldcg(L + (int64_t)(i0 + r) * dp + k0 + cc);  // rows of L_{i,k}
      }
      __syncthreads();
      const int a = tid >> 5, b = tid & 31;
      T acc = T(0);
#pragma unroll 8
      for (int cc = 0; cc < 32; ++cc) acc += Pq[a][cc] * Ta[b][cc];
      T* out = L + (int64_t)(i0 + a) * dp + j0 + b;
      __stcg(out, __ldcg(out) - acc);
      __syncthreads();
    }
    if (!grid_barrier(bar, nb, status)) return;
  }
}

// ----------------------------------------------------------------------------
// Cluster variant: the same blocked factor and look-ahead schedule, with the
// whole matrix resident in the shared memory of one 16-CTA thread-block
// cluster, so a step ends with a hardware cluster barrier instead of a
// grid barrier through global memory.  Lower tile (i, j), j <= i, number
// q = i(i+1)/2 + j, lives in slot q / 16 of CTA q % 16; tiles of other CTAs
// are copied into local scratch through distributed shared memory before
// use.  Each step's items are the same as k_chol_coop's (panel(k) items
// first applying update k-1 to their own tiles and refactoring the diagonal
// tile, update(k-1) items for the remaining trailing tiles), each done by
// the CTA that owns the tile it writes, in the same arithmetic order, so L
// and D are identical to k_chol_coop's.  The input is read straight from H
// (identity padding), and the results go to the same L / Dinv layout.
// ----------------------------------------------------------------------------
constexpr int kClusterCtas = 16;
constexpr int kTileElems = 32 * 33;

template <typename T>
size_t chol_cluster_smem(int Tt) {
  const int ntiles = Tt * (Tt + 1) / 2;
  const int slots = (ntiles + kClusterCtas - 1) / kClusterCtas;
  return (size_t)(slots + 4) * kTileElems * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) k_chol_cluster(const double* __restrict__ H, int d, int dp,
                                                      int Tt, T* __restrict__ L,
                                                      T* __restrict__ Dinv, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char cl_smem[];
  T* base = reinterpret_cast<T*>(cl_smem);
  const int ntiles = Tt * (Tt + 1) / 2;
  const int slots = (ntiles + kClusterCtas - 1) / kClusterCtas;
  typedef T Tile[33];
  Tile* Dk = reinterpret_cast<Tile*>(base + (size_t)(slots + 0) * kTileElems);
  Tile* Ta = reinterpret_cast<Tile*>(base + (size_t)(slots + 1) * kTileElems);
  Tile* Tb = reinterpret_cast<Tile*>(base + (size_t)(slots + 2) * kTileElems);
  Tile* Tc = reinterpret_cast<Tile*>(base + (size_t)(slots + 3) * kTileElems);
  __shared__ int spd;
  const int tid = threadIdx.x;
  const int me = (int)cl.block_rank();
  auto tnum = [](int i, int j) { return i * (i + 1) / 2 + j; };
  auto local_tile = [&](int q) { return reinterpret_cast<Tile*>(base + (size_t)(q / kClusterCtas) * kTileElems); };
  // copy tile q (any CTA) into local scratch dst
  auto fetch = [&](Tile* dst, int q) {
    const T* src = cl.map_shared_rank(base + (size_t)(q / kClusterCtas) * kTileElems, q % kClusterCtas);
    for (int e = tid; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;
      dst[r][c] = src[r * 33 + c];
    }
  };
  // load the owned tiles of H (identity beyond d)
  for (int q = me; q < ntiles; q += kClusterCtas) {
    int i = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
    while (tnum(i + 1, 0) <= q) ++i;
    while (tnum(i, 0) > q) --i;
    const int j = q - tnum(i, 0);
    Tile* t = local_tile(q);
    for (int e = tid; e < 1024; e += blockDim.x) {
      const int r = e >> 5, c = e & 31;
      const int gi = i * 32 + r, gj = j * 32 + c;
      T v;
      if (gi < d && gj < d) v = (T)H[(int64_t)gi * d + gj];
      else v = (gi == gj) ? T(1) : T(0);
      t[r][c] = v;
    }
  }
  cl.sync();
  for (int k = 0; k < Tt; ++k) {
    const int k0 = k * 32;
    // panel(k): tile rows k..Tt-1 of column k
    for (int i = k; i < Tt; ++i) {
      const int qi = tnum(i, k);
      if (qi % kClusterCtas != me) continue;
      const int c = i - k, i0 = i * 32;
      fetch(Dk, tnum(k, k));
      if (k >= 1) fetch(Tb, tnum(k, k - 1));
      if (c > 0 && k >= 1) fetch(Tc, tnum(i, k - 1));
      __syncthreads();
      Tile* own = local_tile(qi);
      if (k >= 1) {
        tile_sub_pqt(Dk, Tb, Tb);
        if (c > 0) tile_sub_pqt(own, Tc, Tb);
      }
      Tile* pan = own;
      if (c == 0) {
        for (int e = tid; e < 1024; e += blockDim.x) Ta[e >> 5][e & 31] = ((e >> 5) == (e & 31)) ? T(1) : T(0);
        __syncthreads();
        pan = Ta;
      }
      panel_factor<T>(Dk, pan, true, &spd, min(32, d - k0));
      note_sweep(spd, c == 0, status);
      if (c == 0) {
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int r = e >> 5, q = e & 31;
          Dinv[(int64_t)k * 1024 + e] = (q <= r) ? Ta[q][r] : T(0);  // (L_kk^{-T})^T
        }
      } else {
        for (int e = tid; e < 1024; e += blockDim.x) {
          const int a = e >> 5, b = e & 31;
          L[(int64_t)(i0 + a) * dp + k0 + b] = own[a][b];
          L[(int64_t)(k0 + a) * dp + i0 + b] = own[b][a];  // transpose into tile (k, i)
        }
      }
      __syncthreads();
    }
    // update(k-1) of tile (i, j), k < j <= i
    if (k >= 1) {
      for (int i = k + 1; i < Tt; ++i)
        for (int j = k + 1; j <= i; ++j) {
          const int q = tnum(i, j);
          if (q % kClusterCtas != me) continue;
          fetch(Ta, tnum(i, k - 1));
          fetch(Tb, tnum(j, k - 1));
          __syncthreads();
          tile_sub_pqt(local_tile(q), Ta, Tb);
        }
    }
    cl.sync();
  }
}

template <typename T>
static cudaError_t chol_cluster_launch(const double* H, int d, T* L, T* Dinv, int* status,
                                       cudaStream_t st, bool* used) {
  *used = false;
  const int dp = chol_padded(d), Tt = dp / 32;
  const size_t smem = chol_cluster_smem<T>(Tt);
  if (smem > 200 * 1024) return cudaSuccess;
  // per device: can a 16-CTA cluster with 200 KB of shared memory a CTA run?
  static std::atomic<int> ok_dev[64];  // 0 unknown, 1 yes, 2 no
  int dev = 0;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
  }
  if (dev >= 64) return cudaSuccess;
  int ok = ok_dev[dev].load() == 1;
  if (ok_dev[dev].load() == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_cluster<T>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = ensure_smem((const void*)k_chol_cluster<T>, 200 * 1024);
    int nclusters = 0;
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kClusterCtas);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 200 * 1024;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kClusterCtas;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_chol_cluster<T>, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();
    ok = (e == cudaSuccess && nclusters >= 1) ? 1 : 0;
    ok_dev[dev].store(ok ? 1 : 2);
  }
  if (!ok) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kClusterCtas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_chol_cluster<T>, H, d, dp, Tt, L, Dinv, status);
  note_launches(1);
  if (e != cudaSuccess) return e;
  *used = true;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t chol_impl(const double* H, int d, double shift, T* L, T* Dinv, unsigned* bar,
                             int* status, cudaStream_t st, bool allow_cluster, int max_ctas) {
  int dp = chol_padded(d), Tt = dp / 32;
  if (allow_cluster && shift == 0.0) {
    bool used = false;
    cudaError_t e = chol_cluster_launch<T>(H, d, L, Dinv, status, st, &used);
    if (e != cudaSuccess || used) return e;
  }
  const int blocks = (int)std::min<int64_t>(((int64_t)dp * dp + 255) / 256, 2048);
  { k_chol_init<T><<<blocks, 256, 0, st>>>(H, d, dp, shift, L); note_launches(1); }
  cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  constexpr bool two_phase = sizeof(T) == 8;
  const void* fn;
  if constexpr (two_phase) fn = (const void*)k_chol_coop2<T>;
  else fn = (const void*)k_chol_coop<T>;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, 0)) != cudaSuccess)
    return e;
  if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
  // one CTA per SM at most; no more CTAs than the largest phase has items
  const int most = two_phase ? std::max(Tt, 2 * Tt * (Tt - 1))
                             : std::max(Tt, Tt + (Tt - 2) * (Tt - 1) / 2);
  int grid = std::min(sms, most);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  grid = std::max(grid, 1);
  void* args[] = {(void*)&L,  (void*)&Dinv, (void*)&d,     (void*)&dp,
                  (void*)&Tt, (void*)&bar,  (void*)&status};
  e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, st);
  note_launches(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const double* H, int d, int f32, void* Lbuf, void* Dinv, unsigned* bar,
                            int* status, cudaStream_t st, int allow_cluster, double shift,
                            int max_ctas) {
  return f32 ? chol_impl<float>(H, d, shift, (float*)Lbuf, (float*)Dinv, bar, status, st,
                                allow_cluster != 0, max_ctas)
             : chol_impl<double>(H, d, shift, (double*)Lbuf, (double*)Dinv, bar, status, st,
                                 allow_cluster != 0, max_ctas);
}

// ----------------------------------------------------------------------------
// Solve L L^T delta = v in one CTA (32 warps), left-looking by 32-row tiles.
// mode 0: x += delta, step_norm = max |delta|;  mode 1: out = delta.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_solve(const T* __restrict__ L,
                                                     const T* __restrict__ Dinv, int d, int dp,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ x,
                                                     double* __restrict__ step_norm, int mode,
                                                     int dinv_in_smem) {
  extern __shared__ unsigned char sm_raw[];
  T* y = reinterpret_cast<T*>(sm_raw);  // dp: right-hand side, then the solution
  T* Ds = y + dp;                       // Tt * 1024 when dinv_in_smem
  __shared__ T t[32];
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int Tt = dp / 32;
  for (int i = tid; i < dp; i += blockDim.x) y[i] = (i < d) ? (T)v[i] : T(0);
  if (dinv_in_smem)
    for (int e = tid; e < Tt * 1024; e += blockDim.x) Ds[e] = Dinv[e];
  const T* Dk = dinv_in_smem ? Ds : Dinv;
  __syncthreads();
  if constexpr (sizeof(T) == 8) {
    // FP64 (a few tiles at the plain form's sizes): the plain left-looking
    // sweeps; the prefetch below measured slower there (d = 50 / 200).
    // forward: y_k = D_k (v_k - sum_{j < k} L_kj y_j)
    for (int k = 0; k < Tt; ++k) {
      const int k0 = k * 32, r = k0 + w;
      const T* Lr = L + (int64_t)r * dp;
      T s = T(0);
      for (int c = lane; c < k0; c += 32) s += Lr[c] * y[c];
      s = warp_sum(s);
      if (lane == 0) t[w] = y[r] - s;
      __syncthreads();
      T yv = Dk[(int64_t)k * 1024 + w * 32 + lane] * t[lane];
      yv = warp_sum(yv);
      if (lane == 0) y[r] = yv;
      __syncthreads();
    }
    // backward: z_k = D_k^T (y_k - sum_{j > k} (L^T)_kj z_j), (L^T)_kj stored in tile (k, j)
    for (int k = Tt - 1; k >= 0; --k) {
      const int k0 = k * 32, r = k0 + w;
      const T* Ur = L + (int64_t)r * dp;
      T s = T(0);
      for (int c = k0 + 32 + lane; c < dp; c += 32) s += Ur[c] * y[c];
      s = warp_sum(s);
      if (lane == 0) t[w] = y[r] - s;
      __syncthreads();
      T zv = Dk[(int64_t)k * 1024 + lane * 32 + w] * t[lane];
      zv = warp_sum(zv);
      if (lane == 0) y[r] = zv;
      __syncthreads();
    }
  } else {
    // FP32: both sweeps are software-pipelined: in step k each warp issues the loads
    // of the next step's row over the tiles whose solution is already known
    // (up to kPre tiles in registers, the rest loaded after the step) and adds
    // them up after the step's barriers, so their L2 latency overlaps the
    // step's dependent chain; the row of step k then only adds its last tile.
    // A lane adds its tiles in a fixed order (ascending forward, descending
    // backward), the same whichever step prefetched them.
    constexpr int kPre = 16;
    // forward: y_k = D_k (v_k - sum_{j < k} L_kj y_j)
    T part = T(0);  // row k0 + w: this lane's sum over tiles j < k - 1
    for (int k = 0; k < Tt; ++k) {
      const int k0 = k * 32, r = k0 + w;
      const bool nxt = k + 1 < Tt;
      const T* Ln = L + (int64_t)(r + 32) * dp;  // the next step's row
      T nl[kPre];
#pragma unroll
      for (int q = 0; q < kPre; ++q) nl[q] = (nxt && q < k) ? Ln[lane + 32 * q] : T(0);
      T s = part;
      if (k >= 1) s += L[(int64_t)r * dp + k0 - 32 + lane] * y[k0 - 32 + lane];
      s = warp_sum(s);
      if (lane == 0) t[w] = y[r] - s;
      __syncthreads();
      T yv = Dk[(int64_t)k * 1024 + w * 32 + lane] * t[lane];
      yv = warp_sum(yv);
      if (lane == 0) y[r] = yv;
      __syncthreads();
      T pn = T(0);
      if (nxt) {
#pragma unroll
        for (int q = 0; q < kPre; ++q)
          if (q < k) pn += nl[q] * y[lane + 32 * q];
        for (int q = kPre; q < k; ++q) pn += Ln[lane + 32 * q] * y[lane + 32 * q];
      }
      part = pn;
    }
    // backward: z_k = D_k^T (y_k - sum_{j > k} (L^T)_kj z_j), (L^T)_kj stored in
    // tile (k, j); a lane adds the tiles j = Tt-1, Tt-2, ..., k+1 in that order
    part = T(0);  // row k0 + w: this lane's sum over tiles j > k + 1
    for (int k = Tt - 1; k >= 0; --k) {
      const int k0 = k * 32, r = k0 + w;
      const bool nxt = k >= 1;
      const T* Un = L + (int64_t)(r - 32) * dp;  // the next step's row (tile k - 1)
      const int known = Tt - 1 - k;                // tiles Tt-1 .. k+1 are solved
      T nl[kPre];
#pragma unroll
      for (int q = 0; q < kPre; ++q)
        nl[q] = (nxt && q < known) ? Un[(Tt - 1 - q) * 32 + lane] : T(0);
      T s = part;
      if (k + 1 < Tt) s += L[(int64_t)r * dp + k0 + 32 + lane] * y[k0 + 32 + lane];
      s = warp_sum(s);
      if (lane == 0) t[w] = y[r] - s;
      __syncthreads();
      T zv = Dk[(int64_t)k * 1024 + lane * 32 + w] * t[lane];
      zv = warp_sum(zv);
      if (lane == 0) y[r] = zv;
      __syncthreads();
      T pn = T(0);
      if (nxt) {
#pragma unroll
        for (int q = 0; q < kPre; ++q)
          if (q < known) pn += nl[q] * y[(Tt - 1 - q) * 32 + lane];
        for (int q = kPre; q < known; ++q) {
          const int c = (Tt - 1 - q) * 32 + lane;
          pn += Un[c] * y[c];
        }
      }
      part = pn;
    }
  }
  double mx = 0.0;
  for (int i = tid; i < d; i += blockDim.x) {
    const double dl = (double)y[i];
    if (mode == 0) {
      x[i] += dl;
      mx = fmax(mx, fabs(dl));
    } else {
      x[i] = dl;
    }
  }
  if (mode == 0) {
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[w] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m2 = fmax(m2, red[q]);
      if (step_norm) *step_norm = m2;
    }
  }
}

template <typename T>
static cudaError_t solve_impl(const T* L, const T* Dinv, int d, const double* v, double* x,
                              double* step_norm, int mode, cudaStream_t st) {
  const int dp = chol_padded(d);
  const size_t base = (size_t)dp * sizeof(T);
  const size_t dinv = (size_t)(dp / 32) * 1024 * sizeof(T);
  const int in_smem = (base + dinv) <= 200 * 1024;
  const size_t smem = base + (in_smem ? dinv : 0);
  {
    cudaError_t e = ensure_smem((const void*)k_chol_solve<T>, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  k_chol_solve<T><<<1, 1024, smem, st>>>(L, Dinv, d, dp, v, x, step_norm, mode, in_smem);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol_step(const void* Lbuf, const void* Dinv, int d, int f32, const double* g,
                             double* x, double* step_norm, cudaStream_t st) {
  return f32 ? solve_impl<float>((const float*)Lbuf, (const float*)Dinv, d, g, x, step_norm, 0, st)
             : solve_impl<double>((const double*)Lbuf, (const double*)Dinv, d, g, x, step_norm, 0,
                                  st);
}

cudaError_t launch_chol_apply(const void* Lbuf, const void* Dinv, int d, int f32, const double* v,
                              double* out, cudaStream_t st) {
  return f32 ? solve_impl<float>((const float*)Lbuf, (const float*)Dinv, d, v, out, nullptr, 1, st)
             : solve_impl<double>((const double*)Lbuf, (const double*)Dinv, d, v, out, nullptr, 1,
                                  st);
}

// ----------------------------------------------------------------------------
// H^{-1} = L^{-T} L^{-1} from the factor, one CTA per 32-column block c of the
// identity (used by the penalised l1 step's active-set pass, which needs
// arbitrary columns of the inverse):
//   forward   Y_k = D_k (E_kc - sum_{c <= j < k} L_kj Y_j)   for k >= c
//             (Y_k = 0 for k < c: L is lower triangular),
//   backward  X_k = D_k^T (Y_k - sum_{j > k} (L^T)_kj X_j)   for k = Tt-1..0,
// with the Y / X tiles in shared memory and each thread reading its row of
// every L tile straight from global memory (eight threads share a row, so
// L1 serves most of it).  Skipped entirely when *need == 0.
// ----------------------------------------------------------------------------
// 32 consecutive values (16-byte aligned) into registers with vector loads.
IHS_DEV void load32(const float* __restrict__ p, float (&r)[32]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    r[4 * i] = v.x; r[4 * i + 1] = v.y; r[4 * i + 2] = v.z; r[4 * i + 3] = v.w;
  }
}
IHS_DEV void load32(const double* __restrict__ p, double (&r)[32]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
    r[2 * i] = v.x; r[2 * i + 1] = v.y;
  }
}

template <typename T>
size_t chol_inverse_smem(int Tt) { return (size_t)(Tt + 1) * 32 * 33 * sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(256) k_chol_inverse(const T* __restrict__ L,
                                                      const T* __restrict__ Dinv, int d, int dp,
                                                      T* __restrict__ Hinv,
                                                      const int* __restrict__ need) {
  if (need && *need == 0) return;
  extern __shared__ __align__(16) unsigned char inv_smem[];
  typedef T Row[33];
  Row* Ys = reinterpret_cast<Row*>(inv_smem);  // Tt tiles of 32 rows: rows k*32.., this column block
  Row* Tmp = Ys + dp;                          // one tile: staging for the D_k products
  const int Tt = dp / 32, c = blockIdx.x, tid = threadIdx.x;
  const int a = tid >> 3, b0 = (tid & 7) * 4;
  for (int k = 0; k < c; ++k)
    for (int e = tid; e < 1024; e += blockDim.x) Ys[k * 32 + (e >> 5)][e & 31] = T(0);
  // forward
  for (int k = c; k < Tt; ++k) {
    T acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] = (k == c && a == b0 + v) ? T(1) : T(0);
    const T* Lrow = L + (int64_t)(k * 32 + a) * dp;
    T lr[32];
    if (c < k) load32(Lrow + c * 32, lr);
    for (int j = c; j < k; ++j) {
      T cur[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) cur[q] = lr[q];
      if (j + 1 < k) load32(Lrow + (j + 1) * 32, lr);  // next tile's row in flight
#pragma unroll
      for (int q = 0; q < 32; ++q)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] -= cur[q] * Ys[j * 32 + q][b0 + v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Tmp[a][b0 + v] = acc[v];
    __syncthreads();
    const T* Dr = Dinv + (int64_t)k * 1024 + a * 32;  // row a of D_k
    T out[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const T dq = __ldg(Dr + q);
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] += dq * Tmp[q][b0 + v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Ys[(k) * 32 + a][b0 + v] = out[v];
    __syncthreads();
  }
  // backward (X_k overwrites Y_k)
  for (int k = Tt - 1; k >= 0; --k) {
    T acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] = Ys[(k) * 32 + a][b0 + v];
    const T* Urow = L + (int64_t)(k * 32 + a) * dp;  // row of the stored L^T tiles (k, j)
    T ur[32];
    if (k + 1 < Tt) load32(Urow + (k + 1) * 32, ur);
    for (int j = k + 1; j < Tt; ++j) {
      T cur[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) cur[q] = ur[q];
      if (j + 1 < Tt) load32(Urow + (j + 1) * 32, ur);
#pragma unroll
      for (int q = 0; q < 32; ++q)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] -= cur[q] * Ys[j * 32 + q][b0 + v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Tmp[a][b0 + v] = acc[v];
    __syncthreads();
    const T* Dc = Dinv + (int64_t)k * 1024 + a;  // column a of D_k
    T out[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const T dq = __ldg(Dc + q * 32);
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] += dq * Tmp[q][b0 + v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Ys[(k) * 32 + a][b0 + v] = out[v];
    __syncthreads();
  }
  for (int e = tid; e < dp * 32; e += blockDim.x) {
    const int r = e >> 5, cc = e & 31, col = c * 32 + cc;
    if (r < d && col < d) Hinv[(int64_t)r * d + col] = Ys[r][cc];
  }
}

size_t chol_inverse_smem_bytes(int d, int f32) {
  const int Tt = chol_padded(d) / 32;
  return f32 ? chol_inverse_smem<float>(Tt) : chol_inverse_smem<double>(Tt);
}

cudaError_t launch_chol_inverse(const void* Lbuf, const void* Dinv, int d, int f32, void* Hinv,
                                const int* need, cudaStream_t st) {
  const int dp = chol_padded(d), Tt = dp / 32;
  const size_t smem = chol_inverse_smem_bytes(d, f32);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (f32) {
    if ((e = ensure_smem((const void*)k_chol_inverse<float>, 220 * 1024)) != cudaSuccess)
      return e;
    k_chol_inverse<float><<<Tt, 256, smem, st>>>((const float*)Lbuf, (const float*)Dinv, d, dp,
                                                 (float*)Hinv, need);
  } else {
    if ((e = ensure_smem((const void*)k_chol_inverse<double>, 220 * 1024)) != cudaSuccess)
      return e;
    k_chol_inverse<double><<<Tt, 256, smem, st>>>((const double*)Lbuf, (const double*)Dinv, d,
                                                  dp, (double*)Hinv, need);
  }
  note_launches(1);
  return cudaGetLastError();
}
