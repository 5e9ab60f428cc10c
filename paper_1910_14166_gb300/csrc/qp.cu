// qp.cu -- the l1-ball subproblem of Eq. 2 (LASSO, C = {x : ||x||_1 <= R}):
//     x^{t+1} = argmin_{||x||_1 <= R} 1/2 (x - x^t)^T H (x - x^t) - g^T (x - x^t),
// solved exactly (Sec. 3: each subproblem "is solved exactly"), in one CTA:
//
//  1. Newton point: if x^t + H^{-1} g lies in the ball it is the answer.
//  2. Face solve on the support of the previous solution: on a face with
//     support S and signs sigma the KKT conditions are the bordered system
//         [H_SS sigma; sigma^T 0] [dS; mu] = [g_S + H_{S,S^c} x^t_{S^c}; R - sigma^T x^t_S]
//     for the increment dS = x_S - x^t_S and multiplier mu.  The point is
//     accepted only if mu >= 0, every x_S keeps its sign and
//     |(H (x - x^t) - g)_j| <= mu off S -- then it is the unique optimum.
//  3. Otherwise FISTA (Beck & Teboulle 2009) in FP32, preconditioned by
//     diag(H)^{-1}, with the exact projection onto the l1 ball in that
//     metric (a weighted form of Michelot's fixed-point threshold, exact
//     after finitely many passes), finds the support, and a face solve is
//     tried every kFaceEvery iterations.
// The face system is factored in the factor precision of the mode (FP32 in
// the mixed form) and refined with FP64 residuals, so dS and mu are FP64
// accurate.  Failure to certify within the iteration cap records
// DEV_NOT_CONVERGED and leaves the last feasible FISTA point.
//
// The penalised form (the experiments' LASSO, Sec. 5: + lambda ||x||_1
// instead of the ball) takes the same path: the full face first (every index
// in the support, signs from x^t, else from H^{-1} g: one more solve with the
// sketched factor, the answer when no sign changes), the previous face (x = 0
// included), then proximal FISTA (soft threshold at lambda D_j / L, the same
// preconditioner) with periodic faces, whose system has no border,
//     H_SS dS = g_S + H_{S,S^c} x^t_{S^c} - lambda sigma,
// and whose off-support test is |(H (x - x^t) - g)_j| <= lambda.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "internal.h"

constexpr int kQpThreads = 1024;
constexpr int kQpMaxD = 1024;
constexpr int kFaceEvery = 25;
static_assert(kQpMaxD <= kQpThreads, "the QP epilogue gives each thread one entry");
// Faces with at most kFaceSm<TF> indices are factored and solved in shared
// memory (row stride kFaceSm + 1, odd, so column walks hit distinct banks);
// larger faces use the global-memory path.
template <typename TF>
struct FaceSm {
  static constexpr int n = sizeof(TF) == 4 ? 160 : 128;
  static constexpr int ld = n + 1;
  static constexpr size_t bytes = (size_t)n * ld * sizeof(TF) + (size_t)2 * n * sizeof(double);
};

size_t qp_work_bytes(int d) {
  const size_t dp = (size_t)chol_padded(d);
  return (size_t)d * d * 4 + dp * dp * 8 + (size_t)9 * d * 8 + (size_t)(d + 4) * 4 + 256;
}

// ---- block reductions (1024 threads) --------------------------------------
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : T(0);
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

struct QpShared {
  double xt[kQpMaxD];    // x^t
  double gd[kQpMaxD];    // g
  double z[kQpMaxD + 1]; // face solution dS, then mu at [k]
  double ra[kQpMaxD + 1];
  float fx[kQpMaxD], fy[kQpMaxD], fv[kQpMaxD];
  float fxt[kQpMaxD];
  float dg[kQpMaxD];     // FISTA's diagonal preconditioner, 1 / H_jj
  int S[kQpMaxD];
  int k;           // support size
  int accept;
  double redd[33];
  float redf[33];
};

// ---- the FP32 product Hf v, on one CTA or spread over a cluster ----------
// One CTA reads the d x d matrix (4 MB at d = 1000) from L2 for every product
// at about 64 bytes a clock, some 30 us a product, and the l1 step's power
// iteration and FISTA take tens to hundreds of them.  When the step is
// launched as a thread-block cluster, rank 0 runs the step alone and the
// other CTAs only serve its products: rank 0 posts the command (the shared
// addresses of v and out) and meets the cluster at a barrier; every CTA then
// computes a contiguous slice of the rows, the helpers reading v from rank
// 0's shared memory and storing their results into rank 0's out through
// distributed shared memory, and a second barrier publishes them.  Each row
// is still summed by one warp in the same order, so a product is the same
// bit for bit on one CTA or on a cluster.  Rank 0 posts an exit command when
// its step ends, whichever way it ends, and stays resident through one more
// barrier, until every helper has read it.  Every barrier is passed by every
// thread of every CTA: rank 0 calls matvec_f (two barriers) only from
// block-uniform code, and the exit takes two barriers on both sides.
struct MvCmd {
  int op;  // 1: product, 0: exit
  uint32_t v_off, out_off;  // shared-window addresses of v and out in rank 0
};
__shared__ MvCmd g_mvcmd;

IHS_DEV uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
IHS_DEV uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster arrives (release) and waits (acquire).
IHS_DEV void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
// A shared-window address of this CTA mapped to the same offset in CTA `rank`.
IHS_DEV uint32_t cl_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
IHS_DEV float cl_ld_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
IHS_DEV uint32_t cl_ld_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
IHS_DEV void cl_st_f32(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Rows [r0, r1) of Hf v, a warp a row, v in this CTA's shared memory.
__device__ void matvec_rows(const float* __restrict__ Hf, int d, const float* v, int r0, int r1,
                            float* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = r0 + w; i < r1; i += (int)(blockDim.x >> 5)) {
    const float* row = Hf + (int64_t)i * d;
    float s = 0.f;
    for (int j = lane; j < d; j += 32) s = fmaf(row[j], v[j], s);
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
}

// y = Hf * v (FP32, warp per row).  All threads of the CTA call it; in a
// cluster launch only rank 0 runs the step and calls it (see above).
__device__ void matvec_f(const float* __restrict__ Hf, int d, const float* v, float* out) {
  const int C = (int)cl_size();
  if (C == 1) {
    matvec_rows(Hf, d, v, 0, d, out);
    return;
  }
  if (threadIdx.x == 0) g_mvcmd = MvCmd{1, smem_u32(v), smem_u32(out)};
  cl_sync();  // the command and v are visible to the helpers
  matvec_rows(Hf, d, v, 0, (int)((int64_t)d / C), out);
  cl_sync();  // every slice of out is written
}

// The helpers' side (ranks 1 .. C-1): serve rank 0's products until it exits.
__device__ void matvec_helper(const float* __restrict__ Hf, int d) {
  const int lane = threadIdx.x & 31;
  const uint32_t c = cl_rank(), C = cl_size();
  const int r0 = (int)((int64_t)d * c / C), r1 = (int)((int64_t)d * (c + 1) / C);
  const uint32_t cmd0 = cl_map(smem_u32(&g_mvcmd), 0);
  for (;;) {
    cl_sync();  // a command is posted
    if (cl_ld_u32(cmd0) == 0u) {
      cl_sync();  // rank 0 stays resident until every helper has read it
      break;
    }
    const uint32_t v0 = cl_map(cl_ld_u32(cmd0 + 4), 0), out0 = cl_map(cl_ld_u32(cmd0 + 8), 0);
    // lane l keeps v[l + 32 q] (read from rank 0) in vr[q]; each row is
    // summed in the same order as matvec_rows
    float vr[32];
#pragma unroll
    for (int q = 0; q < 32; ++q)
      vr[q] = (lane + 32 * q < d) ? cl_ld_f32(v0 + 4u * (uint32_t)(lane + 32 * q)) : 0.f;
    for (int i = r0 + (int)(threadIdx.x >> 5); i < r1; i += (int)(blockDim.x >> 5)) {
      const float* row = Hf + (int64_t)i * d;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = lane + 32 * q;
        if (j < d) s = fmaf(row[j], vr[q], s);
      }
      s = warp_sum(s);
      if (lane == 0) cl_st_f32(out0 + 4u * (uint32_t)i, s);
    }
    cl_sync();  // this slice of out is written
  }
}

// Projection onto the l1 ball in the metric of diag(D)^{-1}:
//   argmin_{||y||_1 <= R} sum_j (y_j - v_j)^2 / (2 D_j),
// y_j = sign(v_j) max(|v_j| - theta D_j, 0) with the theta >= 0 that puts y on
// the sphere.  theta by the weighted form of Michelot's iteration: on the
// active set A = {j : |v_j| > theta D_j}, theta = (sum_A |v_j| - R) /
// sum_A D_j; from the whole set it increases monotonically to the root
// (each step's theta is at most the root, and the active set shrinks).
__device__ void project_l1_w(float* v, const float* D, int d, float R, QpShared& sh) {
  float a = 0.f, w = 0.f;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    a += fabsf(v[j]);
    w += D[j];
  }
  const float tot = block_sum(a, sh.redf);
  if (tot <= R) return;
  const float W0 = block_sum(w, sh.redf);
  float theta = fmaxf((tot - R) / W0, 0.f);
  int prev = d;
  for (int it = 0; it < d + 1; ++it) {
    float s = 0.f, ws = 0.f, c = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      const float u = fabsf(v[j]);
      if (u > theta * D[j]) {
        s += u;
        ws += D[j];
        c += 1.f;
      }
    }
    const float S = block_sum(s, sh.redf);
    const float WS = block_sum(ws, sh.redf);
    const int cnt = (int)block_sum(c, sh.redf);
    if (cnt == 0 || !(WS > 0.f)) break;
    const float nt = (S - R) / WS;
    const bool stop = (cnt == prev) || !(nt > theta);
    theta = fmaxf(theta, nt);
    prev = cnt;
    if (stop) break;
  }
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const float u = fabsf(v[j]) - theta * D[j];
    v[j] = u > 0.f ? copysignf(u, v[j]) : 0.f;
  }
  __syncthreads();
}

// ---- small dense Cholesky of M = H_SS (k x k, stride ld) in TF, in place --
template <typename TF>
__device__ bool chol_small(TF* M, int k, int ld, QpShared& sh) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      TF p = M[(int64_t)j * ld + j];
      if (!(p > TF(0))) { bad = 1; p = TF(1); }
      M[(int64_t)j * ld + j] = sqrt(p);
    }
    __syncthreads();
    const TF piv = M[(int64_t)j * ld + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) M[(int64_t)i * ld + j] /= piv;
    __syncthreads();
    const int rem = k - j - 1;
    const int64_t cnt = (int64_t)rem * (rem + 1) / 2;
    for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
      // (r, c) with j < c <= r < k
      int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((int64_t)(r + 1) * (r + 2) / 2 <= e) ++r;
      while ((int64_t)r * (r + 1) / 2 > e) --r;
      const int c = (int)(e - (int64_t)r * (r + 1) / 2);
      const int rr = j + 1 + r, cc = j + 1 + c;
      M[(int64_t)rr * ld + cc] -= M[(int64_t)rr * ld + j] * M[(int64_t)cc * ld + j];
    }
    __syncthreads();
  }
  return bad == 0;
}

// out = M^{-1} v with M = L L^T (L in the lower triangle of M), in place in out.
template <typename TF>
__device__ void chol_small_solve(const TF* L, int k, int ld, double* v) {
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) v[j] = (double)((TF)v[j] / L[(int64_t)j * ld + j]);
    __syncthreads();
    const TF yj = (TF)v[j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x)
      v[i] = (double)((TF)v[i] - L[(int64_t)i * ld + j] * yj);
    __syncthreads();
  }
  for (int j = k - 1; j >= 0; --j) {
    if (threadIdx.x == 0) v[j] = (double)((TF)v[j] / L[(int64_t)j * ld + j]);
    __syncthreads();
    const TF zj = (TF)v[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x)
      v[i] = (double)((TF)v[i] - L[(int64_t)j * ld + i] * zj);
    __syncthreads();
  }
}

// Shared-memory variant: M (k x k, row stride ld) in place, right-looking
// with one barrier per column.  Step j applies the rank-1 update of pivot
// column j (still unscaled, so the update uses M_rj M_cj / p_j) to the
// trailing triangle and, in the same phase, scales column j-1 by its square
// root pivot -- the two touch disjoint entries.
template <typename TF>
__device__ bool chol_sm(TF* M, int k, int ld) {
  __shared__ TF dg[kQpMaxD];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int j = 0; j <= k; ++j) {
    if (j >= 1) {
      const TF dj = dg[j - 1];
      for (int r = j + threadIdx.x; r < k; r += blockDim.x) M[r * ld + (j - 1)] /= dj;
      if (threadIdx.x == 0) M[(j - 1) * ld + (j - 1)] = dj;
    }
    if (j < k) {
      TF p = M[j * ld + j];
      if (!(p > TF(0))) {
        if (threadIdx.x == 0) bad = 1;
        p = TF(1);
      }
      if (threadIdx.x == 0) dg[j] = sqrt(p);
      const TF ip = TF(1) / p;
      for (int r = j + 1 + w; r < k; r += nw) {
        const TF a = M[r * ld + j] * ip;
        for (int c = j + 1 + lane; c <= r; c += 32) M[r * ld + c] -= a * M[c * ld + j];
      }
    }
    __syncthreads();
  }
  return bad == 0;
}

// v <- M^{-1} v with M = L L^T from chol_sm, by warp 0 alone (forward then
// backward substitution, column by column, each lane owning every 32nd entry);
// the arithmetic is in TF like chol_small_solve.  All threads must call it.
template <typename TF>
__device__ void chol_sm_solve(const TF* L, int k, int ld, double* v) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int j = 0; j < k; ++j) {
      const TF yj = (TF)v[j] / L[j * ld + j];
      for (int i = j + 1 + lane; i < k; i += 32) v[i] = (double)((TF)v[i] - L[i * ld + j] * yj);
      __syncwarp();
      if (lane == 0) v[j] = (double)yj;
      __syncwarp();
    }
    for (int j = k - 1; j >= 0; --j) {
      const TF zj = (TF)v[j] / L[j * ld + j];
      for (int i = lane; i < j; i += 32) v[i] = (double)((TF)v[i] - L[j * ld + i] * zj);
      __syncwarp();
      if (lane == 0) v[j] = (double)zj;
      __syncwarp();
    }
  }
  __syncthreads();
}

// Face solve for support sh.S[0..k) with signs sign(sig_src): fills sh.z
// (dS, mu at [k]); returns false if the face matrix is not positive definite.
template <typename TF>
__device__ void face_apply(bool small, const TF* Ls, int k, int ld, double* v) {
  if (small) chol_sm_solve<TF>(Ls, k, ld, v);
  else chol_small_solve<TF>(Ls, k, ld, v);
}

// Ms: shared-memory face area (FaceSm<TF>::bytes) used when k <= FaceSm<TF>::n;
// otherwise the factor lives in Lg (global, stride ldg) and the two vectors in wg.
// pen: the penalised form, where the face system has no border: H_SS dS =
// g_S + H_{S,S^c} x^t_{S^c} - lambda sigma (R = lambda), and the multiplier
// slot sh.z[k] holds lambda for the off-support test.
template <typename TF>
__device__ bool face_solve(const double* __restrict__ H, int d, double R, bool pen,
                           const float* sig_src, TF* Lg, int ldg, double* wg, TF* Ms,
                           QpShared& sh) {
  const int k = sh.k;
  const bool small = k <= FaceSm<TF>::n;
  TF* Ls = small ? Ms : Lg;
  const int ld = small ? FaceSm<TF>::ld : ldg;
  double* wv = small ? reinterpret_cast<double*>(Ms + (size_t)FaceSm<TF>::n * FaceSm<TF>::ld) : wg;
  double* res = small ? wv + FaceSm<TF>::n : wg + d;
  // gather M = H_SS
  for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
    const int a = (int)(e / k), b = (int)(e - (int64_t)a * k);
    Ls[(int64_t)a * ld + b] = (TF)H[(int64_t)sh.S[a] * d + sh.S[b]];
  }
  __syncthreads();
  if (small ? !chol_sm<TF>(Ls, k, ld) : !chol_small<TF>(Ls, k, ld, sh)) return false;
  // w = M^{-1} sigma (the border's direction; not needed in the penalised form)
  double sTw = 1.0;
  if (!pen) {
    for (int a = threadIdx.x; a < k; a += blockDim.x) wv[a] = sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0;
    __syncthreads();
    face_apply<TF>(small, Ls, k, ld, wv);
    double sw = 0.0;
    for (int a = threadIdx.x; a < k; a += blockDim.x)
      sw += (sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0) * wv[a];
    sTw = block_sum(sw, sh.redd);
  }
  // right-hand side: ra = g_S + H_{S,S^c} x^t_{S^c},  beta = R - sigma^T x^t_S
  // (S^c part: x^t_l for l not in S)
  __shared__ unsigned char inS[kQpMaxD];
  for (int j = threadIdx.x; j < d; j += blockDim.x) inS[j] = 0;
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) inS[sh.S[a]] = 1;
  __syncthreads();
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  for (int a = wi; a < k; a += (int)(blockDim.x >> 5)) {
    const double* row = H + (int64_t)sh.S[a] * d;
    double s = 0.0;
    for (int l = lane; l < d; l += 32)
      if (!inS[l] && sh.xt[l] != 0.0) s = fma(row[l], sh.xt[l], s);
    s = warp_sum(s);
    if (lane == 0) sh.ra[a] = sh.gd[sh.S[a]] + s;
  }
  double bl = 0.0;
  for (int a = threadIdx.x; a < k; a += blockDim.x)
    bl += (sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0) * sh.xt[sh.S[a]];
  const double beta = R - block_sum(bl, sh.redd);
  // solve + FP64 refinement: z = 0 (mu = lambda, fixed, when penalised), then
  // residual steps
  for (int a = threadIdx.x; a <= k; a += blockDim.x) sh.z[a] = (pen && a == k) ? R : 0.0;
  __syncthreads();
  const int rounds = sizeof(TF) == 4 ? 4 : 2;
  for (int it = 0; it < rounds; ++it) {
    // residual res = rhs - K z in FP64: ra - (H_SS z + mu sigma), beta - sigma^T z
    for (int a = wi; a < k; a += (int)(blockDim.x >> 5)) {
      const double* row = H + (int64_t)sh.S[a] * d;
      double s = 0.0;
      for (int b = lane; b < k; b += 32) s = fma(row[sh.S[b]], sh.z[b], s);
      s = warp_sum(s);
      if (lane == 0)
        res[a] = sh.ra[a] - s - sh.z[k] * (sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0);
    }
    double sz = 0.0;
    for (int a = threadIdx.x; a < k; a += blockDim.x)
      sz += (sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0) * sh.z[a];
    const double rb = beta - block_sum(sz, sh.redd);
    // correction: u = M^{-1} res; dmu = (sigma^T u - rb) / sigma^T w; dz = u - dmu w
    face_apply<TF>(small, Ls, k, ld, res);
    double su = 0.0;
    for (int a = threadIdx.x; a < k; a += blockDim.x)
      su += (sig_src[sh.S[a]] > 0.f ? 1.0 : -1.0) * res[a];
    const double sTu = block_sum(su, sh.redd);
    const double dmu = pen ? 0.0 : (sTu - rb) / sTw;
    // (the penalised form leaves w unset: it has no border, and dmu = 0)
    for (int a = threadIdx.x; a < k; a += blockDim.x)
      sh.z[a] += pen ? res[a] : res[a] - dmu * wv[a];
    if (threadIdx.x == 0) sh.z[k] += dmu;
    __syncthreads();
  }
  return true;
}

// Check the KKT conditions of the face candidate; on success write x.
template <typename TF>
__device__ bool face_accept(const float* __restrict__ Hf, int d, const float* sig_src, double tol,
                            double* __restrict__ x, QpShared& sh) {
  const int k = sh.k;
  const double mu = sh.z[k];
  __shared__ int okf;
  if (threadIdx.x == 0) okf = (mu >= -tol) ? 1 : 0;
  __syncthreads();
  // candidate increment in FP32 for the off-support test: fv = x - x^t
  for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fv[j] = (float)(-sh.xt[j]);
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const int j = sh.S[a];
    const double xn = sh.xt[j] + sh.z[a];
    const bool pos = sig_src[j] > 0.f;
    if (!(pos ? xn > 0.0 : xn < 0.0)) okf = 0;
    sh.fv[j] = (float)sh.z[a];
  }
  __syncthreads();
  if (!okf) return false;
  // off support: |(H dx - g)_j| <= mu
  matvec_f(Hf, d, sh.fv, sh.fy);
  __syncthreads();
  double gscale = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) gscale = fmax(gscale, fabs(sh.gd[j]));
  for (int o = 16; o > 0; o >>= 1) gscale = fmax(gscale, __shfl_xor_sync(0xffffffffu, gscale, o));
  if ((threadIdx.x & 31) == 0) sh.redd[threadIdx.x >> 5] = gscale;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh.redd[w]);
    sh.redd[32] = m;
  }
  __syncthreads();
  gscale = sh.redd[32];
  __shared__ unsigned char inS2[kQpMaxD];
  for (int j = threadIdx.x; j < d; j += blockDim.x) inS2[j] = 0;
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) inS2[sh.S[a]] = 1;
  __syncthreads();
  const double slack = 1e-5 * (gscale + fabs(mu)) + tol;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    if (inS2[j]) continue;
    const double gj = (double)sh.fy[j] - sh.gd[j];
    if (fabs(gj) > mu + slack) okf = 0;
  }
  __syncthreads();
  if (!okf) return false;
  for (int j = threadIdx.x; j < d; j += blockDim.x) sh.ra[j] = 0.0;
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) sh.ra[sh.S[a]] = sh.xt[sh.S[a]] + sh.z[a];
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) x[j] = sh.ra[j];
  return true;
}

// Sign used for index j by the penalised full face: that of x^t_j, else that
// of u_j = (H^{-1} g)_j, else 0 (no sign: the full face is not tried).
__host__ __device__ __forceinline__ double pen_sign(double xt, double u) {
  if (xt != 0.0) return xt > 0.0 ? 1.0 : -1.0;
  return u > 0.0 ? 1.0 : (u < 0.0 ? -1.0 : 0.0);
}

// rhs_j = g_j - lambda pen_sign(x^t_j, u_j)
__global__ void k_pen_rhs(const double* __restrict__ xt, const double* __restrict__ g,
                          const double* __restrict__ u, double lam, int d,
                          double* __restrict__ rhs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
    rhs[j] = g[j] - lam * pen_sign(xt[j], u[j]);
}

// After a step: record the support of the new x (indices in increasing
// order; for the ball only when x lies on the sphere) for the next step's
// first face, and the step size max |x - x^t|.  d <= blockDim.x.
__device__ void qp_epilogue(const double* x, const double* xt, int d, double R, bool pen,
                            double* step_norm, int* support, double* redd) {
  __syncthreads();
  const int j0 = threadIdx.x;
  const double xj = j0 < d ? x[j0] : 0.0;
  const double l1 = block_sum(fabs(xj), redd);
  double mx = j0 < d ? fabs(xj - xt[j0]) : 0.0;
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ int wcnt[33];
  const bool nz = (pen || l1 >= R * (1.0 - 1e-12)) && j0 < d && xj != 0.0;
  const unsigned bal = __ballot_sync(0xffffffffu, nz);
  if ((threadIdx.x & 31) == 0) {
    redd[threadIdx.x >> 5] = mx;
    wcnt[threadIdx.x >> 5] = __popc(bal);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    int acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, redd[w]);
      const int c = wcnt[w];
      wcnt[w] = acc;
      acc += c;
    }
    *step_norm = m;
    support[d] = acc;
  }
  __syncthreads();
  if (nz) support[wcnt[threadIdx.x >> 5] + __popc(bal & lanemask_lt())] = j0;
}

// Support of v (indices in increasing order) into sh.S / sh.k, and an
// order-free signature of (support, signs) returned to every thread.
// d <= blockDim.x: one entry per thread.
__device__ unsigned long long support_of(const float* v, int d, QpShared& sh) {
  __shared__ int wc[33];
  __shared__ unsigned long long ws[32];
  const int j = threadIdx.x, lane = j & 31, w = j >> 5;
  const bool nz = j < d && v[j] != 0.f;
  const unsigned bal = __ballot_sync(0xffffffffu, nz);
  unsigned long long h =
      nz ? sm64_finalise(2ull * (unsigned long long)j + (v[j] < 0.f ? 2ull : 1ull)) : 0ull;
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if (lane == 0) {
    wc[w] = __popc(bal);
    ws[w] = h;
  }
  __syncthreads();
  if (j == 0) {
    int acc = 0;
    unsigned long long sig = 0ull;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      const int c = wc[q];
      wc[q] = acc;
      acc += c;
      sig += ws[q];
    }
    sh.k = acc;
    ws[0] = sig;
  }
  __syncthreads();
  if (nz) sh.S[wc[w] + __popc(bal & lanemask_lt())] = j;
  const unsigned long long sig = ws[0];
  __syncthreads();
  return sig;
}

template <typename TF>
__device__ void l1_step_body(
    const double* __restrict__ H, const float* __restrict__ Hf, int d,
    const double* __restrict__ g, const double* __restrict__ du, const double* __restrict__ uvec,
    double R, int pen, int phase, int* __restrict__ need, int max_iter,
    double tol, double* __restrict__ x, double* __restrict__ step_norm, int* __restrict__ support,
    int* __restrict__ iters, double* __restrict__ wv, TF* __restrict__ Ls, int ld,
    float* __restrict__ evec, int* status) {
  extern __shared__ __align__(16) unsigned char qp_smem[];
  QpShared& sh = *reinterpret_cast<QpShared*>(qp_smem);
  TF* Ms = reinterpret_cast<TF*>(qp_smem + (sizeof(QpShared) + 15) / 16 * 16);
  // phase 1 (penalised form): only if the earlier passes left the step open
  if (phase == 1 && *need == 0) return;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    sh.xt[j] = x[j];
    sh.gd[j] = g[j];
    sh.fxt[j] = (float)x[j];
  }
  __syncthreads();
  bool done = phase == 1;
  // 1. Newton point.  Ball: du = H^{-1} g; x^t + du is the answer if it lies
  //    in the ball.  Penalty: du = H^{-1} (g - lambda sigma) with sigma the
  //    signs of x^t (of H^{-1} g where x^t is 0), the stationary point of the
  //    face with every index in the support; it is the answer if no sign
  //    changes and no entry is zero.
  if (!pen) {
    double a = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) a += fabs(sh.xt[j] + du[j]);
    const double l1 = block_sum(a, sh.redd);
    if (l1 <= R) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) x[j] = sh.xt[j] + du[j];
      if (threadIdx.x == 0) support[d] = 0;
      done = true;
    }
  } else if (!done) {
    __shared__ int flips;
    if (threadIdx.x == 0) flips = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      const double sj = pen_sign(sh.xt[j], uvec[j]);
      const double xn = sh.xt[j] + du[j];
      if (!(sj * xn > 0.0)) flips = 1;
    }
    __syncthreads();
    if (!flips) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) x[j] = sh.xt[j] + du[j];
      done = true;
    }
    __syncthreads();
  }
  // 2. previous face (signs of x^t on the stored support; in the penalised
  //    form an empty support is the face x = 0, tried too)
  if (!done) {
    if (threadIdx.x == 0) sh.k = support[d];
    __syncthreads();
    // (penalised form: a face too large for shared memory is left to the
    // active-set pass, which works on its small zero set instead)
    if ((sh.k > 0 || pen) && !(pen && sh.k > FaceSm<TF>::n)) {
      for (int a = threadIdx.x; a < sh.k; a += blockDim.x) sh.S[a] = support[a];
      for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fv[j] = sh.fxt[j];
      __syncthreads();
      // a stored index whose x^t entry is zero has no sign: skip the attempt
      __shared__ int zero_sign;
      if (threadIdx.x == 0) zero_sign = 0;
      __syncthreads();
      for (int a = threadIdx.x; a < sh.k; a += blockDim.x)
        if (sh.xt[sh.S[a]] == 0.0) zero_sign = 1;
      __syncthreads();
      if (!zero_sign) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fx[j] = sh.xt[j] > 0.0 ? 1.f : -1.f;
        __syncthreads();
        if (face_solve<TF>(H, d, R, pen, sh.fx, Ls, ld, wv, Ms, sh) &&
            face_accept<TF>(Hf, d, sh.fx, tol, x, sh))
          done = true;
      }
    }
    __syncthreads();
  }
  if (phase == 1) done = false;
  // penalised form, phase 0: leave the rest to the active-set pass and phase 1
  if (pen && phase == 0 && !done) {
    if (threadIdx.x == 0) *need = 1;
    return;
  }
  // 3. FISTA + periodic face solves
  if (!done) {
    // FISTA with a diagonal (Jacobi) preconditioner D = diag(H)^{-1}: in the
    // variables y = D^{-1/2} x the Hessian D^{1/2} H D^{1/2} has a unit
    // diagonal, which removes the spread of the column scales (a Zipf
    // column distribution puts H's diagonal over three decades, and plain
    // FISTA then needs hundreds of iterations).  In x: the step is
    // x - D (H (x - x^t) - g) / L with L the top eigenvalue of
    // D^{1/2} H D^{1/2}, and the projection is onto the ball in the metric of
    // D^{-1} (the penalty's soft threshold scales by D_j likewise).  FISTA
    // only has to find the face: every accepted point is the face solution
    // certified by the KKT conditions.
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      const float hjj = Hf[(int64_t)j * d + j];
      sh.dg[j] = hjj > 0.f ? 1.f / hjj : 1.f;
    }
    // L by power iteration on D^{1/2} H D^{1/2}.  It starts from the top
    // eigenvector estimate left by the previous step when there is one: the
    // Hessians of successive steps are sketches of the same A^T A and share
    // their dominant direction up to the sketch's distortion.
    float e2 = 0.f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      const float u = evec[j];
      sh.fv[j] = u;
      e2 += u * u;
    }
    const bool warm = block_sum(e2, sh.redf) > 0.f;
    if (!warm)
      for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fv[j] = 1.0f + 0.01f * (float)(j % 7);
    __syncthreads();
    float lam = 1.f;
    const int npow = warm ? 12 : 40;
    for (int it = 0; it < npow; ++it) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fx[j] = sqrtf(sh.dg[j]) * sh.fv[j];
      __syncthreads();
      matvec_f(Hf, d, sh.fx, sh.fy);
      __syncthreads();
      float a = 0.f;
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        sh.fy[j] *= sqrtf(sh.dg[j]);
        a += sh.fy[j] * sh.fy[j];
      }
      const float nrm = sqrtf(block_sum(a, sh.redf));
      float b = 0.f;
      for (int j = threadIdx.x; j < d; j += blockDim.x) b += sh.fy[j] * sh.fv[j];
      lam = block_sum(b, sh.redf);
      for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fv[j] = sh.fy[j] / fmaxf(nrm, 1e-30f);
      __syncthreads();
    }
    for (int j = threadIdx.x; j < d; j += blockDim.x) evec[j] = sh.fv[j];
    const float Lip = 1.1f * fmaxf(lam, 1e-30f);
    const float Rf = (float)R;
    for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fx[j] = sh.fxt[j];
    __syncthreads();
    if (!pen) project_l1_w(sh.fx, sh.dg, d, Rf, sh);
    for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fy[j] = sh.fx[j];
    __syncthreads();
    float tk = 1.f;
    unsigned long long prev_sig = 0ull, failed_sig = 0ull;
    const int cap = max_iter > 0 ? max_iter : 20000;
    int it = 0;
    for (; it < cap && !done; ++it) {
      // grad at y: Hf (y - x^t) - g
      for (int j = threadIdx.x; j < d; j += blockDim.x) sh.fv[j] = sh.fy[j] - sh.fxt[j];
      __syncthreads();
      float* gv = sh.fv;  // reuse: matvec writes into a separate buffer below
      __shared__ float hv[kQpMaxD];
      matvec_f(Hf, d, gv, hv);
      __syncthreads();
      for (int j = threadIdx.x; j < d; j += blockDim.x)
        sh.fv[j] = sh.fy[j] - sh.dg[j] * (hv[j] - (float)sh.gd[j]) / Lip;
      __syncthreads();
      if (pen) {
        // proximal step of lambda ||.||_1 in the metric of D^{-1}: soft
        // threshold at lambda D_j / L
        const float tau = Rf / Lip;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
          const float u = fabsf(sh.fv[j]) - tau * sh.dg[j];
          sh.fv[j] = u > 0.f ? copysignf(u, sh.fv[j]) : 0.f;
        }
        __syncthreads();
      } else {
        project_l1_w(sh.fv, sh.dg, d, Rf, sh);
      }
      const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * tk * tk));
      const float mom = (tk - 1.f) / tn;
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float xn = sh.fv[j];
        sh.fy[j] = xn + mom * (xn - sh.fx[j]);
        sh.fx[j] = xn;
      }
      tk = tn;
      __syncthreads();
      if ((it + 1) % kFaceEvery == 0) {
        // Face of the FISTA iterate.  A (support, signs) pair whose face
        // already failed is not tried again (the face point depends on
        // nothing else), and a support too large for the shared-memory
        // factor is tried only once it has held over a whole interval.
        const unsigned long long sig = support_of(sh.fx, d, sh);
        const bool stable = sig == prev_sig;
        prev_sig = sig;
        if ((sh.k > 0 || pen) && sig != failed_sig && (sh.k <= FaceSm<TF>::n || stable)) {
          if (face_solve<TF>(H, d, R, pen, sh.fx, Ls, ld, wv, Ms, sh) &&
              face_accept<TF>(Hf, d, sh.fx, tol, x, sh))
            done = true;
          else
            failed_sig = sig;
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) atomicAdd(iters, it);
    if (!done) {
      set_status(status, DEV_NOT_CONVERGED);
      for (int j = threadIdx.x; j < d; j += blockDim.x) x[j] = (double)sh.fx[j];
      if (threadIdx.x == 0) support[d] = 0;
      done = true;
    }
  }
  __syncthreads();
  qp_epilogue(x, sh.xt, d, R, pen, step_norm, support, sh.redd);
  if (threadIdx.x == 0 && need) *need = 0;
}

// The l1 step: one CTA, or a cluster whose ranks 1 .. C-1 only serve rank
// 0's FP32 products (matvec_f).  Rank 0 posts the exit command once the step
// has ended, on every path out of l1_step_body.
template <typename TF>
__global__ void __launch_bounds__(kQpThreads, 1) k_l1_step(
    const double* __restrict__ H, const float* __restrict__ Hf, int d,
    const double* __restrict__ g, const double* __restrict__ du, const double* __restrict__ uvec,
    double R, int pen, int phase, int* __restrict__ need, int max_iter,
    double tol, double* __restrict__ x, double* __restrict__ step_norm, int* __restrict__ support,
    int* __restrict__ iters, double* __restrict__ wv, TF* __restrict__ Ls, int ld,
    float* __restrict__ evec, int* status) {
  const bool clustered = cl_size() > 1;
  if (clustered && cl_rank() != 0) {
    matvec_helper(Hf, d);
    return;
  }
  l1_step_body<TF>(H, Hf, d, g, du, uvec, R, pen, phase, need, max_iter, tol, x, step_norm,
                   support, iters, wv, Ls, ld, evec, status);
  if (clustered) {
    __syncthreads();
    if (threadIdx.x == 0) g_mvcmd.op = 0;
    cl_sync();  // the exit command is posted
    cl_sync();  // every helper has read it (rank 0's shared memory stays valid until then)
  }
}

// ----------------------------------------------------------------------------
// Penalised form, active-set pass (a primal-dual active-set method, i.e. a
// semismooth Newton method on the optimality conditions; Hintermueller, Ito &
// Kunisch 2002).  Faces whose zero set Z is small -- the common case for
// lambda small against A^T b, where the support covers most indices -- are
// solved with H^{-1} at hand (from the sketched factor): the face with zero
// set Z and signs sigma elsewhere is the KKT system
//     H dl + E_Z nu = g - lambda sigma~,   E_Z^T (x^t + dl) = 0
// (sigma~ = sigma off Z, 0 on Z), solved for nu' = nu - g_Z (which, like
// dl, vanishes at the optimum): p = H^{-1} v with v = g - lambda sigma off Z
// and 0 on Z, nu' = ((H^{-1})_ZZ)^{-1} (p_Z + x^t_Z), dl = p - (H^{-1})_{:,Z} nu' (in the
// plain form refined once with FP64 residuals of that system; the mixed form
// keeps the factor-precision point, as its OLS step does, and runs its
// products in FP32).  The point is the answer when every
// index off Z keeps its sign and |nu_j| <= lambda on Z (nu_j = -(H dl - g)_j
// there).  Each round takes the signs and zeros from the current point x and
// its dual y = g - H (x - x^t) by the diagonally scaled proximal rule
// sigma_j = sign(z_j) if |z_j| > lambda else 0, z_j = H_jj x_j + y_j,
// starting from x = x^t, y = g; at most kActiveRounds rounds,
// |Z| <= FaceSm<TF>::n, and a repeated pattern ends the pass.
constexpr int kActiveRounds = 32;

struct PenShared {
  double xt[kQpMaxD], gd[kQpMaxD], dl[kQpMaxD], p[kQpMaxD], v[kQpMaxD], r1[kQpMaxD];
  double vt[kQpMaxD];  // a matvec operand in the kernel's arithmetic type (float or double)
  int Z[kQpMaxD];
  int pos[kQpMaxD];  // index in Z, or -1
  signed char sg[kQpMaxD];
  int zc;
  int flag, best;
  double bestv;
  double redd[33];
};

// out_j = sum_i M[j, i] v_i, M d x d row-major in TM, accumulated in TM
// (FP32 in the mixed form: GB300's FP64 rate is 1/64 of FP32 and a d = 1000
// matrix-vector product in FP64 costs a quarter millisecond on one SM).
template <typename TM>
__device__ void matvec_d(const TM* __restrict__ M, int d, const TM* v, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < d; j += (int)(blockDim.x >> 5)) {
    const TM* row = M + (int64_t)j * d;
    TM s = TM(0);
    for (int i = lane; i < d; i += 32) s += row[i] * v[i];
    s = warp_sum(s);
    if (lane == 0) out[j] = (double)s;
  }
}

// out_j = base_j - sum_a Hinv[j, Z_a] nu_a (accumulated in TF)
template <typename TF>
__device__ void sub_cols(const TF* __restrict__ Hinv, int d, const int* Z, int zc, const double* nu,
                         const double* base, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < d; j += (int)(blockDim.x >> 5)) {
    const TF* row = Hinv + (int64_t)j * d;
    TF s = TF(0);
    for (int a = lane; a < zc; a += 32) s += row[Z[a]] * (TF)nu[a];
    s = warp_sum(s);
    if (lane == 0) out[j] = base[j] - (double)s;
  }
}

template <typename TF>
__global__ void __launch_bounds__(kQpThreads, 1) k_pen_active(
    const double* __restrict__ H, const float* __restrict__ Hf, const TF* __restrict__ Hinv, int d,
    const double* __restrict__ g, double lam, double* __restrict__ x,
    double* __restrict__ step_norm, int* __restrict__ support, int* __restrict__ need) {
  if (*need == 0) return;
  extern __shared__ __align__(16) unsigned char pa_smem[];
  PenShared& P = *reinterpret_cast<PenShared*>(pa_smem);
  TF* M = reinterpret_cast<TF*>(pa_smem + (sizeof(PenShared) + 15) / 16 * 16);
  constexpr int zmax = FaceSm<TF>::n, ld = FaceSm<TF>::ld;
  double* nu = reinterpret_cast<double*>(M + (size_t)zmax * ld);
  double* nu2 = nu + zmax;
  const int tid = threadIdx.x;
  TF* vt = reinterpret_cast<TF*>(P.vt);
  // H in the arithmetic type: FP64 H (plain form) or its FP32 copy (mixed)
  const TF* Ht = sizeof(TF) == 8 ? reinterpret_cast<const TF*>(H) : reinterpret_cast<const TF*>(Hf);
  for (int j = tid; j < d; j += blockDim.x) {
    P.xt[j] = x[j];
    P.gd[j] = g[j];
    P.dl[j] = 0.0;       // x - x^t
    P.r1[j] = g[j];      // y = g - H (x - x^t)
  }
  __shared__ int changed;
  bool accepted = false;
  int rounds_used = 0;
  for (int round = 0; round < kActiveRounds; ++round) {
    __syncthreads();
    rounds_used = round + 1;
    // signs and zeros from the current point and its dual
    if (tid == 0) changed = (round == 0);
    __syncthreads();
    for (int j = tid; j < d; j += blockDim.x) {
      const double xj = (round == 0) ? P.xt[j] : (P.sg[j] == 0 ? 0.0 : P.xt[j] + P.dl[j]);
      const double z = H[(int64_t)j * d + j] * xj + P.r1[j];
      const signed char sj = fabs(z) > lam ? (z > 0.0 ? 1 : -1) : 0;
      if (round > 0 && sj != P.sg[j]) changed = 1;
      P.sg[j] = sj;
    }
    __syncthreads();
    if (!changed) break;  // the same pattern again: no progress
    // Z list in index order
    if (tid == 0) {
      int c = 0;
      for (int j = 0; j < d; ++j) {
        P.pos[j] = -1;
        if (P.sg[j] == 0) {
          if (c < kQpMaxD) P.Z[c] = j;
          P.pos[j] = c;
          ++c;
        }
      }
      P.zc = c;
    }
    __syncthreads();
    const int zc = P.zc;
    if (zc > zmax) break;
    // right-hand side in the shifted form nu = g_Z + nu': g_j - lambda sigma_j
    // off Z and 0 on Z, so p, nu' and dl all vanish at the optimum and the
    // factor-precision products carry no O(lambda) cancellation
    for (int j = tid; j < d; j += blockDim.x) {
      P.v[j] = P.sg[j] != 0 ? P.gd[j] - lam * (double)P.sg[j] : 0.0;
      vt[j] = (TF)P.v[j];
    }
    __syncthreads();
    matvec_d<TF>(Hinv, d, vt, P.p);
    __syncthreads();
    // M = (H^{-1})_ZZ, factored in TF
    for (int e = tid; e < zc * zc; e += blockDim.x) {
      const int a = e / zc, b = e - a * zc;
      M[a * ld + b] = Hinv[(int64_t)P.Z[a] * d + P.Z[b]];
    }
    __syncthreads();
    if (!chol_sm<TF>(M, zc, ld)) break;
    for (int a = tid; a < zc; a += blockDim.x) nu[a] = P.p[P.Z[a]] + P.xt[P.Z[a]];
    __syncthreads();
    chol_sm_solve<TF>(M, zc, ld, nu);
    sub_cols<TF>(Hinv, d, P.Z, zc, nu, P.p, P.dl);
    __syncthreads();
    // refinement of the bordered system (plain form; the mixed form keeps the
    // factor-precision point, as its OLS step does)
    const int nref = sizeof(TF) == 4 ? 0 : 1;
    for (int it = 0; it < nref; ++it) {
      for (int j = tid; j < d; j += blockDim.x) vt[j] = (TF)P.dl[j];
      __syncthreads();
      matvec_d<TF>(Ht, d, vt, P.r1);  // r1 = H dl
      __syncthreads();
      for (int j = tid; j < d; j += blockDim.x) {
        const int a = P.pos[j];
        P.r1[j] = P.v[j] - P.r1[j] - (a >= 0 ? nu[a] : 0.0);
      }
      __syncthreads();
      for (int j = tid; j < d; j += blockDim.x) vt[j] = (TF)P.r1[j];
      __syncthreads();
      matvec_d<TF>(Hinv, d, vt, P.p);  // p = H^{-1} r1
      __syncthreads();
      for (int a = tid; a < zc; a += blockDim.x)
        nu2[a] = P.p[P.Z[a]] - (-P.xt[P.Z[a]] - P.dl[P.Z[a]]);
      __syncthreads();
      chol_sm_solve<TF>(M, zc, ld, nu2);
      sub_cols<TF>(Hinv, d, P.Z, zc, nu2, P.p, P.r1);  // r1 <- correction
      __syncthreads();
      for (int j = tid; j < d; j += blockDim.x) P.dl[j] += P.r1[j];
      for (int a = tid; a < zc; a += blockDim.x) nu[a] += nu2[a];
      __syncthreads();
    }
    // optimality: signs off Z, |nu| <= lambda on Z
    if (tid == 0) {
      P.flag = 0;
      P.best = -1;
      P.bestv = 0.0;
    }
    __syncthreads();
    for (int j = tid; j < d; j += blockDim.x) {
      if (P.sg[j] != 0 && !((double)P.sg[j] * (P.xt[j] + P.dl[j]) > 0.0)) atomicOr(&P.flag, 1);
    }
    __syncthreads();
    const double lim = lam * (1.0 + 1e-9);
    if (tid == 0) {
      for (int a = 0; a < zc; ++a) {
        const double over = fabs(P.gd[P.Z[a]] + nu[a]) - lim;
        if (over > P.bestv) {
          P.bestv = over;
          P.best = a;
        }
      }
    }
    __syncthreads();
    if (P.flag == 0 && P.best < 0) {
      for (int j = tid; j < d; j += blockDim.x) x[j] = P.sg[j] == 0 ? 0.0 : P.xt[j] + P.dl[j];
      accepted = true;
      break;
    }
    // dual at the new point: y = g - H dl (x - x^t = dl, with dl_Z = -x^t_Z)
    for (int j = tid; j < d; j += blockDim.x) vt[j] = (TF)P.dl[j];
    __syncthreads();
    matvec_d<TF>(Ht, d, vt, P.r1);
    __syncthreads();
    for (int j = tid; j < d; j += blockDim.x) P.r1[j] = P.gd[j] - P.r1[j];
  }
  __syncthreads();
  if (tid == 0) atomicAdd(need + 1, rounds_used);
  if (accepted) {
    qp_epilogue(x, P.xt, d, lam, true, step_norm, support, P.redd);
    if (tid == 0) *need = 0;
  }
}

size_t pen_active_smem(int f32) {
  const size_t base = (sizeof(PenShared) + 15) / 16 * 16;
  return base + (f32 ? FaceSm<float>::bytes : FaceSm<double>::bytes);
}

__global__ void k_to_float(const double* __restrict__ a, int64_t n, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// The l1 step's launch: for d >= kL1ClusterMinD a cluster of kL1Cluster
// CTAs (one SM each), rank 0 running the step and the others serving its
// FP32 products, where this GPU can hold such a cluster at this shared-memory
// size (checked once per device and size class); one CTA otherwise.
constexpr int kL1Cluster = 8;
constexpr int kL1ClusterMinD = 512;

template <typename TF, typename... Args>
static cudaError_t launch_l1_kernel(size_t smem, int d, cudaStream_t st, Args... args) {
  const void* fn = (const void*)k_l1_step<TF>;
  cudaError_t e = ensure_smem(fn, (int)smem);
  if (e != cudaSuccess) return e;
  int C = 1;
  if (d >= kL1ClusterMinD) {
    static std::atomic<int> ok_dev[64][2];  // [device][TF is double]: 0 unknown, 1 yes, 2 no
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    const int ti = sizeof(TF) == 8 ? 1 : 0;
    if (dev < 64) {
      if (ok_dev[dev][ti].load() == 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kL1Cluster);
        cfg.blockDim = dim3(kQpThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kL1Cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        const cudaError_t q = cudaOccupancyMaxActiveClusters(&nclusters, k_l1_step<TF>, &cfg);
        if (q != cudaSuccess) cudaGetLastError();
        ok_dev[dev][ti].store(q == cudaSuccess && nclusters >= 1 ? 1 : 2);
      }
      if (ok_dev[dev][ti].load() == 1) C = kL1Cluster;
    }
  }
  // The step is on the solve's critical path while the next iteration's
  // sketch chain runs beside it: launch it at the device's highest priority,
  // so that SMs freed by the chain's kernels go to the step first.
  int lo = 0, hi = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kQpThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = hi;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = C;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = C > 1 ? 2 : 1;
  e = cudaLaunchKernelEx(&cfg, k_l1_step<TF>, args...);
  note_launches(1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_l1_step(const double* H, const void* Lbuf, const void* Dinv, int f32, int d,
                           const double* g,
                           double R, int pen, int max_iter, double tol, QpWork w, double* x,
                           double* step_norm, int* status, cudaStream_t st) {
  if (d > kQpMaxD) return cudaErrorInvalidValue;
  const int64_t dd = (int64_t)d * d;
  { k_to_float<<<(unsigned)std::min<int64_t>((dd + 255) / 256, 2048), 256, 0, st>>>(H, dd, w.Hf); note_launches(1); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* du = w.dbuf;              // d
  double* wv = w.dbuf + d;          // 2d doubles of face-solve scratch
  double* uvec = w.dbuf + 3 * d;    // penalty: H^{-1} g
  double* rhs = w.dbuf + 4 * d;     // penalty: g - lambda sigma
  if (!pen) {
    e = launch_chol_apply(Lbuf, Dinv, d, f32, g, du, st);
    if (e != cudaSuccess) return e;
  } else {
    e = launch_chol_apply(Lbuf, Dinv, d, f32, g, uvec, st);
    if (e != cudaSuccess) return e;
    { k_pen_rhs<<<(d + 255) / 256, 256, 0, st>>>(x, g, uvec, R, d, rhs); note_launches(1); }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_chol_apply(Lbuf, Dinv, d, f32, rhs, du, st);
    if (e != cudaSuccess) return e;
  }
  const size_t base = (sizeof(QpShared) + 15) / 16 * 16;
  const size_t smem = base + (f32 ? FaceSm<float>::bytes : FaceSm<double>::bytes);
  const int ld = chol_padded(d);
  const double tl = tol > 0 ? tol : 1e-12;
  int* need = pen ? w.need : nullptr;
  // the penalised form runs phase 0, the inverse and the active-set pass, then
  // phase 1 (FISTA) -- each of the later ones exits at once if the step is done
  const bool active = pen && w.Hinv && chol_inverse_smem_bytes(d, f32) <= 220 * 1024;
  auto l1 = [&](int phase) -> cudaError_t {
    if (f32)
      return launch_l1_kernel<float>(smem, d, st, H, (const float*)w.Hf, d, g, (const double*)du,
                                     (const double*)uvec, R, pen, phase, need, max_iter, tl, x,
                                     step_norm, w.support, w.iters, wv, (float*)w.Ls, ld, w.evec,
                                     status);
    return launch_l1_kernel<double>(smem, d, st, H, (const float*)w.Hf, d, g, (const double*)du,
                                    (const double*)uvec, R, pen, phase, need, max_iter, tl, x,
                                    step_norm, w.support, w.iters, wv, (double*)w.Ls, ld, w.evec,
                                    status);
  };
  if ((e = l1(0)) != cudaSuccess) return e;
  if (!pen) return cudaSuccess;
  if (active) {
    if ((e = launch_chol_inverse(Lbuf, Dinv, d, f32, w.Hinv, need, st)) != cudaSuccess) return e;
    const size_t ps = pen_active_smem(f32);
    if (f32) {
      if ((e = ensure_smem((const void*)k_pen_active<float>, (int)ps)) != cudaSuccess) return e;
      k_pen_active<float><<<1, kQpThreads, ps, st>>>(H, w.Hf, (const float*)w.Hinv, d, g, R, x,
                                                     step_norm, w.support, need);
    } else {
      if ((e = ensure_smem((const void*)k_pen_active<double>, (int)ps)) != cudaSuccess) return e;
      k_pen_active<double><<<1, kQpThreads, ps, st>>>(H, w.Hf, (const double*)w.Hinv, d, g, R,
                                                      x, step_norm, w.support, need);
    }
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return l1(1);
}
