// noalloc.cu -- ihs_gradient_noalloc: the dense residual/gradient pass
// g = A^T (b - A x) - lambda x (the linear term of Eq. 2) for callers that
// cannot allocate device memory.
//
// It is a variant of the dense gradient kernels in grad.cu whose per-warp
// partial gradients live in a fixed file-scope device array instead of a
// workspace from ihs_create, and which splits b into float pairs on the fly
// instead of reading a pre-split copy.  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine.
//
// The scratch array is shared by every call in the process: each call
// overwrites the slots it reads (every participating warp writes all d of
// its partials, even when it owns no rows), so nothing needs clearing, but
// two calls in flight on the GPU at the same time race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

// 4 MiB of partial gradients: (warps) x d doubles.
constexpr int64_t kNoAllocScratchDoubles = 512 * 1024;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

constexpr int kNaThreads = 256;

template <int NV, bool VEC4>
__global__ void __launch_bounds__(kNaThreads) k_rg_noalloc_f32(
    const float* __restrict__ A, int64_t lda, int64_t n, int d, const double* __restrict__ b,
    const double* __restrict__ x, double* __restrict__ gpart, int nwarps) {
  extern __shared__ float xs_na[];
  const int dpad = NV * 128;
  float* xh = xs_na;
  float* xl = xs_na + dpad;
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
  const int64_t r0 = min(n, (int64_t)w * per), r1 = min(n, r0 + per);
  constexpr int V = VEC4 ? 4 : 1;
  constexpr int NQ = VEC4 ? NV : NV * 4;
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
  for (int64_t i0 = r0; i0 < r1; i0 += 32) {
    // one FP64 -> float-pair split per lane covers 32 rows
    float bh_l = 0.f, bl_l = 0.f;
    if (i0 + lane < r1) split_double(b[i0 + lane], bh_l, bl_l);
    const int cnt = (int)min((int64_t)32, r1 - i0);
    for (int j = 0; j < cnt; ++j) {
      const float* row = A + (i0 + j) * lda;
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
      float rh = __shfl_sync(0xffffffffu, bh_l, j), rl = __shfl_sync(0xffffffffu, bl_l, j);
      dd_add(rh, rl, -sh, -sl);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int t = 0; t < V; ++t) dd_fma_acc(gh[q][t], gl[q][t], a[q][t], rh, rl);
    }
  }
  double* gp = gpart + (int64_t)w * d;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int c = colq[q] + t;
      if (c < d) gp[c] = (double)gh[q][t] + (double)gl[q][t];
    }
}

template <int NQ>
__global__ void __launch_bounds__(kNaThreads) k_rg_noalloc_f64(
    const double* __restrict__ A, int64_t lda, int64_t n, int d, const double* __restrict__ b,
    const double* __restrict__ x, double* __restrict__ gpart, int nwarps) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int64_t per = (n + nwarps - 1) / nwarps;
  const int64_t r0 = min(n, (int64_t)w * per), r1 = min(n, r0 + per);
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
    const double ri = b[i] - s;
#pragma unroll
    for (int q = 0; q < NQ; ++q) g[q] = fma(a[q], ri, g[q]);
  }
  double* gp = gpart + (int64_t)w * d;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (colq[q] < d) gp[colq[q]] = g[q];
}

// g[c] = sum of the warps' partials in a fixed order, minus lambda x[c].
__global__ void k_noalloc_reduce(const double* __restrict__ gpart, int nwarps, int d,
                                 const double* __restrict__ x, double lam,
                                 double* __restrict__ g) {
  __shared__ double part[8][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (c < d)
    for (int w = wi; w < nwarps; w += 8) acc += gpart[(int64_t)w * d + c];
  part[wi][lane] = acc;
  __syncthreads();
  if (wi == 0 && c < d) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += part[k][lane];
    if (lam != 0.0) s -= lam * x[c];
    g[c] = s;
  }
}

// Device address of the scratch array and the SM count, looked up once per
// device (with that device current) and cached.  A module's __device__ array
// lives in a CUDA context: if the device's primary context is destroyed and
// re-created (cudaDeviceReset), the array is reloaded, possibly at another
// address.  So each cached entry also records the unique id of the context it
// was taken in (cuCtxGetId, reached through the runtime's driver entry-point
// query), and a call made in a different context looks the address up again.
typedef int (*PFN_ctxGetCurrent)(void**);
typedef int (*PFN_ctxGetId)(void*, unsigned long long*);

constexpr int kMaxDevices = 64;
struct ScratchEntry {
  double* addr = nullptr;
  unsigned long long ctx_id = 0;
  int sms = 0;
};
ScratchEntry g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// Unique id of the calling thread's current context (0 when no context is
// current yet); *known = false if the driver entry points cannot be had, and
// the cache is then keyed by device alone.
unsigned long long current_context_id(bool* known) {
  static PFN_ctxGetCurrent get_cur = nullptr;
  static PFN_ctxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (PFN_ctxGetCurrent)p;
    p = nullptr;
    if (cudaGetDriverEntryPoint("cuCtxGetId", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PFN_ctxGetId)p;
  });
  *known = get_cur && get_id;
  if (!*known) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

cudaError_t scratch_for_current_device(double** out, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  bool known = false;
  const unsigned long long id = current_context_id(&known);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchEntry& E = g_scratch[dev];
  // look up on the first call on the device, and again in a new context (or
  // on a thread with no context current yet: the lookup makes one current)
  if (!E.addr || (known && (id == 0 || id != E.ctx_id))) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    E.addr = (double*)p;
    E.ctx_id = known ? current_context_id(&known) : 0;
    E.sms = nsm > 0 ? nsm : 1;
  }
  *out = E.addr;
  *sms = E.sms;
  return cudaSuccess;
}

}  // namespace

extern "C" ihs_status ihs_gradient_noalloc(const ihs_matrix* A, const double* b, const double* x,
                                           double lambda, double* g, void* stream) {
  if (!A || !x || !g) return IHS_ERR_ARG;
  if (A->kind != IHS_DENSE || (A->dtype != IHS_F32 && A->dtype != IHS_F64)) return IHS_ERR_ARG;
  if (A->n < 0 || A->n >= (1ll << 31) || A->d < 1 || A->ld < A->d) return IHS_ERR_ARG;
  // an empty A (n = 0) needs no values and no b: g = -lambda x
  if (A->n > 0 && (A->val == nullptr || b == nullptr)) return IHS_ERR_ARG;
  if (A->d > 1024) return IHS_ERR_UNSUPPORTED;
  const int d = (int)A->d;
  double* scratch = nullptr;
  int sms = 1;
  cudaError_t e = scratch_for_current_device(&scratch, &sms);
  if (e != cudaSuccess) return IHS_ERR_CUDA;
  // warps: as many as the scratch holds, at most 16 per SM of this device,
  // and none with fewer than four rows
  const int64_t by_scratch = kNoAllocScratchDoubles / d;
  int nwarps = (int)std::max<int64_t>(1, std::min<int64_t>({by_scratch, (int64_t)sms * 16,
                                                            (A->n + 3) / 4}));
  if ((int64_t)nwarps * d > kNoAllocScratchDoubles) return IHS_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (nwarps * 32 + kNaThreads - 1) / kNaThreads;
  if (A->dtype == IHS_F32) {
    const bool v4 = (A->ld % 4 == 0) && (A->d % 4 == 0) && ((uintptr_t)A->val % 16 == 0);
    const int nv = (d + 127) / 128;
    const size_t smem = (size_t)2 * nv * 128 * sizeof(float);
    const float* Av = (const float*)A->val;
#define NA32(NV)                                                                        \
  do {                                                                                  \
    if (v4)                                                                             \
      k_rg_noalloc_f32<NV, true><<<blocks, kNaThreads, smem, st>>>(Av, A->ld, A->n, d, b, x, \
                                                                  scratch, nwarps);     \
    else                                                                                \
      k_rg_noalloc_f32<NV, false><<<blocks, kNaThreads, smem, st>>>(Av, A->ld, A->n, d, b, x, \
                                                                   scratch, nwarps);    \
  } while (0)
    switch (nv) {
      case 1: NA32(1); break;
      case 2: NA32(2); break;
      case 3: NA32(3); break;
      case 4: NA32(4); break;
      case 5: NA32(5); break;
      case 6: NA32(6); break;
      case 7: NA32(7); break;
      case 8: NA32(8); break;
      default: return IHS_ERR_UNSUPPORTED;
    }
#undef NA32
  } else {
    const double* Av = (const double*)A->val;
    const int nq = (d + 31) / 32;
#define NA64(NQ) \
  k_rg_noalloc_f64<NQ><<<blocks, kNaThreads, 0, st>>>(Av, A->ld, A->n, d, b, x, scratch, nwarps)
    if (nq <= 2) NA64(2);
    else if (nq <= 4) NA64(4);
    else if (nq <= 8) NA64(8);
    else if (nq <= 16) NA64(16);
    else NA64(32);
#undef NA64
  }
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return IHS_ERR_CUDA;
  k_noalloc_reduce<<<(d + 31) / 32, 256, 0, st>>>(scratch, nwarps, d, x, lambda, g);
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return IHS_ERR_CUDA;
  return IHS_OK;
}
