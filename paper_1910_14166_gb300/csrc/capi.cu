// capi.cu -- the C ABI of include/ihs.h: context, workspaces and the IHS loop
// (Eq. 2): per iteration t, ihs_sketch(t) draws S (Sec. 2), forms SA, the
// Hessian (SA)^T SA / s (+ lambda I) and its Cholesky factor; ihs_step forms
// the exact gradient A^T (b - A x^t) and takes the QP step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

// CTAs of the factor that runs beside the look-ahead fused pass (the pass
// leaves these slots free): 16 for the FP32 factor, which at d <= 512 ends
// well within one pass on 16 SMs.  The FP64 factor takes a few passes' time
// on GB300's FP64 units, so the pass of iteration t forms SA of t +
// kFp64Depth and kFp64Depth factors run at once, each on 16 CTAs and a stream
// of its own (on one stream they would queue, and depth would buy latency,
// not throughput).  Measured on the 1,048,576 x 500 OLS workload (25
// iterations): one factor stream, sorts on st2, 32 CTAs: 29.6 ms; sorts on a
// stream of their own: 26.8 ms; two factor streams of 16 CTAs (depth 2):
// 24.0 ms; three (depth 3, 48 slots taken from the pass): 26.5 ms; three of
// 11 CTAs (33 slots): 27.0 ms.
constexpr int kLookaheadFactorCtas = 16;
constexpr int kLookaheadFactorCtasF64 = 16;
constexpr int kFp64Depth = 2;
// Factor buffers (H, L, D^{-1}): two in rotation, kFp64Depth + 1 when the
// look-ahead pipeline runs kFp64Depth iterations ahead (FP64 factor).
constexpr int kFacBufs = kFp64Depth + 1;

static int64_t g_launches = 0;  // kernel launches issued by the library
void note_launches(int k) { __atomic_add_fetch(&g_launches, (int64_t)k, __ATOMIC_RELAXED); }
int64_t launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

cudaError_t ensure_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> set;  // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& kv : set)
    if (kv.first.first == fn && kv.first.second == dev) {
      if (kv.second >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e == cudaSuccess) kv.second = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) set.push_back({{fn, dev}, bytes});
  return e;
}

struct StageEvents {
  std::vector<cudaEvent_t> ev;     // pool: pairs (start, stop)
  std::vector<int> stage;          // stage of pair k
  std::vector<cudaStream_t> strm;  // stream of pair k
  size_t used = 0;
};

struct ihs_ctx {
  cudaStream_t st = nullptr;   // caller's stream: gradient, step, adjoint
  cudaStream_t st2 = nullptr;  // internal stream: sketch draw, SA, Gram, factor
  cudaEvent_t ev_fac[kFacBufs] = {};  // factor of buffer b ready
  cudaEvent_t ev_use[kFacBufs] = {};  // last step reading buffer b done
  cudaEvent_t ev_join = nullptr;
  cudaEvent_t ev_grad = nullptr;  // gradient pass of the current iteration done
  cudaEvent_t ev_sa = nullptr;    // look-ahead: SA of the next counter formed
  cudaEvent_t ev_gram = nullptr;  // look-ahead: the Gram has read SA (SA free)
  cudaEvent_t ev_tail2 = nullptr; // the tail of the internal stream (joined into the caller's)
  // FP64-factor look-ahead pipeline: a third internal stream for the sorts,
  // so that a sort does not queue behind a factor on st2 (neither needs the
  // other), and kFp64Depth factor streams, each with its own grid-barrier
  // words (fbar[0] is bar); ev_s3 starts these streams after st2 and ev_fgo
  // hands a Gram's result to a factor stream; ev_s3 and ev_fend join them
  // back into st2 at the end of a solve
  cudaStream_t st3 = nullptr;
  cudaEvent_t ev_s3 = nullptr;
  // the in-order (non-fused) pipeline: the chain's factor on a stream of its
  // own, so that the next chain's sketch does not queue behind it
  cudaStream_t fchain = nullptr;
  cudaEvent_t ev_fc_go = nullptr, ev_fc_end = nullptr;
  cudaStream_t fst[kFp64Depth] = {};
  cudaEvent_t ev_fgo[kFp64Depth] = {};
  cudaEvent_t ev_fend[kFp64Depth] = {};
  unsigned* fbar[kFp64Depth] = {};
  bool prof = false;
  StageEvents pe;
  double prof_ms[IHS_NSTAGES] = {};
  int prof_cnt[IHS_NSTAGES] = {};
  int64_t prof_launch0 = 0;
  int sms = 152;
  // problem
  ihs_matrix A{};
  const double* b = nullptr;
  ihs_constraint C{};
  ihs_options opt{};
  int64_t n = 0, d = 0, m = 0;
  int s = 1;
  int prec = 0, acc64 = 1, f32fac = 0;
  bool dense = true;
  // dense path
  DenseA DA{};
  SortPlan sp{};
  void* sort_ws = nullptr;
  uint32_t* perm = nullptr;        // sort output, buffer 0
  int32_t* seg = nullptr;
  int32_t* chunk_first = nullptr;
  uint32_t* perm2 = nullptr;       // buffer 1 (fused pipeline)
  int32_t* seg2 = nullptr;
  int32_t* chunk_first2 = nullptr;
  bool fused = false;              // ihs_solve uses the single fused pass
  bool lookahead = false;          // ... forming SA one iteration ahead
  double* gcta = nullptr;          // per-CTA gradient partials of the fused pass
  cudaEvent_t ev_sort[2] = {};
  cudaEvent_t ev_read[2] = {};
  void* sk_partial = nullptr;
  int rg_warps = 0;
  double* gpart = nullptr;
  float2* bsplit = nullptr;
  // CSR path (CSC copy)
  CscA CA{};
  void* csc_partial = nullptr;
  void* rbuf = nullptr;
  double* item_part = nullptr;
  // sketch / Hessian (H, L, Dinv double-buffered: the next iteration's sketch
  // chain runs while the current step still reads its factor)
  void* SA = nullptr;
  // SRHT comparison sketch: n2 x ldt transform buffer and the sampled rows
  bool srht = false;
  void* srht_T = nullptr;
  int32_t* srht_rows = nullptr;
  // Gaussian comparison sketch: plan and split partials
  bool gauss = false;
  GaussPlan gplan{};
  void* gauss_part = nullptr;
  void* gauss_At = nullptr;  // mixed form: A^T in TF32, K-major (built at create)
  GramPlan gp{};
  void* gop = nullptr;
  float* gpart_f = nullptr;
  double* gpart_d = nullptr;
  double* H[kFacBufs] = {};
  void* L[kFacBufs] = {};
  void* Dinv[kFacBufs] = {};
  int nbuf = 2;  // factor buffers in rotation (la + 1 in the look-ahead pipeline)
  int la = 1;    // look-ahead pipeline: the pass of iteration t forms SA of t + la
  int fac_ctas = kLookaheadFactorCtas;  // look-ahead pipeline: CTAs of the factor
  int fac_slots = kLookaheadFactorCtas;  // CTA slots the fused pass leaves to factors
  // CUDA graph of ihs_solve for launch-bound problems: the whole solve for
  // (t0, iters), captured once and replayed, on an internal copy xg of the
  // iterate so that the graph does not depend on the caller's pointer
  bool graphs = false;
  cudaStream_t gst = nullptr;  // internal stream the graph is captured and launched on
  double* xg = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t g_t0 = -1;
  int g_iters = -1;
  int g_cur_end = 0;
  bool last_graph = false;  // the last ihs_solve ran as a CUDA graph
  unsigned* bar = nullptr;
  int cur = 1;  // buffer of the last sketch
  double* g = nullptr;
  double* step_norm = nullptr;
  int* status = nullptr;
  int* counter = nullptr;
  // adjoint workspace (allocated on first use): v, r, z, p, q (d each), scal[4]
  double* cg = nullptr;
  // exact-Gram partials and the error scalar (allocated on first use)
  double* xg_part = nullptr;
  size_t xg_bytes = 0;
  double* errbuf = nullptr;
  // l1 QP
  QpWork qw{};
  // p = 2 ball: c, x(mu), w, r, du (d each), scalars, and a barrier of its own
  double* l2buf = nullptr;
  unsigned* l2bar = nullptr;
  bool have_sketch = false;
  std::vector<void*> allocs;
};

void prof_stage_begin(void* c, int stage);
void prof_stage_end(void* c);

namespace {

// Record a stage boundary on `s` (timing enabled only).
void stage_begin(ihs_ctx* c, int stage, cudaStream_t s) {
  if (!c->prof) return;
  StageEvents& P = c->pe;
  if (P.used + 2 > P.ev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      P.ev.push_back(e);
    }
    P.stage.resize(P.ev.size() / 2);
    P.strm.resize(P.ev.size() / 2);
  }
  P.stage[P.used / 2] = stage;
  P.strm[P.used / 2] = s;
  cudaEventRecord(P.ev[P.used], s);
}
void stage_end(ihs_ctx* c) {
  if (!c->prof) return;
  StageEvents& P = c->pe;
  if (P.used + 2 > P.ev.size()) return;
  cudaEventRecord(P.ev[P.used + 1], P.strm[P.used / 2]);
  P.used += 2;
}
// Fold completed event pairs into the totals (after a synchronisation).
void stage_collect(ihs_ctx* c) {
  StageEvents& P = c->pe;
  for (size_t k = 0; k < P.used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[k], P.ev[k + 1]) == cudaSuccess) {
      c->prof_ms[P.stage[k / 2]] += ms;
      c->prof_cnt[P.stage[k / 2]] += 1;
    }
  }
  P.used = 0;
}

}  // namespace

void prof_stage_begin(void* c, int stage) {
  if (!c) return;
  ihs_ctx* x = (ihs_ctx*)c;
  // continue on the stream of the stage that the launcher just closed
  const StageEvents& P = x->pe;
  cudaStream_t s = (P.used >= 2) ? P.strm[P.used / 2 - 1] : x->st2;
  stage_begin(x, stage, s);
}
void prof_stage_end(void* c) {
  if (c) stage_end((ihs_ctx*)c);
}

namespace {

ihs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return IHS_OK;
  if (e == cudaErrorMemoryAllocation) return IHS_ERR_OOM;
  return IHS_ERR_CUDA;
}

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_status(e_);  \
  } while (0)

// Library-owned stream-ordered memory pool, one per device, whose release
// threshold is the maximum: what ihs_destroy frees stays in the pool, and the
// next ihs_create on the device takes it back without new device mappings
// (a create with ~25 separate cudaMalloc calls cost milliseconds).
// ihs_trim_memory returns the pool's unused memory to the device.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t library_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if ((e = cudaMemPoolCreate(&g_pool[dev], &props)) != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    if ((e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep)) !=
        cudaSuccess)
      return e;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

template <typename T>
ihs_status dalloc(ihs_ctx* c, T** p, size_t bytes) {
  void* q = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool;
  cudaError_t e = library_pool(&pool);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IHS_ERR_CUDA;
  }
  e = cudaMallocFromPoolAsync(&q, bytes, pool, c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IHS_ERR_OOM;
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return IHS_OK;
}
#define AL(ptr, bytes)                                  \
  do {                                                  \
    ihs_status s_ = dalloc(c, &(ptr), (size_t)(bytes)); \
    if (s_ != IHS_OK) return s_;                        \
  } while (0)

__global__ void k_expand_rows(int64_t n, const void* rowptr, int i64, int32_t* rowexp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = i64 ? ((const int64_t*)rowptr)[i] : ((const int32_t*)rowptr)[i];
    int64_t b = i64 ? ((const int64_t*)rowptr)[i + 1] : ((const int32_t*)rowptr)[i + 1];
    for (int64_t p = a; p < b; ++p) rowexp[p] = (int32_t)i;
  }
}
__global__ void k_csc_gather(int64_t nnz, const uint32_t* perm, const int32_t* rowexp,
                             const void* val, int f32, int32_t* rowidx, void* cval) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t p = perm[q];
    rowidx[q] = rowexp[p];
    if (f32) ((float*)cval)[q] = ((const float*)val)[p];
    else ((double*)cval)[q] = ((const double*)val)[p];
  }
}
__global__ void k_csr_check(int64_t nnz, const int32_t* col, int64_t d, int* bad) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x) {
    int c = col[q];
    if (c < 0 || c >= d) atomicExch(bad, 1);
  }
}

ihs_status build_csc(ihs_ctx* c) {
  const int64_t nnz = c->A.nnz, n = c->n, d = c->d;
  if (nnz >= (1ll << 31)) return IHS_ERR_UNSUPPORTED;
  int* bad;
  AL(bad, sizeof(int));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), c->st));
  if (nnz > 0)
    { k_csr_check<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 8192), 256, 0, c->st>>>(
        nnz, c->A.col, d, bad); note_launches(1); }
  int hbad = 0;
  CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (hbad) return IHS_ERR_ARG;
  // host copy of rowptr for validation
  std::vector<int64_t> rp(n + 1);
  if (c->A.rowptr_i64) {
    CK(cudaMemcpy(rp.data(), c->A.rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
  } else {
    std::vector<int32_t> r32(n + 1);
    CK(cudaMemcpy(r32.data(), c->A.rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i <= n; ++i) rp[i] = r32[i];
  }
  if (rp[0] != 0 || rp[n] != nnz) return IHS_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return IHS_ERR_ARG;

  int32_t* rowexp;
  AL(rowexp, nnz * sizeof(int32_t));
  if (n > 0)
    { k_expand_rows<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, c->st>>>(
        n, c->A.rowptr, c->A.rowptr_i64, rowexp); note_launches(1); }
  SortPlan p = make_sort_plan(nnz, (int)d, 1);
  void* ws;
  AL(ws, sort_workspace_bytes(p));
  uint32_t* perm;
  int32_t* seg;
  AL(perm, nnz * sizeof(uint32_t));
  AL(seg, (d + 1) * sizeof(int32_t));
  CK(launch_sort_keys(p, c->A.col, ws, perm, seg, c->st));
  int32_t* rowidx;
  void* cval;
  const size_t el = (c->A.dtype == IHS_F32) ? 4 : 8;
  AL(rowidx, nnz * sizeof(int32_t));
  AL(cval, nnz * el);
  if (nnz > 0)
    { k_csc_gather<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 8192), 256, 0, c->st>>>(
        nnz, perm, rowexp, c->A.val, c->A.dtype == IHS_F32, rowidx, cval); note_launches(1); }
  CK(cudaGetLastError());
  std::vector<int32_t> cp32(d + 1);
  CK(cudaMemcpyAsync(cp32.data(), seg, (d + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  // work items: column chunks of at most kItem entries (a column with no
  // entries still gets one item so its zero column is written)
  const int64_t kItem = 1 << 14;
  std::vector<int32_t> icol, islot, first(d + 1);
  std::vector<int64_t> ib, ie;
  int nsplit = 0;
  for (int64_t j = 0; j < d; ++j) {
    first[j] = (int32_t)icol.size();
    const int64_t a = cp32[j], e = cp32[j + 1];
    const int64_t k = std::max<int64_t>(1, (e - a + kItem - 1) / kItem);
    for (int64_t q = 0; q < k; ++q) {
      icol.push_back((int32_t)j);
      ib.push_back(a + (e - a) * q / k);
      ie.push_back(a + (e - a) * (q + 1) / k);
      islot.push_back(k > 1 ? nsplit++ : -1);
    }
  }
  first[d] = (int32_t)icol.size();
  std::vector<int64_t> cp64(cp32.begin(), cp32.end());
  const int ni = (int)icol.size();
  int64_t* colptr;
  int32_t *d_icol, *d_islot, *d_first;
  int64_t *d_ib, *d_ie;
  AL(colptr, (d + 1) * sizeof(int64_t));
  AL(d_icol, ni * sizeof(int32_t));
  AL(d_islot, ni * sizeof(int32_t));
  AL(d_first, (d + 1) * sizeof(int32_t));
  AL(d_ib, ni * sizeof(int64_t));
  AL(d_ie, ni * sizeof(int64_t));
  CK(cudaMemcpy(colptr, cp64.data(), (d + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_icol, icol.data(), ni * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_islot, islot.data(), ni * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_first, first.data(), (d + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_ib, ib.data(), ni * sizeof(int64_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_ie, ie.data(), ni * sizeof(int64_t), cudaMemcpyHostToDevice));
  CscA& A = c->CA;
  A.n = n;
  A.d = d;
  A.nnz = nnz;
  A.colptr = colptr;
  A.rowidx = rowidx;
  A.val = cval;
  A.f32 = c->A.dtype == IHS_F32;
  A.nitems = ni;
  A.item_col = d_icol;
  A.item_begin = d_ib;
  A.item_end = d_ie;
  A.item_slot = d_islot;
  A.nsplit_slots = nsplit;
  A.col_first_item = d_first;
  const size_t acc_el = c->acc64 ? 8 : 4;
  AL(c->csc_partial, (size_t)std::max(1, nsplit) * c->m * acc_el);
  AL(c->item_part, ni * sizeof(double));
  AL(c->rbuf, n * 8);
  return IHS_OK;
}

}  // namespace

extern "C" {

const char* ihs_status_str(ihs_status st) {
  switch (st) {
    case IHS_OK: return "ok";
    case IHS_ERR_ARG: return "invalid argument";
    case IHS_ERR_CUDA: return "CUDA error";
    case IHS_ERR_OOM: return "out of device memory";
    case IHS_ERR_NOT_SPD: return "sketched Hessian not positive definite";
    case IHS_ERR_NOT_CONVERGED: return "inner solver did not converge";
    case IHS_ERR_NONFINITE: return "non-finite value";
    case IHS_ERR_TIMEOUT: return "bounded device wait expired";
    case IHS_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

void ihs_destroy(ihs_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  if (c->st2) cudaStreamSynchronize(c->st2);
  for (cudaEvent_t e : c->pe.ev) cudaEventDestroy(e);
  for (int k = 0; k < kFacBufs; ++k) {
    if (c->ev_fac[k]) cudaEventDestroy(c->ev_fac[k]);
    if (c->ev_use[k]) cudaEventDestroy(c->ev_use[k]);
  }
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_grad) cudaEventDestroy(c->ev_grad);
  if (c->ev_sa) cudaEventDestroy(c->ev_sa);
  if (c->ev_gram) cudaEventDestroy(c->ev_gram);
  if (c->ev_tail2) cudaEventDestroy(c->ev_tail2);
  if (c->ev_s3) cudaEventDestroy(c->ev_s3);
  if (c->ev_fc_go) cudaEventDestroy(c->ev_fc_go);
  if (c->ev_fc_end) cudaEventDestroy(c->ev_fc_end);
  if (c->fchain) {
    cudaStreamSynchronize(c->fchain);
    cudaStreamDestroy(c->fchain);
  }
  for (int i = 0; i < kFp64Depth; ++i) {
    if (c->fst[i]) {
      cudaStreamSynchronize(c->fst[i]);
      cudaStreamDestroy(c->fst[i]);
    }
    if (c->ev_fgo[i]) cudaEventDestroy(c->ev_fgo[i]);
    if (c->ev_fend[i]) cudaEventDestroy(c->ev_fend[i]);
  }
  for (int k = 0; k < 2; ++k) {
    if (c->ev_sort[k]) cudaEventDestroy(c->ev_sort[k]);
    if (c->ev_read[k]) cudaEventDestroy(c->ev_read[k]);
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gst) {
    cudaStreamSynchronize(c->gst);
    cudaStreamDestroy(c->gst);
  }
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->st3) {
    cudaStreamSynchronize(c->st3);
    cudaStreamDestroy(c->st3);
  }
  for (void* p : c->allocs) cudaFreeAsync(p, c->st);
  cudaStreamSynchronize(c->st);
  delete c;
}

ihs_status ihs_create(ihs_ctx** out, const ihs_matrix* A, const double* b,
                      const ihs_constraint* C, const ihs_options* opt, void* stream) {
  if (!out || !A || !b || !C || !opt) return IHS_ERR_ARG;
  *out = nullptr;
  if (A->kind != IHS_DENSE && A->kind != IHS_CSR) return IHS_ERR_ARG;
  if (A->dtype != IHS_F64 && A->dtype != IHS_F32) return IHS_ERR_ARG;
  if (A->n < 1 || A->d < 1 || A->val == nullptr) return IHS_ERR_ARG;
  if (A->n >= (1ll << 31)) return IHS_ERR_ARG;
  if (A->d > 1024) return IHS_ERR_UNSUPPORTED;
  if (opt->s < 1 || opt->s > kMaxBlocks || opt->m < 1 || opt->m % opt->s != 0) return IHS_ERR_ARG;
  if (opt->m < A->d) return IHS_ERR_ARG;
  if (opt->precision < IHS_PREC_FP64 || opt->precision > IHS_PREC_BF16) return IHS_ERR_ARG;
  const int known = IHS_FLAG_NO_FUSE | IHS_FLAG_SERIAL | IHS_FLAG_CLUSTER | IHS_FLAG_NO_LOOKAHEAD |
                    IHS_FLAG_FP64_FACTOR | IHS_FLAG_NO_GRAPH;
  if (opt->flags & ~known) return IHS_ERR_ARG;
  if (C->kind != IHS_OLS && C->kind != IHS_L1_BALL && C->kind != IHS_RIDGE &&
      C->kind != IHS_L1_PENALTY && C->kind != IHS_L2_BALL)
    return IHS_ERR_ARG;
  if ((C->kind == IHS_L1_BALL || C->kind == IHS_L1_PENALTY || C->kind == IHS_L2_BALL) &&
      !(C->param > 0))
    return IHS_ERR_ARG;
  if (C->kind == IHS_RIDGE && !(C->param >= 0)) return IHS_ERR_ARG;
  if (A->kind == IHS_DENSE && A->ld < A->d) return IHS_ERR_ARG;
  if (A->kind == IHS_CSR && (A->col == nullptr || A->rowptr == nullptr || A->nnz < 0))
    return IHS_ERR_ARG;
  if (A->kind == IHS_DENSE && (int64_t)opt->s * A->n >= (1ll << 31)) return IHS_ERR_UNSUPPORTED;
  if (opt->sketch != IHS_SKETCH_SPARSE && opt->sketch != IHS_SKETCH_SRHT &&
      opt->sketch != IHS_SKETCH_GAUSSIAN)
    return IHS_ERR_ARG;
  if (opt->sketch != IHS_SKETCH_SPARSE) {
    if (opt->s != 1) return IHS_ERR_ARG;
    if (A->kind != IHS_DENSE) return IHS_ERR_UNSUPPORTED;
    if (opt->sketch == IHS_SKETCH_SRHT && srht_n2(A->n) > (1ll << 31)) return IHS_ERR_UNSUPPORTED;
  }

  ihs_ctx* c = new (std::nothrow) ihs_ctx();
  if (!c) return IHS_ERR_OOM;
  c->st = (cudaStream_t)stream;
  c->A = *A;
  c->b = b;
  c->C = *C;
  c->opt = *opt;
  c->n = A->n;
  c->d = A->d;
  c->m = opt->m;
  c->s = opt->s;
  c->prec = opt->precision;
  c->acc64 = (c->prec == IHS_PREC_FP64);
  c->f32fac = (c->prec != IHS_PREC_FP64) && !(opt->flags & IHS_FLAG_FP64_FACTOR);
  c->dense = (A->kind == IHS_DENSE);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);

  auto fail = [&](ihs_status s) {
    ihs_destroy(c);
    return s;
  };
  const size_t acc_el = c->acc64 ? 8 : 4;
  ihs_status s = IHS_OK;
#define AL2(ptr, bytes)                                   \
  do {                                                    \
    if ((s = dalloc(c, &(ptr), (size_t)(bytes))) != IHS_OK) return fail(s); \
  } while (0)
  if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->fchain, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fc_go, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fc_end, cudaEventDisableTiming) != cudaSuccess)
    return fail(IHS_ERR_CUDA);
  for (int k = 0; k < kFacBufs; ++k) {
    if (cudaEventCreateWithFlags(&c->ev_fac[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_use[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(IHS_ERR_CUDA);
  }
  if (cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_grad, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_sa, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_gram, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tail2, cudaEventDisableTiming) != cudaSuccess)
    return fail(IHS_ERR_CUDA);
  for (int k = 0; k < 2; ++k) {
    if (cudaEventCreateWithFlags(&c->ev_sort[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_read[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(IHS_ERR_CUDA);
  }
  AL2(c->SA, (size_t)c->m * c->d * acc_el);
  const int dp = chol_padded((int)c->d);
  for (int k = 0; k < kFacBufs; ++k) {
    AL2(c->H[k], (size_t)c->d * c->d * sizeof(double));
    AL2(c->L[k], (size_t)dp * dp * (c->f32fac ? 4 : 8));
    AL2(c->Dinv[k], chol_dinv_bytes((int)c->d, c->f32fac));
  }
  AL2(c->bar, 4 * sizeof(unsigned));
  AL2(c->g, c->d * sizeof(double));
  AL2(c->step_norm, sizeof(double));
  AL2(c->status, sizeof(int));
  AL2(c->counter, sizeof(int));
  if (cudaMemsetAsync(c->status, 0, sizeof(int), c->st) != cudaSuccess) return fail(IHS_ERR_CUDA);
  c->gp = make_gram_plan((int)c->m, (int)c->d, c->prec, c->sms);
  if (c->prec == IHS_PREC_FP64) {
    AL2(c->gpart_d, gram_partial_bytes(c->gp));
  } else {
    AL2(c->gpart_f, gram_partial_bytes(c->gp));
    AL2(c->gop, gram_operand_bytes(c->gp));
  }
  if ((A->dtype == IHS_F32)) {
    AL2(c->bsplit, c->n * sizeof(float2));
    if (launch_split_b(b, c->n, c->bsplit, c->st) != cudaSuccess) return fail(IHS_ERR_CUDA);
  }
  if (c->dense) {
    c->DA = DenseA{A->val, A->n, A->d, A->ld, A->dtype == IHS_F32};
    c->srht = opt->sketch == IHS_SKETCH_SRHT;
    c->gauss = opt->sketch == IHS_SKETCH_GAUSSIAN;
    c->fused = !c->acc64 && !c->srht && !c->gauss && fused_supported(c->DA, c->s) &&
               !(opt->flags & IHS_FLAG_NO_FUSE);
    c->lookahead = c->fused && !(opt->flags & IHS_FLAG_NO_LOOKAHEAD);
    // The FP64 factor beside the pass takes a few passes' time (GB300's FP64
    // rate): form SA kFp64Depth iterations ahead, so each factor has that many
    // passes to finish, with kFp64Depth factors in flight on streams of their
    // own and kFp64Depth + 1 factor buffers.
    if (c->lookahead && !c->f32fac) {
      c->la = kFp64Depth;
      c->nbuf = kFp64Depth + 1;
      c->fac_ctas = kLookaheadFactorCtasF64;
      c->fac_slots = kFp64Depth * kLookaheadFactorCtasF64;
      if (cudaStreamCreateWithFlags(&c->st3, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_s3, cudaEventDisableTiming) != cudaSuccess)
        return fail(IHS_ERR_CUDA);
      for (int i = 0; i < kFp64Depth; ++i) {
        if (i > 0) AL2(c->fbar[i], 4 * sizeof(unsigned));
        if (cudaStreamCreateWithFlags(&c->fst[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fgo[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fend[i], cudaEventDisableTiming) != cudaSuccess)
          return fail(IHS_ERR_CUDA);
      }
      c->fbar[0] = c->bar;
    }
    // one warp per chunk; the fused pass runs two CTAs of eight warps per SM,
    // less the SMs' share left to the factors that run beside it
    const int warps = c->lookahead ? (2 * c->sms - c->fac_slots) * 8 : c->sms * 16;
    c->sp = make_sort_plan((int64_t)c->s * c->n, (int)c->m, warps);
    if ((size_t)c->m * sizeof(int32_t) > 200 * 1024) return fail(IHS_ERR_UNSUPPORTED);
    AL2(c->sort_ws, sort_workspace_bytes(c->sp));
    AL2(c->perm, c->sp.P * sizeof(uint32_t));
    AL2(c->seg, (c->m + 1) * sizeof(int32_t));
    AL2(c->chunk_first, c->sp.nchunks * sizeof(int32_t));
    AL2(c->sk_partial, (size_t)2 * c->sp.nchunks * c->d * acc_el);
    c->rg_warps = rg_dense_warps(c->n);
    AL2(c->gpart, rg_partial_bytes(c->rg_warps, c->d));
    if (c->gauss) {
      c->gplan = make_gauss_plan(c->m, c->n, (int)c->d, c->acc64, c->sms);
      AL2(c->gauss_part, c->gplan.partial_bytes);
      if (!c->acc64) {
        AL2(c->gauss_At, c->gplan.at_bytes);
        if (launch_gauss_operand(c->gplan, c->DA, c->gauss_At, c->st) != cudaSuccess)
          return fail(IHS_ERR_CUDA);
      }
    }
    if (c->srht) {
      AL2(c->srht_T, (size_t)srht_n2(c->n) * srht_ldt((int)c->d) * acc_el);
      AL2(c->srht_rows, (size_t)c->m * sizeof(int32_t));
    }
    if (c->fused) {
      AL2(c->perm2, c->sp.P * sizeof(uint32_t));
      AL2(c->seg2, (c->m + 1) * sizeof(int32_t));
      AL2(c->chunk_first2, c->sp.nchunks * sizeof(int32_t));
      AL2(c->gcta, (size_t)fused_ctas(c->sp) * c->d * sizeof(double));
    }
  } else {
    if ((size_t)(c->m / c->s) * acc_el > 200 * 1024) return fail(IHS_ERR_UNSUPPORTED);
    if ((s = build_csc(c)) != IHS_OK) return fail(s);
  }
  if (C->kind == IHS_L2_BALL) {
    AL2(c->l2buf, (size_t)(5 * c->d + 8) * sizeof(double));
    AL2(c->l2bar, 4 * sizeof(unsigned));
  }
  if (C->kind == IHS_L1_BALL || C->kind == IHS_L1_PENALTY) {
    size_t qb = qp_work_bytes((int)c->d);
    uint8_t* q;
    AL2(q, qb);
    const int64_t dd = c->d;
    c->qw.Hf = (float*)q;
    c->qw.Ls = (void*)(q + dd * dd * 4);
    c->qw.evec = (float*)(q + dd * dd * 4 + (size_t)dp * dp * 8);
    c->qw.dbuf = (double*)(q + dd * dd * 4 + (size_t)dp * dp * 8) + dd;
    c->qw.support = (int*)(c->qw.dbuf + 8 * dd);
    c->qw.iters = c->qw.support + dd + 1;
    c->qw.need = c->qw.iters + 1;
    if (C->kind == IHS_L1_PENALTY) AL2(c->qw.Hinv, (size_t)dd * dd * (c->f32fac ? 4 : 8));
    if (cudaMemsetAsync(c->qw.support, 0, (dd + 4) * sizeof(int), c->st) != cudaSuccess ||
        cudaMemsetAsync(c->qw.evec, 0, dd * sizeof(float), c->st) != cudaSuccess)
      return fail(IHS_ERR_CUDA);
  }
  {
    // launch-bound problems (A up to 128 MB) replay their solves as CUDA
    // graphs; the p = 2 ball reads scalars on the host inside its step, and
    // the serial mode exists for stage timing, so neither is captured
    const size_t el = (A->dtype == IHS_F32) ? 4 : 8;
    const size_t a_bytes =
        c->dense ? (size_t)A->n * A->ld * el
                 : (size_t)A->nnz * (el + 4) + (size_t)(A->n + 1) * (A->rowptr_i64 ? 8 : 4);
    // The penalised l1 step is left out too: its one-CTA kernels get an SM
    // only when issued ahead of the sketch chain's full-width kernels, an
    // order the streams keep and a graph does not (1,000,000 x 200 CSR, 15
    // iterations: 19.6 ms as a graph against 17.9 ms on the streams).
    c->graphs = a_bytes <= (128u << 20) && C->kind != IHS_L2_BALL &&
                C->kind != IHS_L1_PENALTY &&
                !(opt->flags & (IHS_FLAG_SERIAL | IHS_FLAG_NO_GRAPH));
    if (c->graphs) {
      AL2(c->xg, c->d * sizeof(double));
      if (cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) != cudaSuccess)
        return fail(IHS_ERR_CUDA);
    }
  }
#undef AL2
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail(IHS_ERR_CUDA);
  *out = c;
  return IHS_OK;
}

}  // extern "C"

namespace {

// Scale of the Gram of the raw SA: 1/s for the sparse embedding (entries
// +-1/sqrt(s)), 1/m for the SRHT (S = m^{-1/2} P H D) and the Gaussian
// sketch (S = G / sqrt(m)).
double gram_scale(const ihs_ctx* c) {
  return (c->srht || c->gauss) ? 1.0 / (double)c->m : 1.0 / c->s;
}

// The factor buffer after b in the rotation.
int next_buf(const ihs_ctx* c, int b) { return (b + 1) % c->nbuf; }

// The sketch chain of counter t into buffer `bf`, on the internal stream:
// draw S and sort (dense), SA, Gram (+ lambda I), Cholesky factor.  Waits
// for the last step that read buffer `bf`; records ev_fac[bf] (and
// after_gram, if given, once the Gram has read SA).  fac_ctas > 0 caps the
// factor's grid.  fstream, if given, takes the factor (after the Gram), so
// that the internal stream is free for the next chain's sketch; ev_fac[bf]
// is then recorded there.
ihs_status sketch_chain(ihs_ctx* c, int64_t t, int bf, int fac_ctas = 0,
                        cudaEvent_t after_gram = nullptr, cudaStream_t fstream = nullptr) {
  cudaStream_t s2 = (c->opt.flags & IHS_FLAG_SERIAL) ? c->st : c->st2;
  CK(cudaStreamWaitEvent(s2, c->ev_use[bf], 0));
  const SketchKeys K = make_keys(c->opt.seed, t, c->s, c->m);
  if (c->gauss) {
    stage_begin(c, IHS_ST_SKETCH, s2);
    CK(launch_gauss(c->gplan, c->DA, c->gauss_At, make_keys(c->opt.seed, t, 3, c->m).key[2],
                    c->gauss_part, c->SA, c->status, s2));
    stage_end(c);
  } else if (c->srht) {
    stage_begin(c, IHS_ST_SKETCH, s2);
    CK(launch_srht(c->DA, make_keys(c->opt.seed, t, 2, c->m), c->m, c->acc64, c->srht_T,
                   c->srht_rows, c->SA, s2));
    stage_end(c);
  } else if (c->dense) {
    stage_begin(c, IHS_ST_SORT, s2);
    CK(launch_sort_sketch(c->sp, K, c->n, c->sort_ws, c->perm, c->seg, c->chunk_first, s2));
    stage_end(c);
    stage_begin(c, IHS_ST_SKETCH, s2);
    CK(launch_sketch_dense(c->DA, c->sp, c->perm, c->seg, c->chunk_first, c->acc64, c->SA,
                           c->sk_partial, c->counter, c->sms, s2, c->prof ? c : nullptr));
    stage_end(c);
  } else {
    stage_begin(c, IHS_ST_SKETCH, s2);
    CK(launch_sketch_csc(c->CA, K, c->m, c->acc64, c->SA, c->csc_partial, s2));
    stage_end(c);
  }
  const double shift = (c->C.kind == IHS_RIDGE) ? c->C.param : 0.0;
  stage_begin(c, IHS_ST_GRAM, s2);
  CK(launch_gram(c->gp, c->SA, c->gop, c->gpart_f, c->gpart_d, gram_scale(c), shift, c->H[bf],
                 c->status, s2));
  stage_end(c);
  if (after_gram) CK(cudaEventRecord(after_gram, s2));
  cudaStream_t sf = s2;
  if (fstream) {
    CK(cudaEventRecord(c->ev_fc_go, s2));
    CK(cudaStreamWaitEvent(fstream, c->ev_fc_go, 0));
    sf = fstream;
  }
  stage_begin(c, IHS_ST_FACTOR, sf);
  CK(launch_cholesky(c->H[bf], (int)c->d, c->f32fac, c->L[bf], c->Dinv[bf], c->bar, c->status,
                     sf, (c->opt.flags & IHS_FLAG_CLUSTER) != 0, 0.0, fac_ctas));
  stage_end(c);
  CK(cudaEventRecord(c->ev_fac[bf], sf));
  return IHS_OK;
}

// The internal stream waits for everything issued so far on the caller's stream.
ihs_status join_caller(ihs_ctx* c) {
  CK(cudaEventRecord(c->ev_join, c->st));
  CK(cudaStreamWaitEvent(c->st2, c->ev_join, 0));
  return IHS_OK;
}

ihs_status gradient_on(ihs_ctx* c, const double* x, double* g, double* r, bool with_b) {
  const double lam = (c->C.kind == IHS_RIDGE) ? c->C.param : 0.0;
  if (c->dense) {
    CK(launch_resid_grad_dense(c->DA, with_b ? c->b : nullptr, with_b ? c->bsplit : nullptr, x, r,
                               c->gpart, c->rg_warps, g, lam, c->st));
  } else {
    CK(launch_resid_csr(c->n, c->d, c->A.rowptr, c->A.rowptr_i64, c->A.col, c->A.val,
                        c->A.dtype == IHS_F32, with_b ? c->b : nullptr,
                        with_b ? c->bsplit : nullptr, x, c->rbuf, r, c->st));
    CK(launch_grad_csc(c->CA, c->rbuf, c->item_part, x, lam, g, c->st));
  }
  return IHS_OK;
}

// p = 2 ball step (see l2ball.cu): the Newton point, else Newton's method on
// the secular equation, factoring H + mu I into buffer bf (its factor is not
// needed after the step) with a barrier word of its own.
ihs_status l2_step(ihs_ctx* c, double* x, int bf) {
  cudaStream_t st = c->st;
  const int d = (int)c->d;
  const double R = c->C.param;
  double* cv = c->l2buf;
  double* xm = cv + d;
  double* w = xm + d;
  double* r = w + d;
  double* du = r + d;
  double* scal = du + d;
  const int nref = c->f32fac ? 2 : 1;
  // out = (H + mu I)^{-1} rhs with the current factor, refined in FP64
  auto solve = [&](double mu, const double* rhs, double* out) -> cudaError_t {
    cudaError_t e = launch_chol_apply(c->L[bf], c->Dinv[bf], d, c->f32fac, rhs, out, st);
    for (int k = 0; k < nref && e == cudaSuccess; ++k) {
      if ((e = launch_l2_matvec(c->H[bf], d, out, mu, rhs, -1.0, r, st)) != cudaSuccess) break;
      if ((e = launch_chol_apply(c->L[bf], c->Dinv[bf], d, c->f32fac, r, du, st)) != cudaSuccess)
        break;
      e = launch_l2_axpy(out, du, d, st);
    }
    return e;
  };
  double h[2];
  CK(launch_l2_matvec(c->H[bf], d, x, 0.0, c->g, 1.0, cv, st));  // c = H x^t + g
  CK(solve(0.0, cv, xm));                                           // Newton point
  CK(launch_l2_dots(xm, xm, d, scal, st));
  CK(cudaMemcpyAsync(h, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (std::sqrt(h[0]) > R) {
    double mu = 0.0;
    for (int it = 0; it < 100; ++it) {
      if (it > 0)
        CK(launch_cholesky(c->H[bf], d, c->f32fac, c->L[bf], c->Dinv[bf], c->l2bar, c->status, st,
                           0, mu));
      if (it > 0) CK(solve(mu, cv, xm));
      CK(launch_chol_apply(c->L[bf], c->Dinv[bf], d, c->f32fac, xm, w, st));  // (H + mu I)^{-1} x
      CK(launch_l2_dots(xm, w, d, scal, st));
      CK(cudaMemcpyAsync(h, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const double nx = std::sqrt(h[0]);
      if (!(nx > 0.0) || !(h[1] > 0.0)) break;
      if (std::fabs(nx - R) <= 1e-15 * R) break;
      const double next = mu + (h[0] / h[1]) * (nx - R) / R;  // phi(mu) / phi'(mu)
      if (!(next > mu)) break;  // at the root to rounding
      mu = next;
    }
  }
  CK(launch_l2_store(xm, d, x, c->step_norm, st));
  return IHS_OK;
}

// QP step of Eq. 2 with buffer bf (gradient already in c->g), on the caller's stream.
ihs_status step_with(ihs_ctx* c, double* x, int bf) {
  CK(cudaStreamWaitEvent(c->st, c->ev_fac[bf], 0));
  stage_begin(c, IHS_ST_STEP, c->st);
  cudaError_t e;
  if (c->C.kind == IHS_L2_BALL) {
    ihs_status s = l2_step(c, x, bf);
    stage_end(c);
    if (s != IHS_OK) return s;
    CK(cudaEventRecord(c->ev_use[bf], c->st));
    return IHS_OK;
  }
  if (c->C.kind == IHS_L1_BALL || c->C.kind == IHS_L1_PENALTY)
    e = launch_l1_step(c->H[bf], c->L[bf], c->Dinv[bf], c->f32fac, (int)c->d, c->g, c->C.param,
                       c->C.kind == IHS_L1_PENALTY, c->opt.qp_max_iter, c->opt.qp_tol, c->qw, x,
                       c->step_norm, c->status, c->st);
  else
    e = launch_chol_step(c->L[bf], c->Dinv[bf], (int)c->d, c->f32fac, c->g, x, c->step_norm,
                         c->st);
  stage_end(c);
  CK(e);
  CK(cudaEventRecord(c->ev_use[bf], c->st));
  return IHS_OK;
}

// Fused pipeline, sort half: draw and sort the pairs of counter t into sort
// buffer pb on the internal stream, after the fused pass that last read it.
ihs_status fused_sort(ihs_ctx* c, int64_t t, int pb, cudaStream_t on = nullptr) {
  cudaStream_t s2 = (c->opt.flags & IHS_FLAG_SERIAL) ? c->st : (on ? on : c->st2);
  CK(cudaStreamWaitEvent(s2, c->ev_read[pb], 0));
  const SketchKeys K = make_keys(c->opt.seed, t, c->s, c->m);
  stage_begin(c, IHS_ST_SORT, s2);
  CK(launch_sort_sketch(c->sp, K, c->n, c->sort_ws, pb ? c->perm2 : c->perm, pb ? c->seg2 : c->seg,
                        pb ? c->chunk_first2 : c->chunk_first, s2));
  stage_end(c);
  CK(cudaEventRecord(c->ev_sort[pb], s2));
  return IHS_OK;
}

// Fused pipeline, main half (caller's stream): one pass over A forming SA(t)
// and g(x), then Gram, factor and step into x.
ihs_status fused_iteration(ihs_ctx* c, double* x, int pb, int bf) {
  cudaStream_t s1 = c->st;
  CK(cudaStreamWaitEvent(s1, c->ev_sort[pb], 0));
  const double lam = (c->C.kind == IHS_RIDGE) ? c->C.param : 0.0;
  stage_begin(c, IHS_ST_SKETCH, s1);
  cudaError_t e = launch_sketch_grad_fused(
      c->DA, c->sp, pb ? c->perm2 : c->perm, pb ? c->seg2 : c->seg,
      pb ? c->chunk_first2 : c->chunk_first, c->bsplit, x, (float*)c->SA, (float*)c->sk_partial,
      c->gcta, c->g, lam, s1, c->prof ? c : nullptr);
  stage_end(c);
  CK(e);
  CK(cudaEventRecord(c->ev_read[pb], s1));
  stage_begin(c, IHS_ST_GRAM, s1);
  CK(launch_gram(c->gp, c->SA, c->gop, c->gpart_f, c->gpart_d, gram_scale(c), lam, c->H[bf],
                 c->status, s1));
  stage_end(c);
  stage_begin(c, IHS_ST_FACTOR, s1);
  CK(launch_cholesky(c->H[bf], (int)c->d, c->f32fac, c->L[bf], c->Dinv[bf], c->bar, c->status,
                     s1, (c->opt.flags & IHS_FLAG_CLUSTER) != 0));
  stage_end(c);
  CK(cudaEventRecord(c->ev_fac[bf], s1));
  return step_with(c, x, bf);
}

// Look-ahead fused pipeline, depth la (1, or 2 with the FP64 factor).  Pass
// k (caller's stream) reads A once for the gradient at x^k and SA of counter
// t0+k+la; the Gram and factor of that counter then run on the internal
// stream beside the steps and passes of the next la iterations (the factor
// on kLookaheadFactorCtas CTAs, the slots the pass leaves free).  Counters
// t0 .. t0+la-1 take sketch-only passes first (their chains on the internal
// stream); the last la passes form the gradient only, in the row order of the
// last sort, so SA, H and the factor left behind are the last iteration's,
// as in the other loops.  Sort buffer u&1 holds counter t0+u for u >= la;
// the sort of t0+k+la+2 follows the Gram and factor of pass k on the
// internal stream.  Counter t0+j uses factor buffer fb(j) of the rotation.
ihs_status fused_lookahead(ihs_ctx* c, double* x, int64_t t0, int iters) {
  const bool serial = (c->opt.flags & IHS_FLAG_SERIAL) != 0;
  cudaStream_t s1 = c->st, s2 = serial ? c->st : c->st2;
  const int fac_ctas = serial ? 0 : c->fac_ctas;
  const double lam = (c->C.kind == IHS_RIDGE) ? c->C.param : 0.0;
  const int la = c->la;
  const int b0 = next_buf(c, c->cur);
  auto fb = [&](int j) { return (b0 + j) % c->nbuf; };
  ihs_status s;
  const int pre = std::min(la, iters);
  for (int j = 0; j < pre; ++j)
    if ((s = sketch_chain(c, t0 + j, fb(j), fac_ctas, c->ev_gram)) != IHS_OK) return s;
  CK(cudaEventRecord(c->ev_read[0], s2));  // the sketch-only passes read sort buffer 0
  // FP64 factors (depth kFp64Depth): the sorts on st3 and the factors going
  // round fst[0 .. la-1], so that neither a sort nor the next factor queues
  // behind a factor; those streams start after everything on st2 so far.
  // Depth 1 keeps the sorts and the factors on st2 (a concurrent sort slows
  // the pass more than it gains).
  const bool multi = !serial && la >= 2 && c->fst[la - 1];
  cudaStream_t s3 = multi ? c->st3 : s2;
  if (multi) {
    CK(cudaEventRecord(c->ev_s3, s2));
    CK(cudaStreamWaitEvent(s3, c->ev_s3, 0));
    for (int i = 0; i < la; ++i) CK(cudaStreamWaitEvent(c->fst[i], c->ev_s3, 0));
  }
  for (int u = la; u < std::min(iters, la + 2); ++u)
    if ((s = fused_sort(c, t0 + u, u & 1, s3)) != IHS_OK) return s;
  // the gradient-only passes read the last counter's sort (buffer 0 when
  // every counter came from a sketch-only pass)
  const int last_pb = iters > la ? (iters - 1) & 1 : 0;
  for (int k = 0; k < iters; ++k) {
    const bool ahead = k + la < iters;
    const int pb = ahead ? (k + la) & 1 : last_pb;
    if (ahead) CK(cudaStreamWaitEvent(s1, c->ev_sort[pb], 0));
    else if (iters > la) CK(cudaStreamWaitEvent(s1, c->ev_sort[pb], 0));
    else CK(cudaStreamWaitEvent(s1, c->ev_read[0], 0));  // the sketch-only passes' sorts
    CK(cudaStreamWaitEvent(s1, c->ev_gram, 0));  // SA no longer needed by the last Gram
    // timed as the gradient stage: the sketch stage is the sketch-only pass
    stage_begin(c, IHS_ST_GRAD, s1);
    cudaError_t e = launch_sketch_grad_fused(
        c->DA, c->sp, pb ? c->perm2 : c->perm, pb ? c->seg2 : c->seg,
        pb ? c->chunk_first2 : c->chunk_first, c->bsplit, x, (float*)c->SA,
        (float*)c->sk_partial, c->gcta, c->g, lam, s1, c->prof ? c : nullptr, ahead);
    stage_end(c);
    CK(e);
    CK(cudaEventRecord(c->ev_read[pb], s1));
    if (ahead) {
      const int nb = fb(k + la);  // factor buffer of counter t0+k+la
      CK(cudaEventRecord(c->ev_sa, s1));
      CK(cudaStreamWaitEvent(s2, c->ev_sa, 0));
      CK(cudaStreamWaitEvent(s2, c->ev_use[nb], 0));  // the last step that read buffer nb
      stage_begin(c, IHS_ST_GRAM, s2);
      CK(launch_gram(c->gp, c->SA, c->gop, c->gpart_f, c->gpart_d, gram_scale(c), lam,
                     c->H[nb], c->status, s2));
      stage_end(c);
      CK(cudaEventRecord(c->ev_gram, s2));
      cudaStream_t sf = s2;
      unsigned* fbar = c->bar;
      if (multi) {
        const int q = k % la;
        sf = c->fst[q];
        fbar = c->fbar[q];
        CK(cudaEventRecord(c->ev_fgo[q], s2));
        CK(cudaStreamWaitEvent(sf, c->ev_fgo[q], 0));
      }
      stage_begin(c, IHS_ST_FACTOR, sf);
      CK(launch_cholesky(c->H[nb], (int)c->d, c->f32fac, c->L[nb], c->Dinv[nb], fbar,
                         c->status, sf, (c->opt.flags & IHS_FLAG_CLUSTER) != 0, 0.0, fac_ctas));
      stage_end(c);
      CK(cudaEventRecord(c->ev_fac[nb], sf));
      if (k + la + 2 < iters && (s = fused_sort(c, t0 + k + la + 2, pb, s3)) != IHS_OK) return s;
    }
    if ((s = step_with(c, x, fb(k))) != IHS_OK) return s;
    c->cur = fb(k);
  }
  if (multi) {  // st2 ends after the last sort and factors (every join of st2 covers them)
    CK(cudaEventRecord(c->ev_s3, s3));
    CK(cudaStreamWaitEvent(s2, c->ev_s3, 0));
    for (int i = 0; i < la; ++i) {
      CK(cudaEventRecord(c->ev_fend[i], c->fst[i]));
      CK(cudaStreamWaitEvent(s2, c->ev_fend[i], 0));
    }
  }
  return IHS_OK;
}

// The solve's work (iterations t0 .. t0+iters-1), issued on the context's
// streams; ihs_solve synchronises afterwards.
ihs_status issue_solve(ihs_ctx* c, double* x, int64_t t0, int iters) {
  if (c->qw.iters) {
    CK(cudaMemsetAsync(c->qw.iters, 0, sizeof(int), c->st));
    CK(cudaMemsetAsync(c->qw.need + 1, 0, sizeof(int), c->st));
  }
  ihs_status s = IHS_OK;
  if (iters > 0 && c->lookahead) {
    if ((s = join_caller(c)) != IHS_OK) return s;
    if ((s = fused_lookahead(c, x, t0, iters)) != IHS_OK) return s;
    c->have_sketch = true;
  } else if (iters > 0 && c->fused) {
    if ((s = join_caller(c)) != IHS_OK) return s;
    if ((s = fused_sort(c, t0, 0)) != IHS_OK) return s;
    int bf = next_buf(c, c->cur);
    for (int k = 0; k < iters; ++k) {
      const int pb = k & 1;
      if (k + 1 < iters && (s = fused_sort(c, t0 + k + 1, pb ^ 1)) != IHS_OK) return s;
      if ((s = fused_iteration(c, x, pb, bf)) != IHS_OK) return s;
      c->cur = bf;
      bf = next_buf(c, bf);
    }
    c->have_sketch = true;
  } else if (iters > 0) {
    if ((s = join_caller(c)) != IHS_OK) return s;
    // the factors on their own stream (joined back into st2 at the end)
    cudaStream_t fs = (c->opt.flags & IHS_FLAG_SERIAL) ? nullptr : c->fchain;
    int bf = next_buf(c, c->cur);
    if ((s = sketch_chain(c, t0, bf, 0, nullptr, fs)) != IHS_OK) return s;
    // The chain of t+1 starts once the gradient pass of t is done, and is
    // issued after the step of t: a gradient pass sharing the GPU with a
    // full-width sketch kernel runs several times slower, and the one-CTA
    // l1 step needs a whole SM, which it gets only if launched first
    // (measured again with the one-CTA-per-chunk CSC sketch: without this
    // wait the 1e7 x 1000 LASSO solve takes 65.9 ms against 42.5 ms).
    for (int k = 0; k < iters; ++k) {
      stage_begin(c, IHS_ST_GRAD, c->st);
      s = gradient_on(c, x, c->g, nullptr, true);
      stage_end(c);
      if (s != IHS_OK) return s;
      CK(cudaEventRecord(c->ev_grad, c->st));
      if ((s = step_with(c, x, bf)) != IHS_OK) return s;
      if (k + 1 < iters) {
        CK(cudaStreamWaitEvent(c->st2, c->ev_grad, 0));
        if ((s = sketch_chain(c, t0 + k + 1, next_buf(c, bf), 0, nullptr, fs)) != IHS_OK)
          return s;
      }
      c->cur = bf;
      bf = next_buf(c, bf);
    }
    if (fs) {
      CK(cudaEventRecord(c->ev_fc_end, fs));
      CK(cudaStreamWaitEvent(c->st2, c->ev_fc_end, 0));
    }
    c->have_sketch = true;
  }
  return s;
}

// Record every event a wait of the solve can name on stream st.  Inside a
// capture this makes each later wait refer to a record within the graph;
// outside, it replaces records made inside a capture (which a wait outside
// the graph may not name) by records ordered after the graph.
cudaError_t record_solve_events(ihs_ctx* c, cudaStream_t st) {
  cudaEvent_t evs[] = {c->ev_join,    c->ev_grad,    c->ev_sa,      c->ev_gram,   c->ev_tail2,
                       c->ev_s3,      c->ev_sort[0], c->ev_sort[1], c->ev_read[0], c->ev_read[1],
                       c->ev_fc_go,   c->ev_fc_end};
  cudaError_t e = cudaSuccess;
  for (cudaEvent_t ev : evs)  // (the FP64-factor pipeline's events exist only there)
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev, st);
  for (int i = 0; i < kFp64Depth && e == cudaSuccess; ++i) {
    if (c->ev_fgo[i]) e = cudaEventRecord(c->ev_fgo[i], st);
    if (c->ev_fend[i] && e == cudaSuccess) e = cudaEventRecord(c->ev_fend[i], st);
  }
  for (int k = 0; k < kFacBufs && e == cudaSuccess; ++k) {
    e = cudaEventRecord(c->ev_fac[k], st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_use[k], st);
  }
  return e;
}

// The solve as a CUDA graph: captured on the first call with a given (t0,
// iters) and replayed afterwards, on the internal copy xg of the iterate and
// on an internal stream (the caller's may be the legacy default stream,
// which cannot be captured), ordered after the caller's stream and the
// internal stream and joined back into the caller's.  Every event a wait in
// the solve can name is recorded again at the start of the capture, so each
// wait refers to a record inside the graph.  If the capture or the
// instantiation fails, graphs are turned off for the context and the solve
// is issued on the streams.
ihs_status solve_graph(ihs_ctx* c, double* x, int64_t t0, int iters) {
  const size_t xb = (size_t)c->d * sizeof(double);
  cudaStream_t caller = c->st, gs = c->gst;
  CK(cudaEventRecord(c->ev_join, caller));
  CK(cudaStreamWaitEvent(gs, c->ev_join, 0));
  CK(cudaEventRecord(c->ev_tail2, c->st2));
  CK(cudaStreamWaitEvent(gs, c->ev_tail2, 0));
  CK(cudaMemcpyAsync(c->xg, x, xb, cudaMemcpyDeviceToDevice, gs));
  if (!(c->gexec && c->g_t0 == t0 && c->g_iters == iters)) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    const int cur0 = c->cur;
    c->st = gs;  // the solve's "caller's stream" while capturing
    bool ok = cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
      ihs_status s = IHS_OK;
      ok = record_solve_events(c, gs) == cudaSuccess;
      if (ok) s = issue_solve(c, c->xg, t0, iters);
      // join the internal stream back
      ok = ok && s == IHS_OK && cudaEventRecord(c->ev_tail2, c->st2) == cudaSuccess &&
           cudaStreamWaitEvent(gs, c->ev_tail2, 0) == cudaSuccess;
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(gs, &g);
      ok = ok && e == cudaSuccess && g != nullptr;
      if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
    }
    c->st = caller;
    if (!ok) {
      cudaGetLastError();
      if (c->gexec) cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
      c->graphs = false;
      c->cur = cur0;
      CK(cudaStreamSynchronize(gs));
      CK(record_solve_events(c, caller));
      return issue_solve(c, x, t0, iters);
    }
    c->g_t0 = t0;
    c->g_iters = iters;
    c->g_cur_end = c->cur;
  }
  CK(cudaGraphLaunch(c->gexec, gs));
  CK(record_solve_events(c, gs));
  c->last_graph = true;
  c->cur = c->g_cur_end;
  c->have_sketch = true;
  CK(cudaMemcpyAsync(x, c->xg, xb, cudaMemcpyDeviceToDevice, gs));
  // the caller's stream continues after the graph
  CK(cudaEventRecord(c->ev_join, gs));
  CK(cudaStreamWaitEvent(caller, c->ev_join, 0));
  return IHS_OK;
}

}  // namespace

extern "C" {

ihs_status ihs_sketch(ihs_ctx* c, int64_t t) {
  if (!c || t < 0) return IHS_ERR_ARG;
  ihs_status s = join_caller(c);
  if (s != IHS_OK) return s;
  const int bf = next_buf(c, c->cur);
  if ((s = sketch_chain(c, t, bf)) != IHS_OK) return s;
  c->cur = bf;
  c->have_sketch = true;
  return IHS_OK;
}

ihs_status ihs_gradient(ihs_ctx* c, const double* x, double* g, double* r) {
  if (!c || !x || !g) return IHS_ERR_ARG;
  return gradient_on(c, x, g, r, true);
}

ihs_status ihs_sketch_gradient(ihs_ctx* c, int64_t t, const double* x, double* g) {
  if (!c || t < 0 || !x || !g) return IHS_ERR_ARG;
  if (!c->fused) {
    ihs_status s = ihs_sketch(c, t);
    if (s != IHS_OK) return s;
    return gradient_on(c, x, g, nullptr, true);
  }
  // Everything on the caller's stream, after what the internal stream holds
  // (a sketch chain may still be writing the sort buffers or SA).
  cudaStream_t st = c->st;
  CK(cudaEventRecord(c->ev_tail2, c->st2));
  CK(cudaStreamWaitEvent(st, c->ev_tail2, 0));
  const int bf = next_buf(c, c->cur);
  CK(cudaStreamWaitEvent(st, c->ev_use[bf], 0));
  const double lam = (c->C.kind == IHS_RIDGE) ? c->C.param : 0.0;
  const SketchKeys K = make_keys(c->opt.seed, t, c->s, c->m);
  stage_begin(c, IHS_ST_SORT, st);
  CK(launch_sort_sketch(c->sp, K, c->n, c->sort_ws, c->perm, c->seg, c->chunk_first, st));
  stage_end(c);
  stage_begin(c, IHS_ST_SKETCH, st);
  cudaError_t e = launch_sketch_grad_fused(c->DA, c->sp, c->perm, c->seg, c->chunk_first,
                                           c->bsplit, x, (float*)c->SA, (float*)c->sk_partial,
                                           c->gcta, g, lam, st, c->prof ? c : nullptr, true);
  stage_end(c);
  CK(e);
  CK(cudaEventRecord(c->ev_read[0], st));
  stage_begin(c, IHS_ST_GRAM, st);
  CK(launch_gram(c->gp, c->SA, c->gop, c->gpart_f, c->gpart_d, gram_scale(c), lam, c->H[bf],
                 c->status, st));
  stage_end(c);
  stage_begin(c, IHS_ST_FACTOR, st);
  CK(launch_cholesky(c->H[bf], (int)c->d, c->f32fac, c->L[bf], c->Dinv[bf], c->bar, c->status,
                     st, (c->opt.flags & IHS_FLAG_CLUSTER) != 0));
  stage_end(c);
  CK(cudaEventRecord(c->ev_fac[bf], st));
  c->cur = bf;
  c->have_sketch = true;
  return IHS_OK;
}

ihs_status ihs_step(ihs_ctx* c, double* x) {
  if (!c || !x) return IHS_ERR_ARG;
  if (!c->have_sketch) return IHS_ERR_ARG;
  stage_begin(c, IHS_ST_GRAD, c->st);
  ihs_status s = gradient_on(c, x, c->g, nullptr, true);
  stage_end(c);
  if (s != IHS_OK) return s;
  return step_with(c, x, c->cur);
}

ihs_status ihs_sync(ihs_ctx* c) {
  if (!c) return IHS_ERR_ARG;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaStreamSynchronize(c->st2));
  int st = 0;
  CK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) CK(cudaMemset(c->status, 0, sizeof(int)));
  return (ihs_status)st;
}

// Pipelined loop: the sketch chain of t+1 (internal stream) is issued before
// the step of t (caller's stream), so it overlaps with the gradient pass and
// the step; double buffering keeps the step's factor intact.
ihs_status ihs_solve(ihs_ctx* c, double* x, int64_t t0, int iters, ihs_report* rep) {
  if (!c || !x || iters < 0 || t0 < 0) return IHS_ERR_ARG;
  c->last_graph = false;
  ihs_status s = (iters > 0 && c->graphs && !c->prof) ? solve_graph(c, x, t0, iters)
                                                      : issue_solve(c, x, t0, iters);
  if (s != IHS_OK) return s;
  ihs_status st = ihs_sync(c);
  if (rep) {
    rep->iters = iters;
    rep->status = st;
    rep->step_norm = 0.0;
    rep->qp_fista_iters = 0;
    rep->qp_active_rounds = 0;
    rep->graph = c->last_graph ? 1 : 0;
    if (iters > 0) cudaMemcpy(&rep->step_norm, c->step_norm, sizeof(double), cudaMemcpyDeviceToHost);
    if (c->qw.iters) {
      cudaMemcpy(&rep->qp_fista_iters, c->qw.iters, sizeof(int), cudaMemcpyDeviceToHost);
      cudaMemcpy(&rep->qp_active_rounds, c->qw.need + 1, sizeof(int), cudaMemcpyDeviceToHost);
    }
  }
  return st;
}

ihs_status ihs_get_sketch(ihs_ctx* c, void* SA_out, int* SA_dtype, double* H_out,
                          double* scale) {
  if (!c) return IHS_ERR_ARG;
  if (SA_dtype) *SA_dtype = c->acc64 ? IHS_F64 : IHS_F32;
  if (scale) *scale = gram_scale(c);
  if ((SA_out || H_out) && !c->have_sketch) return IHS_ERR_ARG;
  const size_t el = c->acc64 ? 8 : 4;
  CK(cudaStreamWaitEvent(c->st, c->ev_fac[c->cur], 0));
  if (SA_out)
    CK(cudaMemcpyAsync(SA_out, c->SA, (size_t)c->m * c->d * el, cudaMemcpyDeviceToDevice, c->st));
  if (H_out)
    CK(cudaMemcpyAsync(H_out, c->H[c->cur], (size_t)c->d * c->d * sizeof(double),
                       cudaMemcpyDeviceToDevice, c->st));
  return IHS_OK;
}

ihs_status ihs_selftest_wait(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* bar = nullptr;
  if (cudaMalloc(&bar, 4 * sizeof(unsigned) + sizeof(int)) != cudaSuccess) return IHS_ERR_OOM;
  int* status = reinterpret_cast<int*>(bar + 4);
  int h = -1;
  cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned) + sizeof(int), st);
  if (e == cudaSuccess) e = launch_barrier_selftest(bar, status, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(bar);
  if (e != cudaSuccess) return IHS_ERR_CUDA;
  return (ihs_status)h;
}

ihs_status ihs_selftest_rsqrt(const double* p, double* out, double* ref, int64_t n,
                              void* stream) {
  if (n <= 0) return IHS_OK;
  if (!p || !out || !ref) return IHS_ERR_ARG;
  if (launch_selftest_rsqrt(p, out, ref, n, (cudaStream_t)stream) != cudaSuccess)
    return IHS_ERR_CUDA;
  return IHS_OK;
}

ihs_status ihs_trim_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int k = 0; k < kMaxDevices; ++k)
    if (g_pool[k]) CK(cudaMemPoolTrimTo(g_pool[k], 0));
  return IHS_OK;
}

ihs_status ihs_exact_gram(ihs_ctx* c, double* G) {
  if (!c || !G) return IHS_ERR_ARG;
  const int d = (int)c->d;
  if (c->dense) {
    const GramPlan g = make_gram_plan((int)std::min<int64_t>(c->n, 0x7fffffff), d, IHS_PREC_FP64,
                                      c->sms);
    const size_t need = gram_partial_bytes(g);
    if (c->xg_bytes < need) {
      ihs_status s = dalloc(c, &c->xg_part, need);
      if (s != IHS_OK) return s;
      c->xg_bytes = need;
    }
    CK(launch_exact_gram_dense(c->A.val, c->A.dtype == IHS_F32, c->n, d, c->A.ld, c->sms,
                               c->xg_part, c->xg_bytes, G, c->status, c->st));
  } else {
    CK(launch_exact_gram_csr(c->n, d, c->A.rowptr, c->A.rowptr_i64, c->A.col, c->A.val,
                             c->A.dtype == IHS_F32, G, c->st));
  }
  return IHS_OK;
}

ihs_status ihs_sketch_error(ihs_ctx* c, int64_t t, const double* G, double* err) {
  if (!c || !G || !err || t < 0) return IHS_ERR_ARG;
  if (!c->errbuf) {
    ihs_status s = dalloc(c, &c->errbuf, sizeof(double));
    if (s != IHS_OK) return s;
  }
  ihs_status s = ihs_sketch(c, t);
  if (s != IHS_OK) return s;
  CK(cudaStreamWaitEvent(c->st, c->ev_fac[c->cur], 0));
  CK(launch_fro_ratio(c->H[c->cur], G, c->d * c->d, c->errbuf, c->st));
  CK(cudaMemcpyAsync(err, c->errbuf, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return ihs_sync(c);
}

ihs_status ihs_adjoint(ihs_ctx* c, const double* x, const double* dLdx, double* dLdb, void* dLdA,
                       ihs_report* rep) {
  if (!c || !x || !dLdx) return IHS_ERR_ARG;
  if (c->C.kind == IHS_L1_BALL || c->C.kind == IHS_L1_PENALTY || c->C.kind == IHS_L2_BALL)
    return IHS_ERR_UNSUPPORTED;
  if (!c->have_sketch) return IHS_ERR_ARG;
  if (dLdA && !c->dense) return IHS_ERR_UNSUPPORTED;
  const int d = (int)c->d;
  if (!c->cg) {
    ihs_status s = dalloc(c, &c->cg, (size_t)(5 * d + 8) * sizeof(double));
    if (s != IHS_OK) return s;
  }
  double *v = c->cg, *r = v + d, *z = r + d, *p = z + d, *q = p + d, *scal = q + d;
  const int bf = c->cur;
  CK(cudaStreamWaitEvent(c->st, c->ev_fac[bf], 0));
  // PCG on (A^T A + lambda I) v = dL/dx with preconditioner (L L^T)^{-1}
  CK(launch_cg_init(dLdx, d, v, r, scal, c->st));
  double h[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(h, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const double rhs2 = h[2];
  const double tol2 = 1e-26 * rhs2;  // |r| <= 1e-13 |dL/dx|
  int it = 0;
  bool conv = (rhs2 == 0.0);
  const int max_it = 200;
  while (!conv && it < max_it) {
    CK(launch_chol_apply(c->L[bf], c->Dinv[bf], d, c->f32fac, r, z, c->st));
    CK(launch_cg_dir(r, z, d, p, scal, it == 0, c->st));
    ihs_status s = gradient_on(c, p, q, nullptr, false);  // q = -(A^T A + lambda I) p
    if (s != IHS_OK) return s;
    CK(launch_cg_step(p, q, d, v, r, scal, c->st));
    ++it;
    double rr = 0.0;
    CK(cudaMemcpyAsync(&rr, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    conv = rr <= tol2;
  }
  CK(cudaEventRecord(c->ev_use[bf], c->st));
  // dL/db = A v  (the residual pass with b = 0 gives -A v)
  if (dLdb) {
    ihs_status s = gradient_on(c, v, q, dLdb, false);
    if (s != IHS_OK) return s;
    CK(launch_negate(dLdb, c->n, c->st));
  }
  if (dLdA) CK(launch_adjoint_dA(c->DA, c->b, x, v, dLdA, c->st));
  ihs_status st = ihs_sync(c);
  if (rep) {
    rep->iters = it;
    rep->status = st;
    rep->qp_fista_iters = 0;
    rep->qp_active_rounds = 0;
    rep->step_norm = 0.0;
    rep->graph = 0;
  }
  if (st != IHS_OK) return st;
  return conv ? IHS_OK : IHS_ERR_NOT_CONVERGED;
}

ihs_status ihs_profile(ihs_ctx* c, int enable) {
  if (!c) return IHS_ERR_ARG;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaStreamSynchronize(c->st2));
  c->pe.used = 0;
  for (int k = 0; k < IHS_NSTAGES; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_cnt[k] = 0;
  }
  c->prof = enable != 0;
  c->prof_launch0 = launches_total();
  return IHS_OK;
}

ihs_status ihs_profile_read(ihs_ctx* c, double* ms, int* count, int64_t* launches) {
  if (!c || !ms) return IHS_ERR_ARG;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaStreamSynchronize(c->st2));
  stage_collect(c);
  for (int k = 0; k < IHS_NSTAGES; ++k) {
    ms[k] = c->prof_ms[k];
    if (count) count[k] = c->prof_cnt[k];
  }
  if (launches) *launches = launches_total() - c->prof_launch0;
  return IHS_OK;
}

ihs_status ihs_hash(uint64_t seed, int64_t t, int s, int64_t m, int64_t n, int32_t* bucket,
                    int8_t* sign, void* stream) {
  if (s < 1 || s > kMaxBlocks || m < 1 || m % s != 0 || n < 0 || t < 0) return IHS_ERR_ARG;
  if (m / s > 0x7fffffffLL || m > 0x7fffffffLL) return IHS_ERR_ARG;
  if (n > 0 && (!bucket || !sign)) return IHS_ERR_ARG;
  const SketchKeys K = make_keys(seed, t, s, m);
  CK(launch_hash(K, n, bucket, sign, (cudaStream_t)stream));
  return IHS_OK;
}

ihs_status ihs_sketch_adjoint(uint64_t seed, int64_t t, int s, int64_t m, int64_t n, int64_t d,
                              const double* G, double* out, void* stream) {
  if (s < 1 || s > kMaxBlocks || m < 1 || m % s != 0 || n < 0 || d < 1 || t < 0)
    return IHS_ERR_ARG;
  if (n > 0 && (!G || !out)) return IHS_ERR_ARG;
  const SketchKeys K = make_keys(seed, t, s, m);
  CK(launch_sketch_adjoint(K, n, d, G, out, (cudaStream_t)stream));
  return IHS_OK;
}

}  // extern "C"
