// internal.h -- host-side launchers shared between the translation units of
// libihs.so.  Nothing here is part of the public ABI (include/ihs.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

// Kernel launches issued by the library (for the profiler's launch count).
void note_launches(int k);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device (the attribute is per device; set once per kernel and
// device, thread-safe).
cudaError_t ensure_smem(const void* fn, int bytes);
int64_t launches_total();

// ---- sketch draw ----------------------------------------------------------
SketchKeys make_keys(uint64_t seed, int64_t t, int s, int64_t m);
cudaError_t launch_hash(const SketchKeys& K, int64_t n, int32_t* bucket, int8_t* sign,
                        cudaStream_t st);

// ---- stable counting sort of (block, row) pairs by global bucket ------------
// Keys come either from the sketch draw (pairs p = k*n + i) or from an int32
// key array (used once to build the CSC copy of a CSR matrix).
struct SortPlan {
  int64_t P = 0;       // number of items
  int m = 0;           // number of buckets
  int tile = 0;        // items per tile
  int ntiles = 0;
  int64_t chunk = 0;   // reduce-chunk size (items) for the segmented reduce
  int nchunks = 0;
};
SortPlan make_sort_plan(int64_t P, int m, int nchunks_target);
size_t sort_workspace_bytes(const SortPlan& p);
// perm[pos] = payload, seg_start[m+1], chunk_first[nchunks]: first bucket whose
// segment contains the chunk's first item.
cudaError_t launch_sort_sketch(const SortPlan& p, const SketchKeys& K, int64_t n, void* ws,
                               uint32_t* perm, int32_t* seg_start, int32_t* chunk_first,
                               cudaStream_t st);
cudaError_t launch_sort_keys(const SortPlan& p, const int32_t* keys, void* ws, uint32_t* perm,
                             int32_t* seg_start, cudaStream_t st);

// ---- sketch SA = S A ---------------------------------------------------------
struct DenseA {
  const void* val;
  int64_t n, d, ld;
  int f32;  // 1: float values, 0: double
};
// SA is m x d row-major in Tacc (double if acc64 else float); partial holds
// 2 * nchunks * d accumulators.
cudaError_t launch_sketch_dense(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                                const int32_t* seg_start, const int32_t* chunk_first, int acc64,
                                void* SA, void* partial, int* counter, int sms, cudaStream_t st,
                                void* prof = nullptr);
// Stage boundaries for the profiler (no-ops when prof is null).
void prof_stage_begin(void* prof, int stage);
void prof_stage_end(void* prof);

struct CscA {
  int64_t n, d, nnz;
  const int64_t* colptr;   // d + 1
  const int32_t* rowidx;   // nnz, ascending within a column
  const void* val;         // nnz
  int f32;
  // work items: column chunks of at most `chunk` entries
  int nitems;
  const int32_t* item_col;     // nitems
  const int64_t* item_begin;   // nitems
  const int64_t* item_end;     // nitems
  const int32_t* item_slot;    // nitems: -1 if the column has one item, else partial slot
  int nsplit_slots;
  const int32_t* col_first_item;  // d + 1 (items of column j: [first[j], first[j+1]))
};
cudaError_t launch_sketch_csc(const CscA& A, const SketchKeys& K, int64_t m, int acc64, void* SA,
                              void* partial, cudaStream_t st);

cudaError_t launch_sketch_fixup_f32(const SortPlan& p, const int32_t* seg, int d,
                                    const float* partial, float* SA, cudaStream_t st);
// One pass over a dense FP32 A forming SA (FP32 accumulation, CountSketch)
// and g = A^T (b - A x) - lam x together; gcta holds fused_ctas(p) * d doubles.
bool fused_supported(const DenseA& A, int s);
int fused_ctas(const SortPlan& p);
cudaError_t launch_sketch_grad_fused(const DenseA& A, const SortPlan& p, const uint32_t* perm,
                                     const int32_t* seg, const int32_t* cf, const float2* bsplit,
                                     const double* x, float* SA, float* partial, double* gcta,
                                     double* g, double lam, cudaStream_t st, void* prof,
                                     bool form_sa = true);

// S^T G gather (G m x d double, out n x d double).
cudaError_t launch_sketch_adjoint(const SketchKeys& K, int64_t n, int64_t d, const double* G,
                                  double* out, cudaStream_t st);

// ---- residual and gradient ----------------------------------------------------
// Dense: g = A^T (b - A x) with FP64-class accuracy; gpart has nwarps*d doubles.
int rg_dense_warps(int64_t n);
// bytes of the dense gradient's partial buffer for nwarps warps (the warp
// partials, then the reduce's slice sums)
size_t rg_partial_bytes(int nwarps, int64_t d);
cudaError_t launch_resid_grad_dense(const DenseA& A, const double* b, const float2* bsplit,
                                    const double* x, double* r, double* gpart, int nwarps,
                                    double* g, double lam, cudaStream_t st);
// CSR rows -> r (stored as double for FP64 values, float2 (hi, lo) for FP32);
// CSC columns -> g.
cudaError_t launch_resid_csr(int64_t n, int64_t d, const void* rowptr, int rowptr_i64,
                             const int32_t* col, const void* val, int f32, const double* b,
                             const float2* bsplit, const double* x, void* rbuf, double* r_out,
                             cudaStream_t st);
cudaError_t launch_grad_csc(const CscA& A, const void* rbuf, double* item_part, const double* x,
                            double lam, double* g, cudaStream_t st);
// g[c] = sum over parts (fixed order) of part[p][c] - lam x[c].
cudaError_t launch_reduce_partials(const double* part, int nparts, int d, const double* x,
                                   double lam, double* g, cudaStream_t st);

// ---- Gram ---------------------------------------------------------------------
struct GramPlan {
  int d = 0, m = 0;
  int prec = 0;            // IHS_PREC_*
  int tiles = 0;           // lower-triangle output tiles
  int tdim = 0;            // output tile edge
  int splits = 0;          // split-K factor
  int64_t ldt = 0;         // leading dimension of the transposed operand (elements)
};
GramPlan make_gram_plan(int m, int d, int prec, int num_sms);
size_t gram_partial_bytes(const GramPlan& g);
size_t gram_operand_bytes(const GramPlan& g);
// SA (m x d, double for FP64, float otherwise) -> H (d x d double, full)
// Exact FP64 Gram A^T A (dense: deterministic split-K; CSR: FP64 atomics) and
// the ratio ||H - G||_F / ||G||_F into out[0] (device).
cudaError_t launch_exact_gram_dense(const void* A, int f32, int64_t n, int d, int64_t lda,
                                    int num_sms, double* partial, size_t partial_bytes, double* G,
                                    int* status, cudaStream_t st);
cudaError_t launch_exact_gram_csr(int64_t n, int d, const void* rowptr, int rowptr_i64,
                                  const int32_t* col, const void* val, int f32, double* G,
                                  cudaStream_t st);
cudaError_t launch_fro_ratio(const double* H, const double* G, int64_t count, double* out,
                             cudaStream_t st);
cudaError_t launch_gram(const GramPlan& g, const void* SA, void* operand, float* partial_f,
                        double* partial_d, double scale, double shift, double* H, int* status,
                        cudaStream_t st);

// ---- dense d x d linear algebra -------------------------------------------------
int chol_padded(int d);  // d rounded up to the 32-tile
// Lbuf: dp x dp (lower: L, upper: L^T tiles); Dinv: dp/32 tiles of 32 x 32;
// bar: 4 unsigned of barrier state (zeroed by the launcher).
size_t chol_dinv_bytes(int d, int f32);
// Factor H + shift I with the 16-CTA cluster kernel when allow_cluster (and
// shift == 0) and the matrix fits in the cluster's shared memory, else with
// the cooperative grid kernel (the two give identical factors).  max_ctas > 0
// caps the grid kernel's CTAs (the factor then leaves the other SMs to a
// kernel running beside it).
cudaError_t launch_selftest_rsqrt(const double* p, double* out, double* ref, int64_t n,
                                  cudaStream_t st);
cudaError_t launch_cholesky(const double* H, int d, int f32, void* Lbuf, void* Dinv, unsigned* bar,
                            int* status, cudaStream_t st, int allow_cluster, double shift = 0.0,
                            int max_ctas = 0);
// x += (L L^T)^{-1} g ; step_norm (device double) gets max |delta|.
cudaError_t launch_chol_step(const void* Lbuf, const void* Dinv, int d, int f32, const double* g,
                             double* x, double* step_norm, cudaStream_t st);
// delta = (L L^T)^{-1} v (no update), for preconditioning.
// H^{-1} (d x d, factor precision) from the factor, skipped when need && !*need;
// the shared memory it needs (must be <= 220 KB: FP32 any d <= 1024, FP64 d <= 832).
// Two CTAs wait at a grid barrier that expects three, with a 4096-poll
// limit: each gives up and records DEV_TIMEOUT in *status (bar: 4 zeroed words).
cudaError_t launch_barrier_selftest(unsigned* bar, int* status, cudaStream_t st);
size_t chol_inverse_smem_bytes(int d, int f32);
cudaError_t launch_chol_inverse(const void* Lbuf, const void* Dinv, int d, int f32, void* Hinv,
                                const int* need, cudaStream_t st);
cudaError_t launch_chol_apply(const void* Lbuf, const void* Dinv, int d, int f32, const double* v,
                              double* out, cudaStream_t st);

// l1-ball QP step (Eq. 2 over {||x||_1 <= R}); H double d x d.
struct QpWork {
  float* Hf;       // d x d float copy of H
  float* evec;     // d floats: top eigenvector estimate of H, kept across steps
                   // (zero at creation: the power iteration then starts cold)
  void* Ls;        // support Cholesky (dp x dp, double)
  int* support;    // d ints, previous face (count in support[d])
  double* dbuf;    // 8 * d doubles of scratch
  int* iters;      // FISTA iterations (device counter)
  int* need;       // penalised form: the step is still open after the previous pass;
                   // need[1]: active-set rounds spent (device counter)
  void* Hinv;      // penalised form: H^{-1} (d x d, factor precision), or null
};
size_t qp_work_bytes(int d);
// The l1 step of Eq. 2: over the ball ||x||_1 <= param (pen = 0) or with the
// penalty param ||x||_1 (pen = 1).
cudaError_t launch_l1_step(const double* H, const void* Lbuf, const void* Dinv, int f32, int d,
                           const double* g, double param, int pen, int max_iter, double tol,
                           QpWork w, double* x, double* step_norm, int* status, cudaStream_t st);

// ---- SRHT (Sec. 2's comparison sketch) ------------------------------------------
// n2 = least power of two >= n; T buffer n2 x srht_ldt(d) (FP64 if acc64 else FP32);
// rows: m int32.  Writes the raw P H D A into SA (m x d).
int64_t srht_n2(int64_t n);
int64_t srht_ldt(int d);
cudaError_t launch_srht(const DenseA& A, const SketchKeys& K, int64_t m, int acc64, void* Tbuf,
                        int32_t* rows, void* SA, cudaStream_t st);

// ---- Gaussian sketch (Sec. 2's dense comparison) --------------------------------
// SA = G A with G generated tile by tile inside the kernel (never stored):
// FP64 SIMT tiles (plain form) or a tcgen05 TF32 kernel (mixed forms), split
// over the rows of A; partial holds partial_bytes, summed in split order.
struct GaussPlan {
  int acc64 = 0;
  int64_t m = 0, n = 0;
  int d = 0;
  int mtiles = 0, ntiles = 0, splits = 0;
  int64_t kchunk = 0;        // plain form: rows of A per split
  int dn = 0;                // mixed form: columns per N tile (multiple of 64, <= 512)
  int dpad = 0;              // mixed form: d rounded up to 64 (rows of the A^T operand)
  int box_rows = 0;          // mixed form: rows of A^T per TMA copy
  int64_t ldt = 0;           // mixed form: n rounded up to 32 (row length of A^T)
  size_t at_bytes = 0;       // mixed form: the A^T operand (dpad x ldt TF32)
  int64_t ldp = 0;           // mixed form: row length of the partials
  int64_t kb_per_split = 0;  // mixed form: 32-row K blocks per split
  int stages = 0, tmem_cols = 0, smem = 0;
  size_t partial_bytes = 0;
};
GaussPlan make_gauss_plan(int64_t m, int64_t n, int d, int acc64, int sms);
// Mixed form: A^T in TF32, K-major, once per context (a no-op in the plain form).
cudaError_t launch_gauss_operand(const GaussPlan& p, const DenseA& A, void* At, cudaStream_t st);
cudaError_t launch_gauss(const GaussPlan& p, const DenseA& A, const void* At, uint64_t key,
                         void* partial, void* SA, int* status, cudaStream_t st);

// ---- p = 2 ball step (host-driven secular iteration; kernels in l2ball.cu) ------
cudaError_t launch_l2_matvec(const double* H, int d, const double* x, double mu, const double* base,
                             double sgn, double* out, cudaStream_t st);
cudaError_t launch_l2_dots(const double* a, const double* b, int d, double* scal, cudaStream_t st);
cudaError_t launch_l2_axpy(double* y, const double* a, int d, cudaStream_t st);
cudaError_t launch_l2_store(const double* src, int d, double* x, double* step_norm,
                            cudaStream_t st);

// ---- adjoint (ridge / OLS) -----------------------------------------------------
cudaError_t launch_cg_init(const double* rhs, int d, double* v, double* r, double* scal,
                           cudaStream_t st);
cudaError_t launch_cg_dir(const double* r, const double* z, int d, double* p, double* scal,
                          int first, cudaStream_t st);
cudaError_t launch_cg_step(const double* p, const double* negq, int d, double* v, double* r,
                           double* scal, cudaStream_t st);
cudaError_t launch_negate(double* a, int64_t n, cudaStream_t st);
cudaError_t launch_adjoint_dA(const DenseA& A, const double* b, const double* x, const double* v,
                              void* out, cudaStream_t st);

// small device vector kernels
cudaError_t launch_split_b(const double* b, int64_t n, float2* out, cudaStream_t st);
