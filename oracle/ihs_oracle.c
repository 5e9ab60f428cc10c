/*
 * ihs_oracle.c -- plain FP64 CPU oracle for the data passes of the Iterative
 * Hessian Sketch with CountSketch / SJLT (Cormode & Dickens, "Iterative Hessian
 * Sketch in Input Sparsity Time", arXiv 1910.14166).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant table with the CUDA library: the hash below is written from the
 * published SplitMix64 definition, independently of the GPU's copy.
 *
 * Every loop here is the plain definition: no blocking, no reordering, one
 * pass in ascending index order, all arithmetic in IEEE double.
 *
 * Functions (all exported with C linkage, plain pointers, row-major arrays):
 *   orc_sm64_at       SplitMix64 stream output (Steele, Lea & Flood 2014)
 *   orc_hash          CountSketch / SJLT bucket and sign per (block, row)  (Sec. 2)
 *   orc_sketch_dense  SA = S A by streaming the rows of a dense A           (Sec. 2, "applied by streaming")
 *   orc_sketch_csr    the same over a CSR matrix                            (Sec. 2)
 *   orc_gram          H = scale * (SA)^T (SA) + shift * I                   (Sec. 1, approximate Hessian)
 *   orc_resid_grad_dense / orc_resid_grad_csr
 *                     r = b - A x,  g = A^T r                               (Eq. 2, linear term)
 *   orc_sketch_adjoint  (S^T G) row by row                                  (adjoint of Sec. 2's map)
 *   orc_srht_draw     SRHT signs D and sampled rows P                       (Sec. 2, SRHT)
 *   orc_srht_sketch_dense  P H D A by its definition, entry by entry        (Sec. 2, SRHT)
 *   orc_gauss_draw    the entries of the Gaussian sketch's G                (Sec. 2, Gaussian)
 *
 * Build: gcc -O2 -std=c11 -shared -fPIC -o libihs_oracle.so ihs_oracle.c
 * (-O2 keeps IEEE semantics: no -ffast-math, no FMA contraction, see below).
 *
 * Multi-core build (the timed CPU baseline only): the same file with
 * -fopenmp.  Each parallel loop gives every thread a disjoint set of outputs
 * (rows of SA by bucket, rows of r, columns of g, rows of H, entries of the
 * draws) and each output is still summed over the same terms in the same
 * ascending order as the serial loop, so the two builds return bit-identical
 * results (a CPU test checks it).  Without -fopenmp the pragmas are ignored
 * and every "owned range" below is the whole range.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The part [lo, hi) of [0, count) owned by the calling thread of the current
 * OpenMP team (all of it outside a team or in the serial build). */
static void owned_range(int64_t count, int64_t* lo, int64_t* hi) {
#ifdef _OPENMP
  const int64_t nt = omp_get_num_threads(), t = omp_get_thread_num();
  *lo = count * t / nt;
  *hi = count * (t + 1) / nt;
#else
  *lo = 0;
  *hi = count;
#endif
}

/* Threads of the multi-core build (ignored by the serial build); returns the
 * number the next parallel region will use. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Keep a*b+c as two roundings so the oracle is plain IEEE double arithmetic. */
#if defined(__GNUC__)
#pragma GCC optimize("fp-contract=off")
#endif

/* SplitMix64 constants, from the published generator (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the state
 * advances by the golden-gamma increment and each output is the state passed
 * through the two xor-shift-multiply rounds of the finaliser. */
#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t sm64_finalise(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Output number j (counting from 0) of a SplitMix64 generator whose initial
 * state is `state`: the generator adds gamma before each output, so output j
 * is the finaliser of state + (j + 1) * gamma (mod 2^64). */
uint64_t orc_sm64_at(uint64_t state, uint64_t j) {
  return sm64_finalise(state + (j + 1) * SM64_GAMMA);
}

/*
 * Sketch draw (Sec. 2, CountSketch and SJLT definitions).  The paper asks
 * for a uniformly random row h(i) per column i of S and a sign that is +1 or
 * -1 with probability 1/2, and builds an SJLT from s independent CountSketches
 * of m/s rows each.  It names no generator; this library's reading is a
 * counter-based SplitMix64 chain, one 64-bit output per row and PAIR of
 * blocks (2p, 2p + 1):
 *     key_seed = out(seed, 0);  key_t = out(key_seed, t);  key_tp = out(key_t, p);
 *     w = out(key_tp, i)
 * where out(x, j) = orc_sm64_at(x, j).  Block 2p takes the high 32 bits of w
 * and block 2p + 1 the low 32 bits: the bucket within the block is the
 * multiply-shift range reduction floor(h32 * mb / 2^32) of that half, with
 * mb = m / s (Lemire 2019), and the sign is -1 when bit 0 of the OTHER half
 * is set (bit 0 of w for block 2p, bit 32 for block 2p + 1).  A bucket is
 * set by its half's high bits, so a sign (the other half's lowest bit) is
 * independent of it up to mb / 2^32.  The global row of S is k * mb + bucket.
 * With s = 1 (CountSketch) only block 0 exists and the draw is the high half
 * and bit 0 of w.
 *
 * Output layout: bucket[k * n + i] (int32, global row in [0, m)),
 *                sign[k * n + i]   (int8, +1 or -1).
 * Returns 0, or -1 if s < 1, m % s != 0, or m/s exceeds 2^31 - 1.
 */
int orc_hash(uint64_t seed, int64_t t, int s, int64_t m, int64_t n,
             int32_t* bucket, int8_t* sign) {
  if (s < 1 || m < 1 || m % s != 0) return -1;
  int64_t mb = m / s;
  if (mb > 2147483647LL) return -1;
  uint64_t key_seed = orc_sm64_at(seed, 0);
  uint64_t key_t = orc_sm64_at(key_seed, (uint64_t)t);
  for (int p = 0; 2 * p < s; ++p) {
    uint64_t key_tp = orc_sm64_at(key_t, (uint64_t)p);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      uint64_t w = orc_sm64_at(key_tp, (uint64_t)i);
      uint64_t hi = w >> 32, lo = w & 0xFFFFFFFFULL;
      int k = 2 * p;
      bucket[(int64_t)k * n + i] = (int32_t)((int64_t)k * mb + (int64_t)((hi * (uint64_t)mb) >> 32));
      sign[(int64_t)k * n + i] = (lo & 1ULL) ? (int8_t)-1 : (int8_t)1;
      if (k + 1 < s) {
        bucket[(int64_t)(k + 1) * n + i] =
            (int32_t)((int64_t)(k + 1) * mb + (int64_t)((lo * (uint64_t)mb) >> 32));
        sign[(int64_t)(k + 1) * n + i] = (hi & 1ULL) ? (int8_t)-1 : (int8_t)1;
      }
    }
  }
  return 0;
}

/*
 * SA = S A for a dense row-major A (n x d, leading dimension lda), following
 * the streaming description of Sec. 2: each row i of A is visited once per
 * block k, in ascending i, and added with its sign into row bucket[k][i] of SA.
 * The entries of S are the raw signs (+-1); the SJLT normalisation by the
 * number of nonzeros per column (App. A, "normalise by the number of
 * nonzeros") is applied later, once, as the Gram scale 1/s.
 * SA is m x d row-major and is overwritten.
 */
void orc_sketch_dense(int64_t n, int64_t d, const double* A, int64_t lda,
                      int64_t m, int s, const int32_t* bucket,
                      const int8_t* sign, double* SA) {
#pragma omp parallel
  {
    int64_t r0, r1; /* the rows of SA (buckets) this thread owns */
    owned_range(m, &r0, &r1);
    for (int64_t q = r0 * d; q < r1 * d; ++q) SA[q] = 0.0;
    for (int k = 0; k < s; ++k) {
      for (int64_t i = 0; i < n; ++i) {
        int64_t row = bucket[(int64_t)k * n + i];
        if (row < r0 || row >= r1) continue;
        double sg = (double)sign[(int64_t)k * n + i];
        for (int64_t j = 0; j < d; ++j) SA[row * d + j] += sg * A[i * lda + j];
      }
    }
  }
}

/*
 * The same product for a CSR matrix (rowptr[n+1], col[nnz], val[nnz]): on
 * seeing nonzero A_ij, bucket h(i) of column j gains sign(i) * A_ij (Sec. 2).
 * rowptr is int64.  SA is m x d row-major and is overwritten.
 */
void orc_sketch_csr(int64_t n, int64_t d, const int64_t* rowptr,
                    const int32_t* col, const double* val, int64_t m, int s,
                    const int32_t* bucket, const int8_t* sign, double* SA) {
#pragma omp parallel
  {
    int64_t r0, r1; /* the rows of SA (buckets) this thread owns */
    owned_range(m, &r0, &r1);
    for (int64_t q = r0 * d; q < r1 * d; ++q) SA[q] = 0.0;
    for (int k = 0; k < s; ++k) {
      for (int64_t i = 0; i < n; ++i) {
        int64_t row = bucket[(int64_t)k * n + i];
        if (row < r0 || row >= r1) continue;
        double sg = (double)sign[(int64_t)k * n + i];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
          SA[row * d + col[p]] += sg * val[p];
      }
    }
  }
}

/*
 * Approximate Hessian H = scale * (SA)^T (SA) + shift * I (Sec. 1: IHS
 * replaces A^T A by the quadratic form of SA).  scale is 1/s for an SJLT with
 * raw +-1 entries; shift is the ridge parameter (0 for OLS and LASSO).
 * Full d x d output, row-major, plain triple loop over r = 0..m-1.
 */
void orc_gram(int64_t m, int64_t d, const double* SA, double scale,
              double shift, double* H) {
#pragma omp parallel for schedule(static)
  for (int64_t a = 0; a < d; ++a) {
    for (int64_t c = 0; c < d; ++c) {
      double acc = 0.0;
      for (int64_t r = 0; r < m; ++r) acc += SA[r * d + a] * SA[r * d + c];
      H[a * d + c] = scale * acc + (a == c ? shift : 0.0);
    }
  }
}

/*
 * Residual and gradient of f(x) = 1/2 ||Ax - b||^2 (Eq. 1): r = b - A x and
 * g = A^T r = -grad f(x), the linear term of the IHS subproblem (Eq. 2).
 * Rows in ascending order; r may be NULL.  The residual of every row is
 * formed first, then g_j = sum_i A_ij r_i over the rows in ascending order
 * (the same additions, in the same order, as one interleaved pass).
 * Returns 0, or -1 if the residual buffer could not be allocated.
 */
int orc_resid_grad_dense(int64_t n, int64_t d, const double* A, int64_t lda,
                         const double* b, const double* x, double* r,
                         double* g) {
  double* rr = r ? r : (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!rr) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ax = 0.0;
    for (int64_t j = 0; j < d; ++j) ax += A[i * lda + j] * x[j];
    rr[i] = b[i] - ax;
  }
#pragma omp parallel
  {
    int64_t j0, j1; /* the entries of g this thread owns */
    owned_range(d, &j0, &j1);
    for (int64_t j = j0; j < j1; ++j) g[j] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double ri = rr[i];
      for (int64_t j = j0; j < j1; ++j) g[j] += A[i * lda + j] * ri;
    }
  }
  if (!r) free(rr);
  return 0;
}

int orc_resid_grad_csr(int64_t n, int64_t d, const int64_t* rowptr,
                       const int32_t* col, const double* val, const double* b,
                       const double* x, double* r, double* g) {
  double* rr = r ? r : (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!rr) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double ax = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) ax += val[p] * x[col[p]];
    rr[i] = b[i] - ax;
  }
#pragma omp parallel
  {
    int64_t j0, j1; /* the entries of g this thread owns */
    owned_range(d, &j0, &j1);
    for (int64_t j = j0; j < j1; ++j) g[j] = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (col[p] >= j0 && col[p] < j1) g[col[p]] += val[p] * rr[i];
  }
  if (!r) free(rr);
  return 0;
}

/*
 * Adjoint of the sketch map: given G (m x d), (S^T G)_i = sum_k sign_k(i) *
 * G[bucket_k(i), :] * entry_scale, with entry_scale = 1/sqrt(s) for the
 * normalised SJLT.  Output n x d row-major.
 */
void orc_sketch_adjoint(int64_t n, int64_t d, int64_t m, int s,
                        const int32_t* bucket, const int8_t* sign,
                        const double* G, double entry_scale, double* out) {
  (void)m;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < d; ++j) out[i * d + j] = 0.0;
    for (int k = 0; k < s; ++k) {
      int64_t row = bucket[(int64_t)k * n + i];
      double sg = (double)sign[(int64_t)k * n + i] * entry_scale;
      for (int64_t j = 0; j < d; ++j) out[i * d + j] += sg * G[row * d + j];
    }
  }
}

/*
 * SRHT draw (Sec. 2: S = P H D, with D diagonal +-1 signs, H the recursively
 * defined (Sylvester) Hadamard transform and P a uniform row sampler).  The
 * paper fixes no generator, no padding and no sampling scheme; this
 * library's reading:
 *   - A is padded with zero rows to n2 = the least power of two >= n;
 *   - D_i is the sign of block 0's word of row i, the same word a
 *     CountSketch with the same (seed, t) uses: sign[i] = -1 iff bit 0 of
 *     out(key_t0, i) is set;
 *   - P takes m rows with replacement: sample r uses w = out(key_t1, r) and
 *     row = floor(hi32(w) * n2 / 2^32), with key_tk as in orc_hash.
 * Output: rows[r] in [0, n2), sign[i] for i < n.  Returns 0, or -1 if n2 is
 * not a power of two >= n or exceeds 2^31.
 */
int orc_srht_draw(uint64_t seed, int64_t t, int64_t m, int64_t n, int64_t n2, int32_t* rows,
                  int8_t* sign) {
  if (n2 < n || n2 < 1 || n2 > 2147483648LL || (n2 & (n2 - 1)) != 0 || m < 1) return -1;
  uint64_t key_seed = orc_sm64_at(seed, 0);
  uint64_t key_t = orc_sm64_at(key_seed, (uint64_t)t);
  uint64_t key_t0 = orc_sm64_at(key_t, 0);
  uint64_t key_t1 = orc_sm64_at(key_t, 1);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t w = orc_sm64_at(key_t0, (uint64_t)i);
    sign[i] = (w & 1ULL) ? (int8_t)-1 : (int8_t)1;
  }
  for (int64_t r = 0; r < m; ++r) {
    uint64_t w = orc_sm64_at(key_t1, (uint64_t)r);
    rows[r] = (int32_t)(((w >> 32) * (uint64_t)n2) >> 32);
  }
  return 0;
}

/* Popcount parity: H[r][i] = (-1)^{popcount(r & i)} for the Sylvester
 * Hadamard matrix H_{2n} = [H_n H_n; H_n -H_n]. */
static int hadamard_sign(uint64_t r, uint64_t i) {
  uint64_t v = r & i;
  int p = 0;
  while (v) {
    p ^= 1;
    v &= v - 1;
  }
  return p ? -1 : 1;
}

/*
 * SA_raw = P H D A for a dense row-major A (n x d, leading dimension lda):
 * row k of SA_raw is sum_{i < n} H[rows[k]][i] sign[i] A_i, in ascending i,
 * in FP64.  The entries of H are the raw +-1; the normalisation (S = m^{-1/2}
 * P H D, so that E[S^T S] = I) is applied as the Gram scale 1/m.  O(m n d):
 * the definition, for small cases.
 */
void orc_srht_sketch_dense(int64_t n, int64_t d, const double* A, int64_t lda, int64_t m,
                           const int32_t* rows, const int8_t* sign, double* SA) {
  for (int64_t k = 0; k < m; ++k) {
    double* out = SA + k * d;
    for (int64_t j = 0; j < d; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double c = (double)(hadamard_sign((uint64_t)rows[k], (uint64_t)i) * sign[i]);
      const double* a = A + i * lda;
      for (int64_t j = 0; j < d; ++j) out[j] += c * a[j];
    }
  }
}

/*
 * Gaussian sketch (Sec. 2: S = G / sqrt(m), G_ij iid N(0, 1)).  The paper
 * names no generator; this library's reading: entry (r, i) of the m x n
 * matrix G uses the word w = out(key_t2, r * n + i) (key_tk as in orc_hash,
 * k = 2) and the Box-Muller transform (Box & Muller 1958) of the two 32-bit
 * halves, u1 = (hi32(w) + 1/2) / 2^32 and u2 = (lo32(w) + 1/2) / 2^32 (both
 * in (0, 1)): g = sqrt(-2 ln u1) cos(2 pi u2), in double.  G is row-major.
 */
#include <math.h>
void orc_gauss_draw(uint64_t seed, int64_t t, int64_t m, int64_t n, double* G) {
  uint64_t key_seed = orc_sm64_at(seed, 0);
  uint64_t key_t = orc_sm64_at(key_seed, (uint64_t)t);
  uint64_t key_t2 = orc_sm64_at(key_t, 2);
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < m; ++r)
    for (int64_t i = 0; i < n; ++i) {
      uint64_t w = orc_sm64_at(key_t2, (uint64_t)(r * n + i));
      double u1 = ((double)(w >> 32) + 0.5) / 4294967296.0;
      double u2 = ((double)(w & 0xFFFFFFFFULL) + 0.5) / 4294967296.0;
      G[r * n + i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    }
}
