/*
 * FT-DGEMM oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the fault-tolerant
 * DGEMM of FT-GEMM (Wu, Zhai, Huang, Jian, Chen, HPDC'23) computes:
 *
 *   C_out = alpha * op(A) * op(B) + beta * C_in          (abstract, §1, §2.1)
 *
 * protected by algorithm-based fault tolerance in the sense of Huang and
 * Abraham (1984), which the paper builds on (§1, §2.2): column and row
 * checksums of C_out are predicted from checksums of the operands and of
 * beta*C_in, compared against reference checksums summed from the computed
 * C_out, and an element found wrong is corrected.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU legs (the
 * cpu_baseline sample, the reference arm, and the sampled-row accuracy checks
 * of its optional --split / --config5 reports, outside any timed region) may
 * load this library.  The GPU library shares no code with it.
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off -fopenmp -shared -fPIC.
 * With contraction off, every product and every sum below is one IEEE
 * double operation rounded to nearest, so the rounding of each result is the
 * textbook one.
 *
 * Storage is column-major (BLAS).  op(X) is X ('N') or X^T ('T'/'C').
 * Argument errors return -i for the i-th argument (BLAS xerbla numbering).
 *
 * Readings of the paper that the paper leaves open (the poster gives no
 * threshold, no verification granularity and no correction rule):
 *  - verification is done once per BM x BN output tile, after the whole
 *    K loop;
 *  - a row or column is flagged when |reference - predicted| exceeds an
 *    a-priori rounding bound tau (orc_tau) or is not finite;
 *  - every flagged row x flagged column intersection (at most 64 per tile)
 *    is recomputed by a length-K dot product from the original inputs;
 *    rows/columns still failing afterwards have their whole tile segment
 *    recomputed; a mismatch that persists after that is a checksum fault;
 *  - a predicted checksum that is not finite marks its row/column
 *    unverifiable (non-finite inputs), never flagged;
 *  - an injected fault flips bit b (0..62) of one accumulator value after the
 *    s-th k-step of BK products (source-level injection, §3.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_U 0x1p-53 /* unit roundoff of IEEE binary64, round to nearest */

typedef struct {
  int64_t detected;      /* elements whose recomputed value differed */
  int64_t corrected;     /* of those, rewritten with the recomputed value */
  int64_t checksum_only; /* rows+cols still mismatching after recomputation */
  int64_t unverifiable;  /* rows+cols with a non-finite predicted checksum */
  int64_t flagged_rows;  /* row mismatches raised by the first verification */
  int64_t flagged_cols;  /* column mismatches raised by the first verification */
  int64_t recomputed;    /* elements recomputed (wrong or not) */
} orc_counts;

typedef struct {
  int64_t row, col;
  int32_t tile, kind; /* kind 0: row x column intersection, 1: segment fallback */
  double delta;       /* value before correction minus recomputed value */
} orc_loc;

static int is_n(char t) { return t == 'N' || t == 'n'; }
static int is_t(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }

/* op(A)(i,k) and op(B)(k,j) for column-major storage. */
static inline double opa(const double *A, int64_t lda, int ta_n, int64_t i, int64_t k) {
  return ta_n ? A[i + k * lda] : A[k + i * lda];
}
static inline double opb(const double *B, int64_t ldb, int tb_n, int64_t k, int64_t j) {
  return tb_n ? B[k + j * ldb] : B[j + k * ldb];
}

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

/* BLAS argument checks; returns 0 or -i. */
static int check_args(char ta, char tb, int64_t M, int64_t N, int64_t K,
                      int64_t lda, int64_t ldb, int64_t ldc) {
  if (!is_n(ta) && !is_t(ta)) return -1;
  if (!is_n(tb) && !is_t(tb)) return -2;
  if (M < 0) return -3;
  if (N < 0) return -4;
  if (K < 0) return -5;
  int64_t arows = is_n(ta) ? M : K, brows = is_n(tb) ? K : N;
  if (lda < max64(1, arows)) return -8;
  if (ldb < max64(1, brows)) return -10;
  if (ldc < max64(1, M)) return -13;
  return 0;
}

/* C <- beta*C with BLAS semantics: beta == 0 writes zeros without reading C. */
static void scale_c(int64_t M, int64_t N, double beta, double *C, int64_t ldc) {
  if (beta == 1.0) return;
  for (int64_t j = 0; j < N; ++j)
    for (int64_t i = 0; i < M; ++i)
      C[i + j * ldc] = (beta == 0.0) ? 0.0 : beta * C[i + j * ldc];
}

/*
 * Plain DGEMM (the operation of §2.1): for every (i,j),
 *   acc = sum_{k=0}^{K-1} op(A)(i,k)*op(B)(k,j)   (ascending k, mult then add)
 *   C(i,j) = alpha*acc + beta*C(i,j)              (beta == 0: C not read)
 * and, when E != NULL, the componentwise error-bound matrix
 *   E(i,j) = |alpha| * sum_k |op(A)(i,k)||op(B)(k,j)| + |beta|*|C_in(i,j)|.
 * Quick returns: M == 0 or N == 0 does nothing; K == 0 or alpha == 0 gives
 * C = beta*C.  nthreads <= 0 uses the OpenMP default.
 */
int orc_gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
             const double *A, int64_t lda, const double *B, int64_t ldb,
             double beta, double *C, int64_t ldc, double *E, int64_t lde,
             int nthreads) {
  int rc = check_args(ta, tb, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  if (E && lde < max64(1, M)) return -15;
  if (M == 0 || N == 0) return 0;
  if (K == 0 || alpha == 0.0) {
    if (E)
      for (int64_t j = 0; j < N; ++j)
        for (int64_t i = 0; i < M; ++i)
          E[i + j * lde] = (beta == 0.0) ? 0.0 : fabs(beta) * fabs(C[i + j * ldc]);
    scale_c(M, N, beta, C, ldc);
    return 0;
  }
  int ta_n = is_n(ta), tb_n = is_n(tb);
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
  {
    double *acc = (double *)malloc(sizeof(double) * (size_t)M);
    double *eac = (double *)malloc(sizeof(double) * (size_t)M);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t j = 0; j < N; ++j) {
      for (int64_t i = 0; i < M; ++i) { acc[i] = 0.0; eac[i] = 0.0; }
      for (int64_t k = 0; k < K; ++k) {
        double b = opb(B, ldb, tb_n, k, j);
        double ab = fabs(b);
        for (int64_t i = 0; i < M; ++i) {
          double a = opa(A, lda, ta_n, i, k);
          acc[i] = acc[i] + a * b;
          eac[i] = eac[i] + fabs(a) * ab;
        }
      }
      for (int64_t i = 0; i < M; ++i) {
        double cin = (beta == 0.0) ? 0.0 : C[i + j * ldc];
        if (E) E[i + j * lde] = fabs(alpha) * eac[i] + ((beta == 0.0) ? 0.0 : fabs(beta) * fabs(cin));
        C[i + j * ldc] = (beta == 0.0) ? alpha * acc[i] : alpha * acc[i] + beta * cin;
      }
    }
    free(acc);
    free(eac);
  }
  return 0;
}

/* Partial dot product sum_{k=0}^{kend-1} op(A)(i,k)*op(B)(k,j), ascending k:
 * the value an accumulator holds after its first kend products. */
double orc_partial(char ta, char tb, int64_t i, int64_t j, int64_t kend,
                   const double *A, int64_t lda, const double *B, int64_t ldb) {
  int ta_n = is_n(ta), tb_n = is_n(tb);
  double acc = 0.0;
  for (int64_t k = 0; k < kend; ++k) acc = acc + opa(A, lda, ta_n, i, k) * opb(B, ldb, tb_n, k, j);
  return acc;
}

/*
 * Whole-matrix checksum invariants (Huang-Abraham encoding, §2.2):
 *   colpred = alpha * (e^T op(A)) op(B) + beta * e^T C_in     (length N)
 *   rowpred = alpha * op(A) (op(B) e)   + beta * C_in e       (length M)
 * Each is a plain O(MK + KN + MN) computation; beta == 0 drops the C terms.
 */
int orc_pred_checksums(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb,
                       double beta, const double *C, int64_t ldc,
                       double *colpred, double *rowpred) {
  int rc = check_args(ta, tb, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  int ta_n = is_n(ta), tb_n = is_n(tb);
  double *ea = (double *)calloc((size_t)(K > 0 ? K : 1), sizeof(double)); /* e^T op(A) */
  double *be = (double *)calloc((size_t)(K > 0 ? K : 1), sizeof(double)); /* op(B) e */
  for (int64_t k = 0; k < K; ++k) {
    double s = 0.0;
    for (int64_t i = 0; i < M; ++i) s = s + opa(A, lda, ta_n, i, k);
    ea[k] = s;
    s = 0.0;
    for (int64_t j = 0; j < N; ++j) s = s + opb(B, ldb, tb_n, k, j);
    be[k] = s;
  }
  for (int64_t j = 0; j < N; ++j) {
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < K; ++k) s = s + ea[k] * opb(B, ldb, tb_n, k, j);
    if (beta != 0.0)
      for (int64_t i = 0; i < M; ++i) c = c + C[i + j * ldc];
    colpred[j] = (beta == 0.0) ? alpha * s : alpha * s + beta * c;
  }
  for (int64_t i = 0; i < M; ++i) {
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < K; ++k) s = s + opa(A, lda, ta_n, i, k) * be[k];
    if (beta != 0.0)
      for (int64_t j = 0; j < N; ++j) c = c + C[i + j * ldc];
    rowpred[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * c;
  }
  free(ea);
  free(be);
  return 0;
}

/*
 * Per-tile operand checksum vectors and the abs sums the threshold uses, by
 * their definitions (the A and B checksums of §2.2/§2.3, per BM-row and
 * BN-column tile):
 *   acs[I*K + k]  = sum_{i in I} op(A)(i,k)          aabsmax[I] = max_k sum_{i in I} |op(A)(i,k)|
 *   arowabs[i]    = sum_k |op(A)(i,k)|
 *   bcs[J*K + k]  = sum_{j in J} op(B)(k,j)          babsmax[J] = max_k sum_{j in J} |op(B)(k,j)|
 *   bcolabs[j]    = sum_k |op(B)(k,j)|
 */
int orc_encode_operands(char ta, char tb, int64_t M, int64_t N, int64_t K,
                        const double *A, int64_t lda, const double *B, int64_t ldb,
                        int64_t BM, int64_t BN,
                        double *acs, double *aabsmax, double *arowabs,
                        double *bcs, double *babsmax, double *bcolabs) {
  int rc = check_args(ta, tb, M, N, K, lda, ldb, max64(1, M));
  if (rc) return rc;
  if (BM <= 0 || BN <= 0) return -11;
  int ta_n = is_n(ta), tb_n = is_n(tb);
  int64_t nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN;
  for (int64_t I = 0; I < nI; ++I) {
    int64_t i0 = I * BM, i1 = i0 + BM < M ? i0 + BM : M;
    double mx = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double s = 0.0, sa = 0.0;
      for (int64_t i = i0; i < i1; ++i) {
        double a = opa(A, lda, ta_n, i, k);
        s = s + a;
        sa = sa + fabs(a);
      }
      acs[I * K + k] = s;
      if (sa > mx) mx = sa;
    }
    aabsmax[I] = mx;
  }
  for (int64_t i = 0; i < M; ++i) {
    double sa = 0.0;
    for (int64_t k = 0; k < K; ++k) sa = sa + fabs(opa(A, lda, ta_n, i, k));
    arowabs[i] = sa;
  }
  for (int64_t J = 0; J < nJ; ++J) {
    int64_t j0 = J * BN, j1 = j0 + BN < N ? j0 + BN : N;
    double mx = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double s = 0.0, sa = 0.0;
      for (int64_t j = j0; j < j1; ++j) {
        double b = opb(B, ldb, tb_n, k, j);
        s = s + b;
        sa = sa + fabs(b);
      }
      bcs[J * K + k] = s;
      if (sa > mx) mx = sa;
    }
    babsmax[J] = mx;
  }
  for (int64_t j = 0; j < N; ++j) {
    double sa = 0.0;
    for (int64_t k = 0; k < K; ++k) sa = sa + fabs(opb(B, ldb, tb_n, k, j));
    bcolabs[j] = sa;
  }
  return 0;
}

/*
 * Detection threshold for one row (or column) checksum of a tile.
 *
 * With n = K + L + 3 (L = number of terms the checksum sums: columns of the
 * tile for a row checksum, rows for a column checksum), the reference sum of
 * the computed outputs and the predicted checksum each differ from the exact
 * checksum by at most gamma_n * S, where (for a row i)
 *   S = |alpha| * sum_k |op(A)(i,k)| * max_k sum_{j in J} |op(B)(k,j)|
 *       + |beta| * sum_{j in J} |C_in(i,j)|
 * bounds sum_{j in J} (|alpha| sum_k |a_ik||b_kj| + |beta||c_ij|) by Hoelder's
 * inequality.  tau = 2.01 * n * u * S + n * 2^-1021 covers both sides,
 * gamma_n = n u / (1 - n u) <= 1.005 n u, the rounding of S itself, and an
 * absolute term for gradual underflow.
 */
double orc_tau(int64_t K, int64_t L, double alpha, double absrow, double absmax,
               double beta, double abscsum) {
  double n = (double)(K + L + 3);
  double S = fabs(alpha) * absrow * absmax + ((beta == 0.0) ? 0.0 : fabs(beta) * abscsum);
  return 2.01 * n * ORC_U * S + n * 0x1p-1021;
}

/* Threshold for comparing a stored element with its recomputation: both are
 * within gamma_{K+3} * E(i,j) of the exact value. */
static double elem_tau(int64_t K, double E) {
  double n = (double)(K + 3);
  return 2.01 * n * ORC_U * E + n * 0x1p-1021;
}

static double flip_bit(double x, int bit) {
  uint64_t u;
  memcpy(&u, &x, 8);
  u ^= (uint64_t)1 << bit;
  memcpy(&x, &u, 8);
  return x;
}

/* splitmix64 (Steele, Lea, Flood 2014; Vigna's reference form): the n-th
 * output (n = 0, 1, ...) of the generator seeded with `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Seeded random fault list: flip f uses splitmix64 outputs 4f..4f+3 for
 * (row mod M, col mod N, kstep mod nksteps, bit mod 63).  out is count x 4. */
void orc_random_flips(uint64_t seed, int64_t count, int64_t M, int64_t N, int64_t nksteps,
                      int64_t *out) {
  for (int64_t f = 0; f < count; ++f) {
    out[4 * f + 0] = (int64_t)(orc_splitmix64(seed, 4 * (uint64_t)f + 0) % (uint64_t)M);
    out[4 * f + 1] = (int64_t)(orc_splitmix64(seed, 4 * (uint64_t)f + 1) % (uint64_t)N);
    out[4 * f + 2] = (int64_t)(orc_splitmix64(seed, 4 * (uint64_t)f + 2) % (uint64_t)nksteps);
    out[4 * f + 3] = (int64_t)(orc_splitmix64(seed, 4 * (uint64_t)f + 3) % 63u);
  }
}

typedef struct {
  char ta, tb;
  int64_t M, N, K;
  double alpha, beta;
  const double *A, *B;
  int64_t lda, ldb;
} prob_t;

/* Recompute one output element from the original inputs and replace it when
 * it differs from the stored value by more than the element bound. */
static void recompute_elem(const prob_t *p, double *out, int64_t mI, int64_t li, int64_t lj,
                           int64_t i, int64_t j, const double *cin, int32_t tile, int32_t kind,
                           orc_counts *cnt, orc_loc *locs, int64_t cap, int64_t *nloc) {
  int ta_n = is_n(p->ta), tb_n = is_n(p->tb);
  double dot = 0.0, ab = 0.0;
  for (int64_t k = 0; k < p->K; ++k) {
    double a = opa(p->A, p->lda, ta_n, i, k), b = opb(p->B, p->ldb, tb_n, k, j);
    dot = dot + a * b;
    ab = ab + fabs(a) * fabs(b);
  }
  double c = cin[li + lj * mI];
  double nv = (p->beta == 0.0) ? p->alpha * dot : p->alpha * dot + p->beta * c;
  double E = fabs(p->alpha) * ab + ((p->beta == 0.0) ? 0.0 : fabs(p->beta) * fabs(c));
  double old = out[li + lj * mI];
  cnt->recomputed++;
  int wrong = (!isfinite(old) && isfinite(nv)) || fabs(old - nv) > elem_tau(p->K, E);
  if (wrong) {
    cnt->detected++;
    cnt->corrected++;
    if (*nloc < cap) {
      orc_loc *L = &locs[*nloc];
      L->row = i; L->col = j; L->tile = tile; L->kind = kind; L->delta = old - nv;
    }
    (*nloc)++;
  }
  out[li + lj * mI] = nv;
}

/*
 * Fault-tolerant DGEMM on the CPU, in the paper's order (§2.2): accumulate
 * each output in k-steps of BK products (applying the injected flips after
 * their k-step), combine with beta*C, then per BM x BN tile encode the
 * predicted checksums, sum the reference checksums from the outputs, verify,
 * locate and correct (the readings in the header).
 *
 * flips: nflips x 4 int64 (row, col, kstep, bit); flip_before/after (may be
 * NULL) receive the accumulator value before and after each flip.
 * locs receives up to cap records; *nloc counts all of them.
 * Tiles are processed in parallel; records are appended in any order.
 */
int orc_ft_gemm(char ta, char tb, int64_t M, int64_t N, int64_t K, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb,
                double beta, double *C, int64_t ldc, int64_t BM, int64_t BN, int64_t BK,
                const int64_t *flips, int64_t nflips, double *flip_before, double *flip_after,
                orc_counts *cnt, orc_loc *locs, int64_t cap, int64_t *nloc, int nthreads) {
  int rc = check_args(ta, tb, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  if (BM <= 0 || BN <= 0 || BK <= 0) return -14;
  memset(cnt, 0, sizeof(*cnt));
  *nloc = 0;
  if (M == 0 || N == 0) return 0;
  if (K == 0 || alpha == 0.0) { scale_c(M, N, beta, C, ldc); return 0; }
  int ta_n = is_n(ta), tb_n = is_n(tb);
  prob_t p = {ta, tb, M, N, K, alpha, beta, A, B, lda, ldb};
  int64_t nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN, ntiles = nI * nJ;
  int64_t nks = (K + BK - 1) / BK;
  const int64_t CAP_X = 64; /* max intersections recomputed per tile */
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
#endif
  {
    double *cin = (double *)malloc(sizeof(double) * (size_t)(BM * BN));
    double *out = (double *)malloc(sizeof(double) * (size_t)(BM * BN));
    double *acc = (double *)malloc(sizeof(double) * (size_t)BM);
    double *acsI = (double *)malloc(sizeof(double) * (size_t)K);
    double *bcsJ = (double *)malloc(sizeof(double) * (size_t)K);
    double *pr = (double *)malloc(sizeof(double) * (size_t)BM);
    double *pc = (double *)malloc(sizeof(double) * (size_t)BN);
    double *taur = (double *)malloc(sizeof(double) * (size_t)BM);
    double *tauc = (double *)malloc(sizeof(double) * (size_t)BN);
    int *frow = (int *)malloc(sizeof(int) * (size_t)BM);
    int *fcol = (int *)malloc(sizeof(int) * (size_t)BN);
    char *seg = (char *)malloc((size_t)(BM * BN));
    orc_counts lc;
    orc_loc *lloc = (orc_loc *)malloc(sizeof(orc_loc) * (size_t)(cap > 0 ? cap : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < ntiles; ++t) {
      int64_t I = t % nI, J = t / nI;
      int64_t i0 = I * BM, j0 = J * BN;
      int64_t mI = (i0 + BM < M ? BM : M - i0), nJt = (j0 + BN < N ? BN : N - j0);
      memset(&lc, 0, sizeof(lc));
      int64_t lnloc = 0;
      for (int64_t lj = 0; lj < nJt; ++lj)
        for (int64_t li = 0; li < mI; ++li)
          cin[li + lj * mI] = (beta == 0.0) ? 0.0 : C[(i0 + li) + (j0 + lj) * ldc];

      /* 1. accumulate in k-steps, inject, combine with beta*C */
      for (int64_t lj = 0; lj < nJt; ++lj) {
        int64_t j = j0 + lj;
        for (int64_t li = 0; li < mI; ++li) acc[li] = 0.0;
        for (int64_t s = 0; s < nks; ++s) {
          int64_t k1 = (s + 1) * BK < K ? (s + 1) * BK : K;
          for (int64_t k = s * BK; k < k1; ++k) {
            double b = opb(B, ldb, tb_n, k, j);
            for (int64_t li = 0; li < mI; ++li) acc[li] = acc[li] + opa(A, lda, ta_n, i0 + li, k) * b;
          }
          for (int64_t f = 0; f < nflips; ++f) {
            const int64_t *fl = &flips[4 * f];
            if (fl[1] == j && fl[2] == s && fl[0] >= i0 && fl[0] < i0 + mI) {
              int64_t li = fl[0] - i0;
              if (flip_before) flip_before[f] = acc[li];
              acc[li] = flip_bit(acc[li], (int)fl[3]);
              if (flip_after) flip_after[f] = acc[li];
            }
          }
        }
        for (int64_t li = 0; li < mI; ++li)
          out[li + lj * mI] = (beta == 0.0) ? alpha * acc[li] : alpha * acc[li] + beta * cin[li + lj * mI];
      }

      /* 2. encode: operand checksums of this tile and the predicted checksums */
      for (int64_t k = 0; k < K; ++k) {
        double s = 0.0;
        for (int64_t li = 0; li < mI; ++li) s = s + opa(A, lda, ta_n, i0 + li, k);
        acsI[k] = s;
        s = 0.0;
        for (int64_t lj = 0; lj < nJt; ++lj) s = s + opb(B, ldb, tb_n, k, j0 + lj);
        bcsJ[k] = s;
      }
      double aabsmax = 0.0, babsmax = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double sa = 0.0, sb = 0.0;
        for (int64_t li = 0; li < mI; ++li) sa = sa + fabs(opa(A, lda, ta_n, i0 + li, k));
        for (int64_t lj = 0; lj < nJt; ++lj) sb = sb + fabs(opb(B, ldb, tb_n, k, j0 + lj));
        if (sa > aabsmax) aabsmax = sa;
        if (sb > babsmax) babsmax = sb;
      }
      for (int64_t lj = 0; lj < nJt; ++lj) {
        int64_t j = j0 + lj;
        double s = 0.0, c = 0.0, ca = 0.0, bab = 0.0;
        for (int64_t k = 0; k < K; ++k) {
          double b = opb(B, ldb, tb_n, k, j);
          s = s + acsI[k] * b;
          bab = bab + fabs(b);
        }
        for (int64_t li = 0; li < mI; ++li) { c = c + cin[li + lj * mI]; ca = ca + fabs(cin[li + lj * mI]); }
        pc[lj] = (beta == 0.0) ? alpha * s : alpha * s + beta * c;
        tauc[lj] = orc_tau(K, mI, alpha, bab, aabsmax, beta, ca);
      }
      for (int64_t li = 0; li < mI; ++li) {
        int64_t i = i0 + li;
        double s = 0.0, c = 0.0, ca = 0.0, aab = 0.0;
        for (int64_t k = 0; k < K; ++k) {
          double a = opa(A, lda, ta_n, i, k);
          s = s + a * bcsJ[k];
          aab = aab + fabs(a);
        }
        for (int64_t lj = 0; lj < nJt; ++lj) { c = c + cin[li + lj * mI]; ca = ca + fabs(cin[li + lj * mI]); }
        pr[li] = (beta == 0.0) ? alpha * s : alpha * s + beta * c;
        taur[li] = orc_tau(K, nJt, alpha, aab, babsmax, beta, ca);
      }

      /* 3. reference checksums and verification */
      int64_t nr = 0, nc = 0;
      for (int64_t li = 0; li < mI; ++li) {
        double rr = 0.0;
        for (int64_t lj = 0; lj < nJt; ++lj) rr = rr + out[li + lj * mI];
        frow[li] = 0;
        if (!isfinite(pr[li])) lc.unverifiable++;
        else if (!(fabs(rr - pr[li]) <= taur[li])) { frow[li] = 1; nr++; }
      }
      for (int64_t lj = 0; lj < nJt; ++lj) {
        double rcs = 0.0;
        for (int64_t li = 0; li < mI; ++li) rcs = rcs + out[li + lj * mI];
        fcol[lj] = 0;
        if (!isfinite(pc[lj])) lc.unverifiable++;
        else if (!(fabs(rcs - pc[lj]) <= tauc[lj])) { fcol[lj] = 1; nc++; }
      }
      lc.flagged_rows += nr;
      lc.flagged_cols += nc;

      /* 4. locate and correct */
      if (nr > 0 || nc > 0) {
        if (nr > 0 && nc > 0 && nr * nc <= CAP_X)
          for (int64_t li = 0; li < mI; ++li)
            if (frow[li])
              for (int64_t lj = 0; lj < nJt; ++lj)
                if (fcol[lj])
                  recompute_elem(&p, out, mI, li, lj, i0 + li, j0 + lj, cin, (int32_t)t, 0,
                                 &lc, lloc, cap, &lnloc);
        /* re-verify the flagged rows and columns */
        for (int64_t li = 0; li < mI; ++li)
          if (frow[li]) {
            double rr = 0.0;
            for (int64_t lj = 0; lj < nJt; ++lj) rr = rr + out[li + lj * mI];
            frow[li] = !(fabs(rr - pr[li]) <= taur[li]);
          }
        for (int64_t lj = 0; lj < nJt; ++lj)
          if (fcol[lj]) {
            double rcs = 0.0;
            for (int64_t li = 0; li < mI; ++li) rcs = rcs + out[li + lj * mI];
            fcol[lj] = !(fabs(rcs - pc[lj]) <= tauc[lj]);
          }
        /* fallback: recompute whole segments of rows/columns still failing */
        int any = 0;
        memset(seg, 0, (size_t)(BM * BN));
        for (int64_t li = 0; li < mI; ++li)
          if (frow[li]) { any = 1; for (int64_t lj = 0; lj < nJt; ++lj) seg[li + lj * mI] = 1; }
        for (int64_t lj = 0; lj < nJt; ++lj)
          if (fcol[lj]) { any = 1; for (int64_t li = 0; li < mI; ++li) seg[li + lj * mI] = 1; }
        if (any) {
          for (int64_t lj = 0; lj < nJt; ++lj)
            for (int64_t li = 0; li < mI; ++li)
              if (seg[li + lj * mI])
                recompute_elem(&p, out, mI, li, lj, i0 + li, j0 + lj, cin, (int32_t)t, 1,
                               &lc, lloc, cap, &lnloc);
          for (int64_t li = 0; li < mI; ++li)
            if (frow[li]) {
              double rr = 0.0;
              for (int64_t lj = 0; lj < nJt; ++lj) rr = rr + out[li + lj * mI];
              if (!(fabs(rr - pr[li]) <= taur[li])) lc.checksum_only++;
            }
          for (int64_t lj = 0; lj < nJt; ++lj)
            if (fcol[lj]) {
              double rcs = 0.0;
              for (int64_t li = 0; li < mI; ++li) rcs = rcs + out[li + lj * mI];
              if (!(fabs(rcs - pc[lj]) <= tauc[lj])) lc.checksum_only++;
            }
        }
      }

      /* 5. store the tile and merge the tile's report */
      for (int64_t lj = 0; lj < nJt; ++lj)
        for (int64_t li = 0; li < mI; ++li) C[(i0 + li) + (j0 + lj) * ldc] = out[li + lj * mI];
#ifdef _OPENMP
#pragma omp critical(orc_report)
#endif
      {
        cnt->detected += lc.detected;
        cnt->corrected += lc.corrected;
        cnt->checksum_only += lc.checksum_only;
        cnt->unverifiable += lc.unverifiable;
        cnt->flagged_rows += lc.flagged_rows;
        cnt->flagged_cols += lc.flagged_cols;
        cnt->recomputed += lc.recomputed;
        for (int64_t q = 0; q < lnloc && q < cap; ++q)
          if (*nloc + q < cap) locs[*nloc + q] = lloc[q];
        *nloc += lnloc;
      }
    }
    free(cin); free(out); free(acc); free(acsI); free(bcsJ); free(pr); free(pc);
    free(taur); free(tauc); free(frow); free(fcol); free(seg); free(lloc);
  }
  (void)nflips;
  return 0;
}
