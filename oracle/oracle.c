/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the fused
 * sufficient-statistics pass (row count n, column sums s = X^T 1 and the
 * upper triangle of S = X^T X) over the paper's Table 1 table and over
 * arbitrary typed columns.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it follows (section names of arxiv 2604.23826, "Building a
 * GPU-Accelerated Multivariate Statistics Platform"):
 *   - Table 1 ("Dataset used in this study"): the twelve column formulas.
 *   - "Data Representation and Sufficient Statistics": column sums and X^T X
 *     accumulated in one pass; mean, covariance and correlation from them.
 *   - "Numerical Considerations": X^T X and N mu mu^T formed separately cancel
 *     catastrophically, so this oracle never does that for real-valued data:
 *     integer-valued columns are summed exactly in __int128, real-valued
 *     products in double-double, and the covariance is the textbook two-pass
 *     form (Chan, Golub & LeVeque 1983), deliberately unlike the one-pass
 *     form of the GPU path.
 *   - "Principal Component Analysis Results": eigenpairs of the p x p
 *     matrix by "standard numerical linear algebra routines"; here cyclic
 *     Jacobi (Golub & Van Loan, Matrix Computations, Sec. 8.5).
 * The random numbers behind Table 1's randBetween are drawn with
 * Philox4x32-10, written from its published definition (Salmon, Moraes,
 * Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 4).
 *
 * Readings where the paper is silent:
 *   - randBetween(a, b) is inclusive on both ends; row i (0-based) draws
 *     (u0, u1, u2, u3) = Philox4x32-10(counter = (i_lo, i_hi, 0, 0),
 *     key = (seed_lo, seed_hi)) and maps u to a + floor(u * (b - a + 1) / 2^32).
 *   - int() truncates toward zero, round() is C's round (half away from zero).
 *   - the identifier A = i + 1 (1-based).
 *
 * Parity status: every exported function here is pinned by tests under
 * tests/ (closed forms, brute force with exact rationals, an independent
 * histogram formulation, published Philox answers, Table 2 -> Table 3).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread (oracle/build.py).
 * -ffp-contract=off matters: the error-free transformations below must not be
 * fused by the compiler.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): a 10-round Feistel-like bijection on */
/* a 128-bit counter, keyed by 64 bits; the round multiplies words 0 and 2 by */
/* two constants, and the key is bumped by two Weyl constants between rounds. */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Table 1 rows.                                                              */
/* Column order: A B C D E F G H cotC I J K  (indices 0..11).                 */
/* Integer-valued columns go to ival[], real-valued ones (cotC, J) to rval[]. */
/* ------------------------------------------------------------------------ */
enum { T1_P = 12, T1_COTC = 8, T1_J = 10 };

int orc_table1_is_real(int j) { return j == T1_COTC || j == T1_J; }

/* randBetween(lo, hi), inclusive, from one 32-bit uniform word. */
static int64_t rand_between(uint32_t u, int64_t lo, int64_t hi) {
  uint64_t span = (uint64_t)(hi - lo + 1);
  return lo + (int64_t)(((uint64_t)u * span) >> 32);
}

/* The derived columns E..K of Table 1 as functions of (B, C, D), each
 * written exactly as the table prints it. */
static void table1_derived(int64_t B, int64_t C, int64_t D, int64_t iv[T1_P], double rv[T1_P]) {
  double b = (double)B, c = (double)C, d = (double)D;
  double E = (double)(int64_t)(log(c) / log(b) * 100.0);          /* int(log C / log B * 100) */
  double F = round((log(d) / log(b)) * 10000.0);                   /* round(log D / log B * 10000) */
  double G = (double)(int64_t)(fabs(cos(c)) * 100.0);             /* int(|cos C| * 100) */
  double H = (double)(int64_t)(fabs(sin(d)) * 100.0);             /* int(|sin D| * 100) */
  double cotC = 1.0 / tan(c);                                      /* 1.0 / tan(C) */
  double I = round(fabs(cotC) * 1000.0);                           /* round(|cotC| * 1000) */
  double J = fabs(tan(d));                                         /* |tan D| */
  int64_t K = D / C;                                               /* integer division */
  iv[4] = (int64_t)E;
  iv[5] = (int64_t)F;
  iv[6] = (int64_t)G;
  iv[7] = (int64_t)H;
  iv[8] = 0;
  rv[8] = cotC;
  iv[9] = (int64_t)I;
  iv[10] = 0;
  rv[10] = J;
  iv[11] = K;
}

/* One row of Table 1: row index i is 0-based, the identifier A = i + 1. */
void orc_table1_row(uint64_t seed, uint64_t i, int64_t iv[T1_P], double rv[T1_P]) {
  uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t u[4];
  orc_philox4x32_10(ctr, key, u);
  for (int j = 0; j < T1_P; ++j) { iv[j] = 0; rv[j] = 0.0; }
  int64_t B = rand_between(u[0], 3, 8);
  int64_t C = rand_between(u[1], 1, 10);
  int64_t D = rand_between(u[2], 1, 100);
  iv[0] = (int64_t)i + 1;
  iv[1] = B;
  iv[2] = C;
  iv[3] = D;
  table1_derived(B, C, D, iv, rv);
  for (int j = 0; j < T1_P; ++j)
    if (!orc_table1_is_real(j)) rv[j] = (double)iv[j];
}

/* n rows starting at row0, row-major n x 12 into both arrays (either may be NULL). */
void orc_table1_rows(uint64_t seed, uint64_t row0, int64_t n, int64_t* ivals, double* rvals) {
  int64_t iv[T1_P];
  double rv[T1_P];
  for (int64_t r = 0; r < n; ++r) {
    orc_table1_row(seed, row0 + (uint64_t)r, iv, rv);
    for (int j = 0; j < T1_P; ++j) {
      if (ivals) ivals[r * T1_P + j] = iv[j];
      if (rvals) rvals[r * T1_P + j] = rv[j];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Double-double arithmetic: Knuth's TwoSum, the FMA form of Dekker's         */
/* TwoProduct, and the accurate double-double add (both halves summed with    */
/* TwoSum, then renormalised), as in Hida, Li & Bailey's QD library paper.    */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}
static inline dd fast_two_sum(double a, double b) { /* requires |a| >= |b| or a == 0 */
  double s = a + b;
  double e = b - (s - a);
  dd r = {s, e};
  return r;
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  dd r = {p, e};
  return r;
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd dd_from_double(double a) { dd r = {a, 0.0}; return r; }
/* a / b by one Newton correction of the double quotient. */
static inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul(dd_from_double(q1), b)));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul(dd_from_double(q2), b)));
  double q3 = r.hi / b.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, dd_from_double(q3));
}
/* Exact for |v| < 2^106. */
static inline dd dd_from_i128(i128 v) {
  double hi = (double)v;
  i128 rest = v - (i128)hi;
  dd r = {hi, (double)rest};
  return fast_two_sum(r.hi, r.lo);
}

/* ------------------------------------------------------------------------ */
/* Exact accumulation of (n, s, S) over typed columns.                        */
/* kinds[j] = 0: integer-valued (given as int64), 1: real-valued (double).    */
/* Pairs of two integer columns are summed exactly in __int128; a pair with a */
/* real column sums the exact product (TwoProduct) in double-double.          */
/* Packed upper-triangle index of (j, k), j <= k: j*p - j*(j-1)/2 + (k - j).  */
/* ------------------------------------------------------------------------ */
#define ORC_MAXP 256

typedef struct {
  int p;
  int64_t n;
  i128* s_int;   /* p */
  dd* s_dd;      /* p */
  i128* S_int;   /* p(p+1)/2 */
  dd* S_dd;      /* p(p+1)/2 */
  int bad;       /* set when an integer value cannot be carried exactly as a double */
} acc_t;

static int tri_index(int p, int j, int k) { return j * p - j * (j - 1) / 2 + (k - j); }

static int acc_init(acc_t* a, int p) {
  size_t T = (size_t)p * (p + 1) / 2;
  a->p = p;
  a->n = 0;
  a->bad = 0;
  a->s_int = calloc(p, sizeof(i128));
  a->s_dd = calloc(p, sizeof(dd));
  a->S_int = calloc(T, sizeof(i128));
  a->S_dd = calloc(T, sizeof(dd));
  return (a->s_int && a->s_dd && a->S_int && a->S_dd) ? 0 : -1;
}
static void acc_free(acc_t* a) {
  free(a->s_int); free(a->s_dd); free(a->S_int); free(a->S_dd);
}
/* dst += src, entry by entry. */
static void acc_merge(acc_t* dst, const acc_t* src) {
  int p = dst->p;
  size_t T = (size_t)p * (p + 1) / 2;
  dst->n += src->n;
  dst->bad |= src->bad;
  for (int j = 0; j < p; ++j) {
    if (__builtin_add_overflow(dst->s_int[j], src->s_int[j], &dst->s_int[j])) dst->bad |= 2;
    dst->s_dd[j] = dd_add(dst->s_dd[j], src->s_dd[j]);
  }
  for (size_t t = 0; t < T; ++t) {
    if (__builtin_add_overflow(dst->S_int[t], src->S_int[t], &dst->S_int[t])) dst->bad |= 2;
    dst->S_dd[t] = dd_add(dst->S_dd[t], src->S_dd[t]);
  }
}

/* One row: x_int[j] valid where kinds[j] == 0, x_real[j] where kinds[j] == 1. */
static void acc_row(acc_t* a, const int* kinds, const int64_t* xi, const double* xr) {
  int p = a->p;
  double xd[ORC_MAXP];
  int any_real = 0;
  for (int j = 0; j < p; ++j) any_real |= kinds[j];
  a->n += 1;
  for (int j = 0; j < p; ++j) {
    if (kinds[j] == 0) {
      if (any_real && (xi[j] > ((int64_t)1 << 53) || xi[j] < -((int64_t)1 << 53))) a->bad = 1;
      xd[j] = (double)xi[j];
      a->s_int[j] += (i128)xi[j];
    } else {
      xd[j] = xr[j];
      a->s_dd[j] = dd_add(a->s_dd[j], dd_from_double(xr[j]));
    }
  }
  int t = 0;
  for (int j = 0; j < p; ++j) {
    for (int k = j; k < p; ++k, ++t) {
      if (kinds[j] == 0 && kinds[k] == 0) {
        i128 prod = (i128)xi[j] * (i128)xi[k]; /* |prod| < 2^126: cannot overflow */
        if (__builtin_add_overflow(a->S_int[t], prod, &a->S_int[t])) a->bad |= 2;
      } else
        a->S_dd[t] = dd_add(a->S_dd[t], two_prod(xd[j], xd[k]));
    }
  }
}

static void put_i128(int64_t* out2, i128 v) {
  out2[0] = (int64_t)(uint64_t)v;              /* low 64 bits  */
  out2[1] = (int64_t)(v >> 64);                /* high 64 bits */
}
static i128 get_i128(const int64_t* in2) {
  return (i128)(((unsigned __int128)(uint64_t)in2[1] << 64) | (uint64_t)in2[0]);
}

static void acc_export(const acc_t* a, int64_t* n_out, int64_t* s_int, double* s_dd, int64_t* S_int,
                       double* S_dd) {
  int p = a->p;
  size_t T = (size_t)p * (p + 1) / 2;
  *n_out = a->n;
  for (int j = 0; j < p; ++j) {
    put_i128(s_int + 2 * j, a->s_int[j]);
    s_dd[2 * j] = a->s_dd[j].hi;
    s_dd[2 * j + 1] = a->s_dd[j].lo;
  }
  for (size_t t = 0; t < T; ++t) {
    put_i128(S_int + 2 * t, a->S_int[t]);
    S_dd[2 * t] = a->S_dd[t].hi;
    S_dd[2 * t + 1] = a->S_dd[t].lo;
  }
}

/* --- threading: contiguous row ranges, partials merged in thread order --- */
typedef struct {
  int p;
  const int* kinds;
  const void* const* cols;
  int64_t r0, r1;
  acc_t acc;
  /* Table 1 mode */
  int table1;
  uint64_t seed;
  uint64_t row0;
} cols_job_t;

static void* cols_worker(void* arg) {
  cols_job_t* job = (cols_job_t*)arg;
  int p = job->p;
  int64_t xi[ORC_MAXP];
  double xr[ORC_MAXP];
  for (int64_t r = job->r0; r < job->r1; ++r) {
    if (job->table1) {
      orc_table1_row(job->seed, job->row0 + (uint64_t)r, xi, xr);
    } else {
      for (int j = 0; j < p; ++j) {
        if (job->kinds[j] == 0)
          xi[j] = ((const int64_t*)job->cols[j])[r];
        else
          xr[j] = ((const double*)job->cols[j])[r];
      }
    }
    acc_row(&job->acc, job->kinds, xi, xr);
  }
  return NULL;
}

static const int T1_KINDS[T1_P] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 1, 0};

static int run_cols(int table1, uint64_t seed, uint64_t row0, int p, const int* kinds, const void* const* cols,
                    int64_t n, int nthreads, int64_t* n_out, int64_t* s_int, double* s_dd, int64_t* S_int,
                    double* S_dd) {
  if (p < 1 || p > ORC_MAXP || n < 0) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n && n > 0) nthreads = (int)n;
  cols_job_t* jobs = calloc(nthreads, sizeof(cols_job_t));
  pthread_t* th = calloc(nthreads, sizeof(pthread_t));
  if (!jobs || !th) return -2;
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].p = p;
    jobs[t].kinds = kinds;
    jobs[t].cols = cols;
    jobs[t].r0 = n * t / nthreads;
    jobs[t].r1 = n * (t + 1) / nthreads;
    jobs[t].table1 = table1;
    jobs[t].seed = seed;
    jobs[t].row0 = row0;
    if (acc_init(&jobs[t].acc, p)) rc = -2;
  }
  if (rc == 0) {
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, cols_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    for (int t = 1; t < nthreads; ++t) acc_merge(&jobs[0].acc, &jobs[t].acc);
    acc_export(&jobs[0].acc, n_out, s_int, s_dd, S_int, S_dd);
    if (jobs[0].acc.bad & 2) rc = 2;
    else if (jobs[0].acc.bad) rc = 1;
  }
  for (int t = 0; t < nthreads; ++t) acc_free(&jobs[t].acc);
  free(jobs);
  free(th);
  return rc;
}

/* (n, s, S) over typed columns.  Returns 0 on success, 1 if an integer value
 * paired with a real column was too large to be carried exactly as a double,
 * 2 if an integer sum left the __int128 range. */
int orc_stats_columns(int p, const int* kinds, const void* const* cols, int64_t n, int nthreads, int64_t* n_out,
                      int64_t* s_int, double* s_dd, int64_t* S_int, double* S_dd) {
  return run_cols(0, 0, 0, p, kinds, cols, n, nthreads, n_out, s_int, s_dd, S_int, S_dd);
}

/* (n, s, S) of Table 1 rows [row0, row0 + n), generated row by row. */
int orc_stats_table1(uint64_t seed, uint64_t row0, int64_t n, int nthreads, int64_t* n_out, int64_t* s_int,
                     double* s_dd, int64_t* S_int, double* S_dd) {
  return run_cols(1, seed, row0, T1_P, T1_KINDS, NULL, n, nthreads, n_out, s_int, s_dd, S_int, S_dd);
}

/* ------------------------------------------------------------------------ */
/* Histogram formulation of Table 1 (an independent check of the per-row      */
/* oracle at any n): every column except A is a function of the cell (B,C,D), */
/* so S_jk = sum over cells of count * f_j * f_k and S_Aj = sum over cells of */
/* (sum of A in the cell) * f_j.  Only the Philox draws are made per row.     */
/* ------------------------------------------------------------------------ */
#define NCELL (6 * 10 * 100)
static int cell_of(int64_t B, int64_t C, int64_t D) { return (int)(((B - 3) * 10 + (C - 1)) * 100 + (D - 1)); }

typedef struct {
  uint64_t seed, row0;
  int64_t r0, r1;
  int64_t count[NCELL];
  i128 sumA[NCELL];
  i128 sumA2;
} hist_job_t;

static void* hist_worker(void* arg) {
  hist_job_t* h = (hist_job_t*)arg;
  uint32_t key[2] = {(uint32_t)h->seed, (uint32_t)(h->seed >> 32)};
  for (int64_t r = h->r0; r < h->r1; ++r) {
    uint64_t i = h->row0 + (uint64_t)r;
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0u, 0u};
    uint32_t u[4];
    orc_philox4x32_10(ctr, key, u);
    int c = cell_of(rand_between(u[0], 3, 8), rand_between(u[1], 1, 10), rand_between(u[2], 1, 100));
    i128 A = (i128)i + 1;
    h->count[c] += 1;
    h->sumA[c] += A;
    h->sumA2 += A * A;
  }
  return NULL;
}

/* Cell counts and per-cell identifier sums (as (lo, hi) pairs) plus sum A^2. */
int orc_hist_table1(uint64_t seed, uint64_t row0, int64_t n, int nthreads, int64_t* count, int64_t* sumA,
                    int64_t* sumA2) {
  if (n < 0) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  hist_job_t* jobs = calloc(nthreads, sizeof(hist_job_t));
  pthread_t* th = calloc(nthreads, sizeof(pthread_t));
  if (!jobs || !th) return -2;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].seed = seed;
    jobs[t].row0 = row0;
    jobs[t].r0 = n * t / nthreads;
    jobs[t].r1 = n * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, hist_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  i128 a2 = 0;
  for (int c = 0; c < NCELL; ++c) {
    int64_t cnt = 0;
    i128 sa = 0;
    for (int t = 0; t < nthreads; ++t) {
      cnt += jobs[t].count[c];
      sa += jobs[t].sumA[c];
    }
    count[c] = cnt;
    put_i128(sumA + 2 * c, sa);
  }
  for (int t = 0; t < nthreads; ++t) a2 += jobs[t].sumA2;
  put_i128(sumA2, a2);
  free(jobs);
  free(th);
  return 0;
}

/* (n, s, S) of Table 1 from the histogram, same output layout as orc_stats_table1. */
int orc_stats_table1_hist(uint64_t seed, uint64_t row0, int64_t n, int nthreads, int64_t* n_out, int64_t* s_int,
                          double* s_dd, int64_t* S_int, double* S_dd) {
  int64_t* count = calloc(NCELL, sizeof(int64_t));
  int64_t* sumA = calloc(2 * NCELL, sizeof(int64_t));
  int64_t sumA2[2];
  if (!count || !sumA) return -2;
  int rc = orc_hist_table1(seed, row0, n, nthreads, count, sumA, sumA2);
  if (rc) return rc;
  acc_t a;
  if (acc_init(&a, T1_P)) return -2;
  i128 totA = 0;
  for (int c = 0; c < NCELL; ++c) totA += get_i128(sumA + 2 * c);
  a.n = n;
  a.s_int[0] = totA;
  a.S_int[tri_index(T1_P, 0, 0)] = get_i128(sumA2);
  for (int B = 3; B <= 8; ++B)
    for (int C = 1; C <= 10; ++C)
      for (int D = 1; D <= 100; ++D) {
        int c = cell_of(B, C, D);
        int64_t cnt = count[c];
        if (cnt == 0) continue;
        i128 sa = get_i128(sumA + 2 * c);
        int64_t iv[T1_P] = {0};
        double rv[T1_P] = {0};
        iv[1] = B; iv[2] = C; iv[3] = D;
        table1_derived(B, C, D, iv, rv);
        for (int j = 1; j < T1_P; ++j)
          if (!T1_KINDS[j]) rv[j] = (double)iv[j];
        dd ddcnt = dd_from_double((double)cnt);
        dd ddsa = dd_from_i128(sa);
        for (int j = 1; j < T1_P; ++j) {
          if (T1_KINDS[j] == 0)
            a.s_int[j] += (i128)cnt * iv[j];
          else
            a.s_dd[j] = dd_add(a.s_dd[j], dd_mul(ddcnt, dd_from_double(rv[j])));
          /* identifier cross term, A <= j */
          int tA = tri_index(T1_P, 0, j);
          if (T1_KINDS[j] == 0)
            a.S_int[tA] += sa * iv[j];
          else
            a.S_dd[tA] = dd_add(a.S_dd[tA], dd_mul(ddsa, dd_from_double(rv[j])));
          for (int k = j; k < T1_P; ++k) {
            int t = tri_index(T1_P, j, k);
            if (T1_KINDS[j] == 0 && T1_KINDS[k] == 0)
              a.S_int[t] += (i128)cnt * ((i128)iv[j] * iv[k]);
            else
              a.S_dd[t] = dd_add(a.S_dd[t], dd_mul(ddcnt, two_prod(rv[j], rv[k])));
          }
        }
      }
  acc_export(&a, n_out, s_int, s_dd, S_int, S_dd);
  acc_free(&a);
  free(count);
  free(sumA);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-pass covariance (textbook form): pass 1 the means, in double-double;  */
/* pass 2 the sum of (x_j - mean_j)(x_k - mean_k) in double-double, divided   */
/* by n - 1.  All p columns; the caller drops the identifier.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int p;
  const int* kinds;
  const void* const* cols;
  int table1;
  uint64_t seed, row0;
  int64_t r0, r1;
  const dd* mean;
  dd* C; /* p*p, full */
} cov_job_t;

static void* cov_worker(void* arg) {
  cov_job_t* job = (cov_job_t*)arg;
  int p = job->p;
  int64_t xi[ORC_MAXP];
  double xr[ORC_MAXP];
  dd dev[ORC_MAXP];
  for (int64_t r = job->r0; r < job->r1; ++r) {
    if (job->table1) {
      orc_table1_row(job->seed, job->row0 + (uint64_t)r, xi, xr);
      for (int j = 0; j < p; ++j)
        if (!job->kinds[j]) xr[j] = (double)xi[j];
    } else {
      for (int j = 0; j < p; ++j)
        xr[j] = job->kinds[j] ? ((const double*)job->cols[j])[r] : (double)((const int64_t*)job->cols[j])[r];
    }
    for (int j = 0; j < p; ++j) dev[j] = dd_add(dd_from_double(xr[j]), dd_neg(job->mean[j]));
    for (int j = 0; j < p; ++j)
      for (int k = j; k < p; ++k) job->C[j * p + k] = dd_add(job->C[j * p + k], dd_mul(dev[j], dev[k]));
  }
  return NULL;
}

static int run_cov(int table1, uint64_t seed, uint64_t row0, int p, const int* kinds, const void* const* cols,
                   int64_t n, int nthreads, double* cov) {
  if (p < 1 || p > ORC_MAXP || n < 2) return -1;
  size_t T = (size_t)p * (p + 1) / 2;
  int64_t n_out;
  int64_t* s_int = calloc(2 * p, sizeof(int64_t));
  double* s_dd = calloc(2 * p, sizeof(double));
  int64_t* S_int = calloc(2 * T, sizeof(int64_t));
  double* S_dd = calloc(2 * T, sizeof(double));
  dd* mean = calloc(p, sizeof(dd));
  if (!s_int || !s_dd || !S_int || !S_dd || !mean) return -2;
  /* pass 1: exact column sums -> means */
  int rc = run_cols(table1, seed, row0, p, kinds, cols, n, nthreads, &n_out, s_int, s_dd, S_int, S_dd);
  if (rc < 0) return rc;
  dd ddn = dd_from_double((double)n);
  for (int j = 0; j < p; ++j) {
    dd s = kinds[j] ? (dd){s_dd[2 * j], s_dd[2 * j + 1]} : dd_from_i128(get_i128(s_int + 2 * j));
    mean[j] = dd_div(s, ddn);
  }
  /* pass 2 */
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = (int)n;
  cov_job_t* jobs = calloc(nthreads, sizeof(cov_job_t));
  pthread_t* th = calloc(nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].p = p;
    jobs[t].kinds = kinds;
    jobs[t].cols = cols;
    jobs[t].table1 = table1;
    jobs[t].seed = seed;
    jobs[t].row0 = row0;
    jobs[t].r0 = n * t / nthreads;
    jobs[t].r1 = n * (t + 1) / nthreads;
    jobs[t].mean = mean;
    jobs[t].C = calloc((size_t)p * p, sizeof(dd));
    pthread_create(&th[t], NULL, cov_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  dd ddn1 = dd_from_double((double)(n - 1));
  for (int j = 0; j < p; ++j)
    for (int k = j; k < p; ++k) {
      dd c = jobs[0].C[j * p + k];
      for (int t = 1; t < nthreads; ++t) c = dd_add(c, jobs[t].C[j * p + k]);
      double v = dd_div(c, ddn1).hi;
      cov[j * p + k] = v;
      cov[k * p + j] = v;
    }
  for (int t = 0; t < nthreads; ++t) free(jobs[t].C);
  free(jobs); free(th); free(s_int); free(s_dd); free(S_int); free(S_dd); free(mean);
  return rc;
}

/* Full p x p covariance (divisor n - 1) of typed columns, two-pass. */
int orc_cov_twopass_columns(int p, const int* kinds, const void* const* cols, int64_t n, int nthreads, double* cov) {
  return run_cov(0, 0, 0, p, kinds, cols, n, nthreads, cov);
}

/* Full 12 x 12 covariance of Table 1 rows [row0, row0 + n), two-pass. */
int orc_cov_twopass_table1(uint64_t seed, uint64_t row0, int64_t n, int nthreads, double* cov) {
  return run_cov(1, seed, row0, T1_P, T1_KINDS, NULL, n, nthreads, cov);
}

/* corr_jk = cov_jk / sqrt(cov_jj cov_kk); NaN where a variance is zero. */
void orc_corr_from_cov(int p, const double* cov, double* corr) {
  for (int j = 0; j < p; ++j)
    for (int k = 0; k < p; ++k) {
      double d = sqrt(cov[j * p + j]) * sqrt(cov[k * p + k]);
      corr[j * p + k] = (d > 0.0) ? cov[j * p + k] / d : NAN;
    }
  for (int j = 0; j < p; ++j)
    if (cov[j * p + j] > 0.0) corr[j * p + j] = 1.0;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigensolver for a symmetric p x p matrix (Golub & Van Loan,  */
/* Matrix Computations, Sec. 8.5): sweep over all (r, s) pairs, each rotation */
/* zeroing a_rs, until the off-diagonal mass is negligible.                  */
/* Output: eigenvalues descending; evecs row k = eigenvector k, its sign      */
/* chosen so that its largest-magnitude component is positive.               */
/* ------------------------------------------------------------------------ */
int orc_jacobi(int p, const double* Ain, double* evals, double* evecs, int max_sweeps) {
  double* A = malloc(sizeof(double) * p * p);
  double* V = malloc(sizeof(double) * p * p);
  if (!A || !V) return -2;
  memcpy(A, Ain, sizeof(double) * p * p);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) V[i * p + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < p * p; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int r = 0; r < p; ++r)
      for (int s = r + 1; s < p; ++s) off += A[r * p + s] * A[r * p + s];
    if (sqrt(2.0 * off) <= 1e-17 * fro || off == 0.0) break;
    for (int r = 0; r < p; ++r)
      for (int s = r + 1; s < p; ++s) {
        double ars = A[r * p + s];
        if (ars == 0.0) continue;
        double theta = (A[s * p + s] - A[r * p + r]) / (2.0 * ars);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double sn = t * c;
        /* A <- J^T A J on rows/cols r, s */
        for (int k = 0; k < p; ++k) {
          double akr = A[k * p + r], aks = A[k * p + s];
          A[k * p + r] = c * akr - sn * aks;
          A[k * p + s] = sn * akr + c * aks;
        }
        for (int k = 0; k < p; ++k) {
          double ark = A[r * p + k], ask = A[s * p + k];
          A[r * p + k] = c * ark - sn * ask;
          A[s * p + k] = sn * ark + c * ask;
        }
        A[r * p + s] = 0.0;
        A[s * p + r] = 0.0;
        /* V <- V J (columns of V are eigenvectors) */
        for (int k = 0; k < p; ++k) {
          double vkr = V[k * p + r], vks = V[k * p + s];
          V[k * p + r] = c * vkr - sn * vks;
          V[k * p + s] = sn * vkr + c * vks;
        }
      }
  }
  /* sort descending (selection sort: p is small) */
  int* order = malloc(sizeof(int) * p);
  for (int i = 0; i < p; ++i) order[i] = i;
  for (int i = 0; i < p; ++i) {
    int best = i;
    for (int j = i + 1; j < p; ++j)
      if (A[order[j] * p + order[j]] > A[order[best] * p + order[best]]) best = j;
    int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
  }
  for (int k = 0; k < p; ++k) {
    int col = order[k];
    evals[k] = A[col * p + col];
    int imax = 0;
    for (int i = 1; i < p; ++i)
      if (fabs(V[i * p + col]) > fabs(V[imax * p + col])) imax = i;
    double sg = V[imax * p + col] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < p; ++i) evecs[k * p + i] = sg * V[i * p + col];
  }
  free(order); free(A); free(V);
  return sweep;
}
