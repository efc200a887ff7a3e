/*
 * CPU oracle for the global short-recurrence SPAI methods (MR, LOMR,
 * Frobenius-CG) with per-column hard thresholding, and for the vector PCG
 * that assesses the resulting approximate inverse.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA library.
 *
 * Plain and slow.  Built twice from this one file: single threaded, and with
 * -fopenmp, where the loops over columns (and the PCG's loops over rows) are
 * shared among threads.  Every column is computed by one thread exactly as
 * in the serial build and every sum over columns or rows is taken after its
 * loop with the same pairwise tree, so both builds give the same bits.
 * Every matrix iterate is a list of columns;
 * each column is a row-sorted list of (row, value) with value != 0.  Build
 * with -ffp-contract=off so that a*b+c is never fused implicitly; the only
 * fused operations are the explicit fma()/fmaf() calls below.
 *
 * What each function follows (sections / equations / algorithms of Venkovic
 * & Anzt, "Global Iterative Methods for Sparse Approximate Inverses of SPD
 * Matrices"):
 *   objective f(M) = ||I - A M||_F^2 ............ Sec. 2, Eqs. (2.3)-(2.4)
 *   MR ........................................... Algorithm 1, Eq. (2.6)
 *   CG with Frobenius products ................... Def. 1, Prop. 2, Algorithm 3
 *   LOMR ......................................... Def. 2, Theorem 3, Algorithm 4
 *   hard thresholding ............................ Sec. 6.1, Eq. (6.2)
 *   explicit residual under dropping ............. Sec. 6.2, Table 2
 *   vector PCG assessment ........................ Sec. 7.1.2 / 7.2
 *
 * Readings where the paper is silent (identical on the CUDA side):
 *   - the cap is per column: cap_j = floor(f * nnz(A[:,j])), clamped to
 *     [1, n]; a column is dropped to its cap_j largest |v|, ties going to the
 *     smaller row index; exact zeros are never stored;
 *   - dropping acts on M and on the search direction (P for MR/CG, Z and P
 *     for LOMR), never on R; the coefficients use the full R;
 *   - (A X)[r,j] = fma chain over k ascending: acc = fma(a_rk, x_kj, acc),
 *     acc starting at +0;  R = I - A M with 1 - s on the diagonal, -s off it;
 *   - column inner products: products x*y (rounded, FP64) over the common
 *     rows, summed exactly in a 128-bit fixed point whose unit is 2^(E-110),
 *     E the largest binary exponent among the terms (each term truncated
 *     toward zero to that unit), then rounded once to FP64 (nearest, ties to
 *     even) -- a sum that does not depend on the order of the terms; the
 *     Frobenius product is a balanced pairwise tree over the column partials
 *     j = 0..n-1 zero-padded to a power of two;
 *   - combinations: M + a P -> fma(a, p, m);  S = d Z + g P -> fma(d, z, g*p);
 *     M + S -> m + s;  R + b P -> fma(b, p, r); all in FP64, then rounded to
 *     the value type;
 *   - PCG: SpMV rows are fma chains over ascending column (as the SpGEMM);
 *     vector inner products are pairwise trees over the index range;
 *   - mixed precision: stored values and A are FP32; the SpGEMM chain and the
 *     residual run in FP32; inner products, coefficients and combinations in
 *     FP64 (FP32 inputs promoted exactly).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MR 0
#define ORC_LOMR 1
#define ORC_CG 2
/* Section 5's left-preconditioned variants with Pi = diag(A)^{-1}:
   MR_SPD (Algorithm 5), LOMR_SPD (Algorithm 8), CG (Algorithm 7) */
#define ORC_MR_PI 3
#define ORC_LOMR_PI 4
#define ORC_CG_PI 5

#define ORC_FLAG_CONVERGED 1
#define ORC_FLAG_FALLBACK 2
#define ORC_FLAG_NONFINITE 4

typedef struct {
  int len, cap;
  int *row;
  double *val;
} ocol;

/* Per-thread scratch: the SpGEMM accumulator (a dense value and flag per
 * row, and the list of rows touched), the buffer of inner-product terms and
 * two column buffers.  One per thread (one in the serial build). */
typedef struct {
  double *acc;
  char *seen;
  int *touched;
  double *tmp;
  int tmpcap;
  ocol c1, c2;
} owork;

typedef struct {
  int n;
  int *rowptr, *colind;
  double *a64; /* FP64 values of A */
  double *av;  /* values used by the SPAI arithmetic (FP32-rounded if mixed) */
  double *pi;  /* pi_k = 1 / a_kk in FP64: the diagonal of Pi = diag(A)^{-1} */
  int mixed;
  int *capj;   /* per-column cap */
  int keep_diag; /* 1: every per-column drop keeps the column's diagonal entry */
  /* iterates */
  ocol *M, *P, *Z;
  /* method continuation state */
  int method;  /* -1 none */
  int it;      /* iterations done by current method */
  double rr;   /* CG: numerator of alpha for the current residual, (R,R) or (R,Pi R) */
  double rr_hist; /* CG: ||R_i||^2 of the current residual */
  int64_t spgemm_count;
  /* scratch, one per thread */
  owork *work;
  int nwork;
} orc_state;

#ifdef _OPENMP
#define ORC_TID() omp_get_thread_num()
#else
#define ORC_TID() 0
#endif

static owork *wk(orc_state *s) { return &s->work[ORC_TID()]; }

static double *wtmp(owork *w, int need) {
  if (need > w->tmpcap) {
    int c = w->tmpcap ? w->tmpcap : 64;
    while (c < need) c *= 2;
    w->tmp = (double *)realloc(w->tmp, sizeof(double) * (size_t)c);
    w->tmpcap = c;
  }
  return w->tmp;
}

/* ---------------------------------------------------------------- columns */

static void col_reserve(ocol *c, int need) {
  if (need <= c->cap) return;
  int nc = c->cap ? c->cap : 4;
  while (nc < need) nc *= 2;
  c->row = (int *)realloc(c->row, sizeof(int) * (size_t)nc);
  c->val = (double *)realloc(c->val, sizeof(double) * (size_t)nc);
  c->cap = nc;
}

static void col_push(ocol *c, int r, double v) {
  col_reserve(c, c->len + 1);
  c->row[c->len] = r;
  c->val[c->len] = v;
  c->len++;
}

static void col_free(ocol *c) {
  free(c->row);
  free(c->val);
  c->row = NULL;
  c->val = NULL;
  c->len = c->cap = 0;
}

static void col_copy(ocol *dst, const ocol *src) {
  dst->len = 0;
  col_reserve(dst, src->len);
  memcpy(dst->row, src->row, sizeof(int) * (size_t)src->len);
  memcpy(dst->val, src->val, sizeof(double) * (size_t)src->len);
  dst->len = src->len;
}

static ocol *mat_new(int n) { return (ocol *)calloc((size_t)n, sizeof(ocol)); }

static void mat_free(ocol *m, int n) {
  if (!m) return;
  for (int j = 0; j < n; j++) col_free(&m[j]);
  free(m);
}

static double rv(const orc_state *s, double x) { return s->mixed ? (double)(float)x : x; }

static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------- pairwise summation */

/* Balanced pairwise sum of t[0..L) zero-padded to the next power of two. */
static double pw_rec(const double *t, int L, int64_t lo, int64_t size) {
  if (size == 1) return lo < L ? t[lo] : 0.0;
  int64_t h = size / 2;
  if (lo >= L) return 0.0 + 0.0; /* all-padding subtree */
  return pw_rec(t, L, lo, h) + pw_rec(t, L, lo + h, h);
}

double orc_pairwise(const double *t, int64_t L) {
  int64_t P = 1;
  while (P < L) P *= 2;
  if (L == 0) return 0.0;
  return pw_rec(t, (int)L, 0, P);
}

static double pairwise64(const double *t, int64_t L) {
  int64_t P = 1;
  while (P < L) P *= 2;
  if (L == 0) return 0.0;
  /* same recursion with 64-bit bounds */
  if (P == 1) return t[0];
  double *buf = (double *)malloc(sizeof(double) * (size_t)P);
  for (int64_t i = 0; i < P; i++) buf[i] = i < L ? t[i] : 0.0;
  /* level by level, pairing adjacent entries: identical to the recursion */
  for (int64_t len = P; len > 1; len /= 2)
    for (int64_t i = 0; i < len / 2; i++) buf[i] = buf[2 * i] + buf[2 * i + 1];
  double r = buf[0];
  free(buf);
  return r;
}

/* Order-free sum of finite FP64 terms (see the header): exact 128-bit fixed
 * point with unit 2^(E-110), E = largest exponent, terms truncated toward
 * zero, one final rounding to nearest-even. */
double orc_fixsum(const double *t, int64_t L) {
  int eb = 0;
  for (int64_t i = 0; i < L; i++) {
    uint64_t bits;
    memcpy(&bits, &t[i], 8);
    int b = (int)((bits >> 52) & 0x7ff);
    uint64_t m = bits & ((1ull << 52) - 1);
    if (b == 0 && m == 0) continue;
    if (b == 0) b = 1;
    if (b > eb) eb = b;
  }
  if (eb == 0) return 0.0;
  __int128 S = 0;
  for (int64_t i = 0; i < L; i++) {
    uint64_t bits;
    memcpy(&bits, &t[i], 8);
    int b = (int)((bits >> 52) & 0x7ff);
    uint64_t m = bits & ((1ull << 52) - 1);
    if (b == 0) b = 1;
    else m |= 1ull << 52;
    if (m == 0) continue;
    int sh = b - eb + 58; /* t = m 2^(b-1075); unit = 2^(eb-1133) */
    unsigned __int128 q;
    if (sh >= 0) q = (unsigned __int128)m << sh;
    else if (sh > -64) q = (unsigned __int128)(m >> (-sh));
    else q = 0;
    if (bits >> 63) S -= (__int128)q;
    else S += (__int128)q;
  }
  if (S == 0) return 0.0;
  int neg = S < 0;
  unsigned __int128 U = neg ? (unsigned __int128)(-S) : (unsigned __int128)S;
  int bl = 0;
  for (unsigned __int128 v = U; v; v >>= 1) bl++;
  uint64_t mant;
  int shift = 0;
  if (bl <= 53) {
    mant = (uint64_t)U;
  } else {
    shift = bl - 53;
    mant = (uint64_t)(U >> shift);
    unsigned __int128 rem = U & (((unsigned __int128)1 << shift) - 1);
    unsigned __int128 half = (unsigned __int128)1 << (shift - 1);
    if (rem > half || (rem == half && (mant & 1))) mant++;
  }
  double r = ldexp((double)mant, shift + eb - 1133);
  return neg ? -r : r;
}

/* column inner product over the common rows, Sec. 2 Eq. (2.1) */
static double col_dot(const ocol *x, const ocol *y, owork *w) {
  double *tmp = wtmp(w, x->len < y->len ? x->len : y->len);
  int a = 0, b = 0, L = 0;
  while (a < x->len && b < y->len) {
    if (x->row[a] < y->row[b]) a++;
    else if (x->row[a] > y->row[b]) b++;
    else {
      tmp[L++] = x->val[a] * y->val[b];
      a++;
      b++;
    }
  }
  return orc_fixsum(tmp, L);
}

static double col_nrm2(const ocol *x, owork *w) {
  double *tmp = wtmp(w, x->len);
  for (int a = 0; a < x->len; a++) tmp[a] = x->val[a] * x->val[a];
  return orc_fixsum(tmp, x->len);
}

/* Pi-weighted column inner product (X, Pi Y) of Section 5: each term is the
 * product of the two values (exact for FP32 values) times pi_k, rounded in
 * FP64, and the terms are summed exactly like col_dot's. */
static double col_wdot(const ocol *x, const ocol *y, const double *pi, owork *w) {
  double *tmp = wtmp(w, x->len < y->len ? x->len : y->len);
  int a = 0, b = 0, L = 0;
  while (a < x->len && b < y->len) {
    if (x->row[a] < y->row[b]) a++;
    else if (x->row[a] > y->row[b]) b++;
    else {
      tmp[L++] = (x->val[a] * y->val[b]) * pi[x->row[a]];
      a++;
      b++;
    }
  }
  return orc_fixsum(tmp, L);
}

static double col_wnrm2(const ocol *x, const double *pi, owork *w) {
  double *tmp = wtmp(w, x->len);
  for (int a = 0; a < x->len; a++) tmp[a] = (x->val[a] * x->val[a]) * pi[x->row[a]];
  return orc_fixsum(tmp, x->len);
}

/* ------------------------------------------------------------- operations */

/* out = A X_j (Sec. 6.2: one SpGEMM column) */
static void spgemm_col(orc_state *s, owork *w, const ocol *x, ocol *out) {
  double *acc = w->acc;
  char *seen = w->seen;
  int *touched = w->touched;
  int nt = 0;
  for (int e = 0; e < x->len; e++) {
    int k = x->row[e];
    double xv = x->val[e];
    for (int q = s->rowptr[k]; q < s->rowptr[k + 1]; q++) {
      int r = s->colind[q];
      double a = s->av[q]; /* a_kr == a_rk: A is exactly symmetric */
      if (!seen[r]) {
        seen[r] = 1;
        acc[r] = 0.0;
        touched[nt++] = r;
      }
      if (s->mixed)
        acc[r] = (double)fmaf((float)a, (float)xv, (float)acc[r]);
      else
        acc[r] = fma(a, xv, acc[r]);
    }
  }
  qsort(touched, (size_t)nt, sizeof(int), cmp_int);
  out->len = 0;
  for (int t = 0; t < nt; t++) {
    int r = touched[t];
    double v = acc[r];
    seen[r] = 0;
    if (v != 0.0) col_push(out, r, v);
  }
}

/* R_j = e_j - (A M)_j, exact zeros removed (Algorithm 1, explicit residual) */
static void residual_col(orc_state *s, int j, const ocol *am, ocol *out) {
  out->len = 0;
  int placed = 0;
  for (int e = 0; e <= am->len; e++) {
    int r = e < am->len ? am->row[e] : 2147483647;
    double sv = e < am->len ? am->val[e] : 0.0;
    if (!placed && j < r) { /* diagonal not produced by A M */
      col_push(out, j, 1.0);
      placed = 1;
    }
    if (e == am->len) break;
    double v;
    if (r == j) {
      placed = 1;
      v = s->mixed ? (double)(1.0f - (float)sv) : 1.0 - sv;
    } else {
      v = -sv;
    }
    if (v != 0.0) col_push(out, r, v);
  }
}

/* Z_j = (Pi R)_j: z_k = pi_k r_k in FP64, rounded to the value type, exact
 * zeros removed (Algorithms 5, 7, 8: Z := Pi R) */
static void pi_col(orc_state *s, const ocol *r, ocol *out) {
  out->len = 0;
  for (int e = 0; e < r->len; e++) {
    double z = rv(s, s->pi[r->row[e]] * r->val[e]);
    if (z != 0.0) col_push(out, r->row[e], z);
  }
}

/* pattern union of x and y; value from f(x or 0, y or 0); zeros removed */
enum { COMB_AXPY, COMB_LIN, COMB_ADD };
static void combine_col(orc_state *s, int kind, double c1, double c2, const ocol *x, const ocol *y,
                        ocol *out) {
  out->len = 0;
  int a = 0, b = 0;
  while (a < x->len || b < y->len) {
    int r;
    double xv = 0.0, yv = 0.0;
    if (b >= y->len || (a < x->len && x->row[a] < y->row[b])) {
      r = x->row[a];
      xv = x->val[a++];
    } else if (a >= x->len || y->row[b] < x->row[a]) {
      r = y->row[b];
      yv = y->val[b++];
    } else {
      r = x->row[a];
      xv = x->val[a++];
      yv = y->val[b++];
    }
    double v;
    if (kind == COMB_AXPY) v = fma(c1, yv, xv);          /* x + c1*y        */
    else if (kind == COMB_LIN) v = fma(c1, xv, c2 * yv); /* c1*x + c2*y     */
    else v = xv + yv;                                     /* x + y           */
    v = rv(s, v);
    if (v != 0.0) col_push(out, r, v);
  }
}

typedef struct {
  double a;
  int r;
  int keep; /* 1: the row that is always kept (the column's diagonal) */
} dkey;

static int cmp_dkey(const void *p, const void *q) {
  const dkey *u = (const dkey *)p, *w = (const dkey *)q;
  if (u->keep != w->keep) return w->keep - u->keep;
  if (u->a > w->a) return -1;
  if (u->a < w->a) return 1;
  return (u->r > w->r) - (u->r < w->r);
}

/* hard thresholding of one column to its cap (Sec. 6.1, Eq. (6.2), per
 * column); keep_row >= 0 (the column's diagonal, Appendix A's rule that the
 * diagonal is never dropped) is kept whenever present and counts toward cap */
static void drop_col(ocol *c, int cap, int keep_row) {
  if (c->len <= cap) return;
  dkey *k = (dkey *)malloc(sizeof(dkey) * (size_t)c->len);
  for (int e = 0; e < c->len; e++) {
    k[e].a = fabs(c->val[e]);
    k[e].r = c->row[e];
    k[e].keep = c->row[e] == keep_row;
  }
  qsort(k, (size_t)c->len, sizeof(dkey), cmp_dkey);
  int *keep = (int *)malloc(sizeof(int) * (size_t)cap);
  for (int e = 0; e < cap; e++) keep[e] = k[e].r;
  qsort(keep, (size_t)cap, sizeof(int), cmp_int);
  int w = 0, q = 0;
  for (int e = 0; e < c->len && q < cap; e++) {
    if (c->row[e] == keep[q]) {
      c->row[w] = c->row[e];
      c->val[w] = c->val[e];
      w++;
      q++;
    }
  }
  c->len = w;
  free(k);
  free(keep);
}

/* test hook: drop one row-sorted column in place, returns the new length */
int orc_drop_column(int len, int *rows, double *vals, int cap, int keep_row) {
  ocol c = {0};
  for (int e = 0; e < len; e++) col_push(&c, rows[e], vals[e]);
  drop_col(&c, cap, keep_row);
  for (int e = 0; e < c.len; e++) {
    rows[e] = c.row[e];
    vals[e] = c.val[e];
  }
  int L = c.len;
  col_free(&c);
  return L;
}

/* ------------------------------------------------------------------ state */

orc_state *orc_new(int n, const int *rowptr, const int *colind, const double *vals, int mixed,
                   double cap_factor) {
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  s->n = n;
  int64_t nnz = rowptr[n];
  s->rowptr = (int *)malloc(sizeof(int) * (size_t)(n + 1));
  s->colind = (int *)malloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
  s->a64 = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  s->av = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  memcpy(s->rowptr, rowptr, sizeof(int) * (size_t)(n + 1));
  memcpy(s->colind, colind, sizeof(int) * (size_t)nnz);
  memcpy(s->a64, vals, sizeof(double) * (size_t)nnz);
  s->mixed = mixed;
  for (int64_t q = 0; q < nnz; q++) s->av[q] = mixed ? (double)(float)vals[q] : vals[q];
  s->capj = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; j++) {
    double c = floor(cap_factor * (double)(rowptr[j + 1] - rowptr[j]));
    if (!(c >= 1.0)) c = 1.0;
    if (c > (double)n) c = (double)n;
    s->capj[j] = (int)c;
  }
  s->M = mat_new(n);
  s->P = mat_new(n);
  s->Z = mat_new(n);
#ifdef _OPENMP
  s->nwork = omp_get_max_threads();
#else
  s->nwork = 1;
#endif
  s->work = (owork *)calloc((size_t)s->nwork, sizeof(owork));
  for (int t = 0; t < s->nwork; t++) {
    s->work[t].acc = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    s->work[t].seen = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    s->work[t].touched = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  }
  s->method = -1;
  s->pi = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; j++) {
    double d = 0.0;
    for (int q = rowptr[j]; q < rowptr[j + 1]; q++)
      if (colind[q] == j) d = vals[q];
    s->pi[j] = 1.0 / d;
  }
  /* M_0 = diag(A)^{-1} */
  for (int j = 0; j < n; j++) {
    double d = 0.0;
    for (int q = rowptr[j]; q < rowptr[j + 1]; q++)
      if (colind[q] == j) d = vals[q];
    double m0 = rv(s, 1.0 / d);
    if (m0 != 0.0) col_push(&s->M[j], j, m0);
  }
  return s;
}

void orc_free(orc_state *s) {
  if (!s) return;
  mat_free(s->M, s->n);
  mat_free(s->P, s->n);
  mat_free(s->Z, s->n);
  free(s->rowptr);
  free(s->colind);
  free(s->a64);
  free(s->av);
  free(s->pi);
  free(s->capj);
  for (int t = 0; t < s->nwork; t++) {
    free(s->work[t].acc);
    free(s->work[t].seen);
    free(s->work[t].touched);
    free(s->work[t].tmp);
    col_free(&s->work[t].c1);
    col_free(&s->work[t].c2);
  }
  free(s->work);
  free(s);
}

/* replace M (CSC input), reset method state */
int orc_set_M(orc_state *s, const int *colptr, const int *rowind, const double *vals) {
  for (int j = 0; j < s->n; j++) {
    s->M[j].len = 0;
    s->P[j].len = 0;
    s->Z[j].len = 0;
    for (int q = colptr[j]; q < colptr[j + 1]; q++)
      if (vals[q] != 0.0) col_push(&s->M[j], rowind[q], rv(s, vals[q]));
  }
  s->method = -1;
  s->it = 0;
  return 0;
}

/* every later per-column drop keeps the column's diagonal entry (on != 0) */
void orc_set_keep_diag(orc_state *s, int on) { s->keep_diag = on != 0; }

int64_t orc_nnz(const orc_state *s, int which) {
  const ocol *m = which == 0 ? s->M : which == 1 ? s->P : s->Z;
  int64_t t = 0;
  for (int j = 0; j < s->n; j++) t += m[j].len;
  return t;
}

/* CSC export of M (which=0), P (1) or Z (2) */
void orc_get(const orc_state *s, int which, int *colptr, int *rowind, double *vals) {
  const ocol *m = which == 0 ? s->M : which == 1 ? s->P : s->Z;
  int64_t t = 0;
  colptr[0] = 0;
  for (int j = 0; j < s->n; j++) {
    for (int e = 0; e < m[j].len; e++) {
      rowind[t] = m[j].row[e];
      vals[t] = m[j].val[e];
      t++;
    }
    colptr[j + 1] = (int)t;
  }
}

int64_t orc_spgemm_count(const orc_state *s) { return s->spgemm_count; }

/* -------------------------------------------------------------- the passes */

/* R = I - A M for all columns; returns ||R||_F^2 (global pairwise) */
static double residual_all(orc_state *s, ocol *R, double *partial) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
  for (int j = 0; j < s->n; j++) {
    owork *w = wk(s);
    spgemm_col(s, w, &s->M[j], &w->c1);
    residual_col(s, j, &w->c1, &R[j]);
    partial[j] = col_nrm2(&R[j], w);
  }
  s->spgemm_count++;
  return pairwise64(partial, s->n);
}

static void product_all(orc_state *s, ocol *X, ocol *out) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
  for (int j = 0; j < s->n; j++) spgemm_col(s, wk(s), &X[j], &out[j]);
  s->spgemm_count++;
}

static int isfin(double x) { return !isnan(x) && !isinf(x); }

/*
 * Run `iters` iterations of `method`; continue the current method's
 * recurrence when the previous call used the same method, otherwise start
 * it from the current M with empty directions.
 *   drop: 0 none, 1 top-k per column on M and directions, 2 directions only
 *   resnorm[0..iters]: ||R_i||_F (entries past an early stop are left alone)
 *   coef[2*i], coef[2*i+1]: (alpha_i, 0) for MR, (delta_i, gamma_i) for
 *   LOMR, (alpha_i, beta_{i+1}) for CG.
 *   nnzhist[0..iters] (may be NULL): nnz(M_i) of the iterate whose residual
 *   resnorm[i] records.
 * ORC_MR_PI / ORC_LOMR_PI / ORC_CG_PI run the Pi-preconditioned forms
 * (Algorithms 5, 8, 7 with Pi = diag(A)^{-1}): the direction is built from
 * Z = Pi R instead of R, and every coefficient inner product is the
 * Pi-weighted one; (P, A P) of CG stays unweighted, and resnorm still
 * records ||R_i||_F.
 * Returns the number of iterations done; *flags gets ORC_FLAG_* bits.
 */
int orc_run(orc_state *s, int method, int iters, int drop, double *resnorm, double *coef,
            int64_t *nnzhist, int *flags) {
  int n = s->n;
#define KEEP(j) (s->keep_diag ? (j) : -1)
#define NNZ(i) do { if (nnzhist) nnzhist[i] = orc_nnz(s, 0); } while (0)
  const int use_pi = method >= ORC_MR_PI;
  const int base = use_pi ? method - ORC_MR_PI : method;
  int done = 0;
  *flags = 0;
  int cont = (s->method == method);
  if (!cont) {
    for (int j = 0; j < n; j++) {
      s->P[j].len = 0;
      s->Z[j].len = 0;
    }
    s->it = 0;
    s->method = method;
  }
  ocol *R = mat_new(n), *Q = mat_new(n), *U = mat_new(n), *V = mat_new(n), *S = mat_new(n);
  double *partial = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p2 = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p3 = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p4 = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p5 = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int dropM = (drop == 1), dropD = (drop >= 1);

  if (base == ORC_MR) {
    /* Algorithm 1 with explicit residual, P_i = D(R_i); with Pi
       (Algorithm 5): P_i = D(Pi R_i), alpha = (Pi R, A P) / (A P, Pi A P) */
    for (int i = 0; i < iters; i++) {
      NNZ(i);
      double rr = residual_all(s, R, partial);
      resnorm[i] = sqrt(rr);
      if (rr == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        if (use_pi) pi_col(s, &R[j], &s->P[j]);
        else col_copy(&s->P[j], &R[j]);
        if (dropD) drop_col(&s->P[j], s->capj[j], KEEP(j));
      }
      product_all(s, s->P, Q);
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        p2[j] = use_pi ? col_wdot(&R[j], &Q[j], s->pi, w) : col_dot(&R[j], &Q[j], w);
        p3[j] = use_pi ? col_wnrm2(&Q[j], s->pi, w) : col_nrm2(&Q[j], w);
      }
      double rq = pairwise64(p2, n), qq = pairwise64(p3, n);
      if (qq == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
      double alpha = rq / qq;
      if (!isfin(alpha)) { *flags |= ORC_FLAG_NONFINITE; break; }
      coef[2 * i] = alpha;
      coef[2 * i + 1] = 0.0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        combine_col(s, COMB_AXPY, alpha, 0.0, &s->M[j], &s->P[j], &w->c2);
        if (dropM) drop_col(&w->c2, s->capj[j], KEEP(j));
        col_copy(&s->M[j], &w->c2);
      }
      done++;
      s->it++;
    }
    if (done == iters) {
      NNZ(iters);
      resnorm[iters] = sqrt(residual_all(s, R, partial));
    }
  } else if (base == ORC_LOMR) {
    /* Algorithm 4 with explicit residual: Z_i = D(R_i), P_i = D(S_i),
       M_{i+1} = D(M_i + S_i), S_i = delta Z_i + gamma P_{i-1}. s->P holds
       P_{i-1} between iterations. */
    for (int i = 0; i < iters; i++) {
      NNZ(i);
      double rr = residual_all(s, R, partial);
      resnorm[i] = sqrt(rr);
      if (rr == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        if (use_pi) pi_col(s, &R[j], &s->Z[j]);
        else col_copy(&s->Z[j], &R[j]);
        if (dropD) drop_col(&s->Z[j], s->capj[j], KEEP(j));
      }
      product_all(s, s->Z, U);
      product_all(s, s->P, V);
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        if (use_pi) { /* Algorithm 8: (AZ, Pi AZ), ..., (Pi R, AZ), (Pi R, AP) */
          partial[j] = col_wnrm2(&U[j], s->pi, w);
          p2[j] = col_wnrm2(&V[j], s->pi, w);
          p3[j] = col_wdot(&U[j], &V[j], s->pi, w);
          p4[j] = col_wdot(&U[j], &R[j], s->pi, w);
          p5[j] = col_wdot(&V[j], &R[j], s->pi, w);
        } else {
          partial[j] = col_nrm2(&U[j], w);
          p2[j] = col_nrm2(&V[j], w);
          p3[j] = col_dot(&U[j], &V[j], w);
          p4[j] = col_dot(&U[j], &R[j], w);
          p5[j] = col_dot(&V[j], &R[j], w);
        }
      }
      double uu = pairwise64(partial, n), vv = pairwise64(p2, n), uv = pairwise64(p3, n);
      double ur = pairwise64(p4, n), vr = pairwise64(p5, n);
      if (uu == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
      double t1 = uu * vv, t2 = uv * uv;
      double c = t1 - t2;
      double delta, gamma;
      double eps = 2.220446049250313e-16;
      if (vv == 0.0 || c <= 64.0 * eps * t1) {
        delta = ur / uu;
        gamma = 0.0;
        if (vv != 0.0) *flags |= ORC_FLAG_FALLBACK;
      } else {
        double d1 = vv * ur, d2 = uv * vr;
        double g1 = uu * vr, g2 = uv * ur;
        delta = (d1 - d2) / c;
        gamma = (g1 - g2) / c;
      }
      if (!isfin(delta) || !isfin(gamma)) { *flags |= ORC_FLAG_NONFINITE; break; }
      coef[2 * i] = delta;
      coef[2 * i + 1] = gamma;
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        combine_col(s, COMB_LIN, delta, gamma, &s->Z[j], &s->P[j], &S[j]);
        col_copy(&s->P[j], &S[j]);
        if (dropD) drop_col(&s->P[j], s->capj[j], KEEP(j));
        combine_col(s, COMB_ADD, 0.0, 0.0, &s->M[j], &S[j], &w->c2);
        if (dropM) drop_col(&w->c2, s->capj[j], KEEP(j));
        col_copy(&s->M[j], &w->c2);
      }
      done++;
      s->it++;
    }
    if (done == iters) {
      NNZ(iters);
      resnorm[iters] = sqrt(residual_all(s, R, partial));
    }
  } else if (base == ORC_CG) {
    /* Algorithm 3 with explicit residual: P_0 = D(R_0),
       P_{i+1} = D(R_{i+1} + beta P_i).  With Pi (Algorithm 7): Z = Pi R,
       P_0 = D(Z_0), P_{i+1} = D(Z_{i+1} + beta P_i), alpha = (R, Z)/(P, AP),
       beta = (R_{i+1}, Z_{i+1}) / (R_i, Z_i).  s->P holds P_i, s->rr the
       numerator (R_i, R_i) or (R_i, Pi R_i). */
    double rz;
    NNZ(0);
    if (!cont || s->it == 0) {
      double rr0 = residual_all(s, R, partial);
      resnorm[0] = sqrt(rr0);
      if (use_pi) {
  #pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
        for (int j = 0; j < n; j++) partial[j] = col_wnrm2(&R[j], s->pi, wk(s));
        rz = pairwise64(partial, n);
      } else {
        rz = rr0;
      }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        if (use_pi) pi_col(s, &R[j], &s->P[j]);
        else col_copy(&s->P[j], &R[j]);
        if (dropD) drop_col(&s->P[j], s->capj[j], KEEP(j));
      }
    } else {
      rz = s->rr;
      resnorm[0] = sqrt(s->rr_hist);
    }
    for (int i = 0; i < iters; i++) {
      if (rz == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
      product_all(s, s->P, Q);
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) p2[j] = col_dot(&s->P[j], &Q[j], wk(s));
      double pq = pairwise64(p2, n);
      if (pq == 0.0) { *flags |= ORC_FLAG_CONVERGED; break; }
      double alpha = rz / pq;
      if (!isfin(alpha)) { *flags |= ORC_FLAG_NONFINITE; break; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        combine_col(s, COMB_AXPY, alpha, 0.0, &s->M[j], &s->P[j], &w->c2);
        if (dropM) drop_col(&w->c2, s->capj[j], KEEP(j));
        col_copy(&s->M[j], &w->c2);
      }
      NNZ(i + 1);
      double rr1 = residual_all(s, R, partial);
      resnorm[i + 1] = sqrt(rr1);
      double rz1 = rr1;
      if (use_pi) {
  #pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
        for (int j = 0; j < n; j++) partial[j] = col_wnrm2(&R[j], s->pi, wk(s));
        rz1 = pairwise64(partial, n);
      }
      double beta = rz1 / rz;
      coef[2 * i] = alpha;
      coef[2 * i + 1] = beta;
      done++;
      s->it++;
      s->rr = rz1;
      s->rr_hist = rr1;
      if (rz1 == 0.0) { *flags |= ORC_FLAG_CONVERGED; rz = rz1; break; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
      for (int j = 0; j < n; j++) {
        owork *w = wk(s);
        if (use_pi) {
          pi_col(s, &R[j], &S[j]);
          combine_col(s, COMB_AXPY, beta, 0.0, &S[j], &s->P[j], &w->c2);
        } else {
          combine_col(s, COMB_AXPY, beta, 0.0, &R[j], &s->P[j], &w->c2);
        }
        if (dropD) drop_col(&w->c2, s->capj[j], KEEP(j));
        col_copy(&s->P[j], &w->c2);
      }
      rz = rz1;
    }
  }
  if (*flags & (ORC_FLAG_CONVERGED | ORC_FLAG_NONFINITE)) s->method = -1;
  mat_free(R, n);
  mat_free(Q, n);
  mat_free(U, n);
  mat_free(V, n);
  mat_free(S, n);
  free(partial);
  free(p2);
  free(p3);
  free(p4);
  free(p5);
#undef KEEP
#undef NNZ
  return done;
}

/* ||I - A M||_F in FP64 from the stored M (FP32 values promoted exactly) */
double orc_residual_norm(orc_state *s) {
  int n = s->n;
  double *saved = s->av;
  int mixed = s->mixed;
  s->av = s->a64;
  s->mixed = 0;
  double *partial = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 64) num_threads(s->nwork)
  for (int j = 0; j < n; j++) {
    owork *w = wk(s);
    spgemm_col(s, w, &s->M[j], &w->c1);
    residual_col(s, j, &w->c1, &w->c2);
    partial[j] = col_nrm2(&w->c2, w);
  }
  double rr = pairwise64(partial, n);
  s->av = saved;
  s->mixed = mixed;
  free(partial);
  return sqrt(rr);
}

/* R_j and (A P)_j of one column, for sampled checks of large runs */
int orc_column_residual(orc_state *s, int j, int *rows, double *vals) {
  ocol am = {0}, r = {0};
  spgemm_col(s, &s->work[0], &s->M[j], &am);
  residual_col(s, j, &am, &r);
  int L = r.len;
  if (rows) {
    memcpy(rows, r.row, sizeof(int) * (size_t)L);
    memcpy(vals, r.val, sizeof(double) * (size_t)L);
  }
  col_free(&am);
  col_free(&r);
  return L;
}

/* A x for one column x (rows sorted, len entries) with the method's
 * arithmetic (spgemm_col: fma chains over ascending k in the value type,
 * exact zeros removed); out_rows/out_vals may be NULL to get the length. */
int orc_product_column(orc_state *s, int len, const int *rows, const double *vals, int *out_rows,
                       double *out_vals) {
  ocol x = {0}, y = {0};
  for (int e = 0; e < len; e++) col_push(&x, rows[e], vals[e]);
  spgemm_col(s, &s->work[0], &x, &y);
  int L = y.len;
  if (out_rows) {
    memcpy(out_rows, y.row, sizeof(int) * (size_t)L);
    memcpy(out_vals, y.val, sizeof(double) * (size_t)L);
  }
  col_free(&x);
  col_free(&y);
  return L;
}

/* -------------------------------------------------------------------- PCG */

/* y_i = fma chain over row i, ascending column: acc = fma(m_ij, x_j, acc) */
static void spmv_rows(int n, const int *rp, const int *ci, const double *v, const double *x, double *y,
                      double *tmp) {
  (void)tmp;
#pragma omp parallel for schedule(static, 4096)
  for (int i = 0; i < n; i++) {
    double acc = 0.0;
    for (int q = rp[i]; q < rp[i + 1]; q++) acc = fma(v[q], x[ci[q]], acc);
    y[i] = acc;
  }
}

/* The FP32-values SpMV of the mixed PCG: the operand is rounded to FP32,
 * each row is an FP32 fma chain over ascending column with FP32 values, and
 * the row result is widened to FP64. */
static void spmv_rows_f32(int n, const int *rp, const int *ci, const float *v, const double *x,
                          double *y, float *x32) {
#pragma omp parallel for schedule(static, 4096)
  for (int i = 0; i < n; i++) x32[i] = (float)x[i];
#pragma omp parallel for schedule(static, 4096)
  for (int i = 0; i < n; i++) {
    float acc = 0.0f;
    for (int q = rp[i]; q < rp[i + 1]; q++) acc = fmaf(v[q], x32[ci[q]], acc);
    y[i] = (double)acc;
  }
}

static double vdot(int n, const double *x, const double *y, double *tmp) {
#pragma omp parallel for schedule(static, 4096)
  for (int i = 0; i < n; i++) tmp[i] = x[i] * y[i];
  return pairwise64(tmp, n);
}

/* Rows of M (CSC input) as CSR with column-sorted rows, or (sym != 0) the
 * rows of its symmetric part S = (M + M^T)/2, s_ij = 0.5 (m_ij + m_ji) in
 * FP64 with exact zeros dropped (the paper symmetrises M, Appendix A step 1). */
static void build_rows(int n, const int *mcolptr, const int *mrowind, const double *mvals, int sym,
                       int **rp_out, int **ci_out, double **v_out) {
  int nnz = mcolptr[n];
  int *mrp = (int *)calloc((size_t)n + 1, sizeof(int));
  int *mci = (int *)malloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
  double *mv = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  for (int e = 0; e < nnz; e++) mrp[mrowind[e] + 1]++;
  for (int i = 0; i < n; i++) mrp[i + 1] += mrp[i];
  int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; i++) fill[i] = mrp[i];
  for (int j = 0; j < n; j++)
    for (int e = mcolptr[j]; e < mcolptr[j + 1]; e++) {
      int i = mrowind[e];
      mci[fill[i]] = j;
      mv[fill[i]] = mvals[e];
      fill[i]++;
    }
  free(fill);
  if (sym) {
    int *srp = (int *)calloc((size_t)n + 1, sizeof(int));
    int *sci = (int *)malloc(sizeof(int) * (size_t)(2 * nnz + 1));
    double *sv = (double *)malloc(sizeof(double) * (size_t)(2 * nnz + 1));
    int t = 0;
    for (int i = 0; i < n; i++) { /* row i of M is CSR row i; row i of M^T is CSC column i */
      int a = mrp[i], ae = mrp[i + 1], b2 = mcolptr[i], be = mcolptr[i + 1];
      while (a < ae || b2 < be) {
        int c;
        double u = 0.0, w = 0.0;
        if (b2 >= be || (a < ae && mci[a] < mrowind[b2])) { c = mci[a]; u = mv[a++]; }
        else if (a >= ae || mrowind[b2] < mci[a]) { c = mrowind[b2]; w = mvals[b2++]; }
        else { c = mci[a]; u = mv[a++]; w = mvals[b2++]; }
        double val = 0.5 * (u + w);
        if (val != 0.0) { sci[t] = c; sv[t] = val; t++; }
      }
      srp[i + 1] = t;
    }
    free(mrp); free(mci); free(mv);
    mrp = srp; mci = sci; mv = sv;
  }
  *rp_out = mrp;
  *ci_out = mci;
  *v_out = mv;
}

/*
 * Vector PCG on A x = b, x_0 = 0, preconditioner z = Prec(r):
 *   precond 0: z = r; 1: z = r / diag(A); 2: z = M r with M given in CSC;
 *   3: z = S r with S = (M + M^T)/2, the symmetric part of M (PCG needs a
 *   symmetric preconditioner; the paper symmetrises M, Appendix A step 1).
 * Stops when ||r||_2 <= rtol ||b||_2 (recurrence residual), after maxit
 * iterations, or on breakdown ((p,Ap) or (r,z) zero or non-finite).
 * Returns iterations (= number of A p products); *status: 0 converged,
 * 1 maxit, 2 breakdown.  *relres = ||b - A x||_2 / ||b||_2 (true residual).
 * mixed != 0: the products with A and with M (or S) use FP32 values and an
 * FP32 copy of the operand (spmv_rows_f32); vectors, inner products and the
 * scalars stay FP64, and so does the final true residual.
 */
int orc_pcg(int n, const int *rp, const int *ci, const double *av, int precond, const int *mcolptr,
            const int *mrowind, const double *mvals, const double *b, double rtol, int maxit, double *x,
            int *status, double *relres, int mixed) {
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  double *z = (double *)malloc(sizeof(double) * (size_t)n);
  double *p = (double *)malloc(sizeof(double) * (size_t)n);
  double *q = (double *)malloc(sizeof(double) * (size_t)n);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 64 ? n : 64));
  double *diag = (double *)malloc(sizeof(double) * (size_t)n);
  int *mrp = NULL, *mci = NULL;
  double *mv = NULL;
  for (int i = 0; i < n; i++) {
    diag[i] = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; e++)
      if (ci[e] == i) diag[i] = av[e];
  }
  if (precond == 2 || precond == 3) build_rows(n, mcolptr, mrowind, mvals, precond == 3, &mrp, &mci, &mv);
  float *av32 = NULL, *mv32 = NULL, *x32 = NULL;
  if (mixed) {
    int nnz = rp[n];
    av32 = (float *)malloc(sizeof(float) * (size_t)(nnz ? nnz : 1));
    for (int e = 0; e < nnz; e++) av32[e] = (float)av[e];
    x32 = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (mrp) {
      int mnz = mrp[n];
      mv32 = (float *)malloc(sizeof(float) * (size_t)(mnz ? mnz : 1));
      for (int e = 0; e < mnz; e++) mv32[e] = (float)mv[e];
    }
  }
  for (int i = 0; i < n; i++) {
    x[i] = 0.0;
    r[i] = b[i];
  }
  double bn = sqrt(vdot(n, b, b, tmp));
  int k = 0;
  *status = 0;
#define PREC()                                                     \
  do {                                                             \
    if (precond == 0) for (int i_ = 0; i_ < n; i_++) z[i_] = r[i_]; \
    else if (precond == 1) for (int i_ = 0; i_ < n; i_++) z[i_] = r[i_] / diag[i_]; \
    else if (mixed) spmv_rows_f32(n, mrp, mci, mv32, r, z, x32);   \
    else spmv_rows(n, mrp, mci, mv, r, z, tmp);                    \
  } while (0)
  if (bn == 0.0) goto out;
  PREC();
  double rho = vdot(n, r, z, tmp);
  if (rho == 0.0 || !isfin(rho)) { *status = 2; goto out; }
  for (int i = 0; i < n; i++) p[i] = z[i];
  for (;;) {
    if (k >= maxit) { *status = 1; break; }
    if (mixed) spmv_rows_f32(n, rp, ci, av32, p, q, x32);
    else spmv_rows(n, rp, ci, av, p, q, tmp);
    double pq = vdot(n, p, q, tmp);
    if (pq == 0.0 || !isfin(pq)) { *status = 2; break; }
    double alpha = rho / pq;
#pragma omp parallel for schedule(static, 4096)
    for (int i = 0; i < n; i++) {
      x[i] = fma(alpha, p[i], x[i]);
      r[i] = fma(-alpha, q[i], r[i]);
    }
    k++;
    double rn = sqrt(vdot(n, r, r, tmp));
    if (!isfin(rn)) { *status = 2; break; }
    if (rn <= rtol * bn) { *status = 0; break; }
    PREC();
    double rho1 = vdot(n, r, z, tmp);
    if (rho1 == 0.0 || !isfin(rho1)) { *status = 2; break; }
    double beta = rho1 / rho;
#pragma omp parallel for schedule(static, 4096)
    for (int i = 0; i < n; i++) p[i] = fma(beta, p[i], z[i]);
    rho = rho1;
  }
out:
  if (relres) {
    spmv_rows(n, rp, ci, av, x, q, tmp);
    for (int i = 0; i < n; i++) q[i] = b[i] - q[i];
    *relres = bn > 0 ? sqrt(vdot(n, q, q, tmp)) / bn : 0.0;
  }
#undef PREC
  free(r);
  free(z);
  free(p);
  free(q);
  free(tmp);
  free(diag);
  free(mrp);
  free(mci);
  free(mv);
  free(av32);
  free(mv32);
  free(x32);
  return k;
}

/*
 * Lanczos on the symmetric part S = (M + M^T)/2 of M (definiteness
 * diagnostics: the extremal eigenvalues of the tridiagonal T approach
 * lambda_min(S) and lambda_max(S)), plain three-term recurrence without
 * reorthogonalisation, FP64:
 *   v_1 = v0 / ||v0||, v_0 = 0, beta_0 = 0; for j = 1..m:
 *   w = S v_j (fma chain per row, ascending column); alpha_j = (w, v_j);
 *   w = fma(-beta_{j-1}, v_{j-1}, fma(-alpha_j, v_j, w)); beta_j = ||w||;
 *   stop if beta_j is 0 or not finite; v_{j+1} = w / beta_j.
 * Inner products and norms are the pairwise trees of the PCG.  Writes
 * alpha[0..k), beta[0..k) and returns k, the steps done.
 */
int orc_lanczos(int n, const int *mcolptr, const int *mrowind, const double *mvals, const double *v0,
                int steps, double *alpha, double *beta) {
  int *srp, *sci;
  double *sv;
  build_rows(n, mcolptr, mrowind, mvals, 1, &srp, &sci, &sv);
  size_t nn = (size_t)(n > 0 ? n : 1);
  double *vp = (double *)calloc(nn, sizeof(double));
  double *vc = (double *)malloc(sizeof(double) * nn);
  double *w = (double *)malloc(sizeof(double) * nn);
  double *tmp = (double *)malloc(sizeof(double) * (nn > 64 ? nn : 64));
  double nrm = sqrt(vdot(n, v0, v0, tmp));
  for (int i = 0; i < n; i++) vc[i] = v0[i] / nrm;
  int k = 0;
  double bprev = 0.0;
  for (int j = 0; j < steps; j++) {
    spmv_rows(n, srp, sci, sv, vc, w, tmp);
    double a = vdot(n, w, vc, tmp);
    for (int i = 0; i < n; i++) w[i] = fma(-bprev, vp[i], fma(-a, vc[i], w[i]));
    double b = sqrt(vdot(n, w, w, tmp));
    alpha[j] = a;
    beta[j] = b;
    k = j + 1;
    if (b == 0.0 || !isfin(b)) break;
    for (int i = 0; i < n; i++) {
      vp[i] = vc[i];
      vc[i] = w[i] / b;
    }
    bprev = b;
  }
  free(srp); free(sci); free(sv);
  free(vp); free(vc); free(w); free(tmp);
  return k;
}
