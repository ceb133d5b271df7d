/*
 * CPU oracle for the scaled-ILU Richardson smoother.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, single-threaded FP64
 * statement of what the smoother computes, written step by step from
 * Thomas, Carr, Mullowney, Swirydowicz and Day, "Scaled ILU Smoothers for
 * Navier-Stokes Pressure Projection" (arXiv 2111.09512).  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.  It shares no code
 * with the CUDA library and must be compiled with -ffp-contract=off so that
 * every multiply and add rounds separately, in the order written here.
 *
 * Conventions.  CSR with int64 row pointers, int32 column indices sorted
 * ascending within each row, FP64 values.  Vectors with R right-hand sides
 * are row-major n x R (the R values of one row are adjacent).
 *
 * Factors.  L is unit lower triangular, L = I + L_s; only L_s is stored.  U is
 * upper triangular with its diagonal stored first in each row.  After row
 * scaling (Eq. extractD, Eq. newD) Utilde = D^{-1} U = I + Utilde_s; only
 * Utilde_s and dinv = 1 / diag(U) are stored.
 *
 * Beyond the smoother itself: the polynomial Gauss-Seidel smoother of
 * Sec. 3.1, row/column (Ruiz) scaling (Eq. rowcolScale), power-iteration
 * estimates of ||T_s^p||_2 (Fig. Up), and algebraic multigrid (Sec. 3,
 * Alg. mgcycle) with the ILU smoother on the finest level.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.  Unpinned
 * parts: none of the functions here is left without a pin, but the ILUT drop
 * rule (Saad's dual threshold, which the paper uses without defining it) is
 * pinned only through its limiting cases and stated invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_BADARG 1
#define ORC_ZERO_PIVOT 2
#define ORC_NOT_CONVERGED 3
#define ORC_NOMEM 4

typedef struct orc_lu {
  int64_t n;
  int64_t* lp; /* strict lower part of L, n+1 row pointers */
  int32_t* lc;
  double* lv;
  int64_t* up; /* U with its diagonal first in each row */
  int32_t* uc;
  double* uv;
} orc_lu;

/* ------------------------------------------------------------------------ */
/* small helpers: growable arrays and a binary min-heap of column indices    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t* c;
  double* v;
  int64_t len, cap;
} rowbuf;

static int rb_push(rowbuf* b, int32_t c, double v) {
  if (b->len == b->cap) {
    int64_t cap = b->cap ? 2 * b->cap : 1024;
    int32_t* nc = (int32_t*)realloc(b->c, sizeof(int32_t) * (size_t)cap);
    if (!nc) return 0;
    b->c = nc;
    double* nv = (double*)realloc(b->v, sizeof(double) * (size_t)cap);
    if (!nv) return 0;
    b->v = nv;
    b->cap = cap;
  }
  b->c[b->len] = c;
  b->v[b->len] = v;
  b->len++;
  return 1;
}

typedef struct {
  int32_t* h;
  int64_t len;
} minheap;

static void heap_push(minheap* q, int32_t x) {
  int64_t i = q->len++;
  q->h[i] = x;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (q->h[p] <= q->h[i]) break;
    int32_t t = q->h[p];
    q->h[p] = q->h[i];
    q->h[i] = t;
    i = p;
  }
}

static int32_t heap_pop(minheap* q) {
  int32_t top = q->h[0];
  q->h[0] = q->h[--q->len];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < q->len && q->h[l] < q->h[m]) m = l;
    if (r < q->len && q->h[r] < q->h[m]) m = r;
    if (m == i) break;
    int32_t t = q->h[m];
    q->h[m] = q->h[i];
    q->h[i] = t;
    i = m;
  }
  return top;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static orc_lu* lu_from_rows(int64_t n, rowbuf* L, rowbuf* U, const int64_t* lrow, const int64_t* urow) {
  orc_lu* f = (orc_lu*)calloc(1, sizeof(orc_lu));
  if (!f) return NULL;
  f->n = n;
  f->lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  f->up = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!f->lp || !f->up) {
    free(f->lp);
    free(f->up);
    free(f);
    return NULL;
  }
  memcpy(f->lp, lrow, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(f->up, urow, sizeof(int64_t) * (size_t)(n + 1));
  f->lc = L->c;
  f->lv = L->v;
  f->uc = U->c;
  f->uv = U->v;
  /* keep non-NULL pointers for empty factors */
  if (!f->lc) f->lc = (int32_t*)malloc(sizeof(int32_t));
  if (!f->lv) f->lv = (double*)malloc(sizeof(double));
  if (!f->uc) f->uc = (int32_t*)malloc(sizeof(int32_t));
  if (!f->uv) f->uv = (double*)malloc(sizeof(double));
  return f;
}

void orc_lu_free(orc_lu* f) {
  if (!f) return;
  free(f->lp);
  free(f->lc);
  free(f->lv);
  free(f->up);
  free(f->uc);
  free(f->uv);
  free(f);
}

void orc_lu_nnz(const orc_lu* f, int64_t* nl, int64_t* nu) {
  *nl = f->lp[f->n];
  *nu = f->up[f->n];
}

void orc_lu_copy(const orc_lu* f, int64_t* lp, int32_t* lc, double* lv, int64_t* up, int32_t* uc, double* uv) {
  const int64_t n = f->n;
  memcpy(lp, f->lp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(up, f->up, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(lc, f->lc, sizeof(int32_t) * (size_t)f->lp[n]);
  memcpy(lv, f->lv, sizeof(double) * (size_t)f->lp[n]);
  memcpy(uc, f->uc, sizeof(int32_t) * (size_t)f->up[n]);
  memcpy(uv, f->uv, sizeof(double) * (size_t)f->up[n]);
}

/* CSR sanity: monotone row pointers, in-range strictly ascending columns */
static int csr_ok(int64_t n, const int64_t* rp, const int32_t* ci) {
  if (n < 0 || !rp || rp[0] != 0) return 0;
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) return 0;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return 0;
    }
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* ILU on a fixed pattern (the numeric phase of ILU(0) and ILU(k))           */
/* ------------------------------------------------------------------------ */

/*
 * Numeric incomplete LU on the pattern P (row pointer pp, columns pc, which
 * contains the pattern of A).  IKJ elimination over row i, Saad, "Iterative
 * Methods for Sparse Linear Systems", the variant the paper names for ILU(0)
 * (Matlab ilu with setup type 'nofill', Sec. 5.1; pivoting off, Sec. 4.2):
 *   for k < i in P(i), ascending:  a_ik <- a_ik / a_kk
 *                                  a_ij <- a_ij - a_ik * a_kj  for j > k, j in P(i) and P(k)
 */
static orc_lu* ilu_on_pattern(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, const int64_t* pp,
                              const int32_t* pc, int* status) {
  double* w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  char* inrow = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t* lrow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* urow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* udiag = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  rowbuf L = {0}, U = {0};
  *status = ORC_NOMEM;
  if (!w || !inrow || !lrow || !urow || !udiag) goto fail;
  lrow[0] = urow[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = pp[i]; p < pp[i + 1]; ++p) {
      inrow[pc[p]] = 1;
      w[pc[p]] = 0.0;
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) w[ci[p]] = va[p];
    for (int64_t p = pp[i]; p < pp[i + 1] && pc[p] < i; ++p) {
      const int32_t k = pc[p];
      const double ukk = U.v[udiag[k]];
      w[k] = w[k] / ukk;
      for (int64_t q = udiag[k] + 1; q < urow[k + 1]; ++q) {
        const int32_t j = U.c[q];
        if (inrow[j]) w[j] = w[j] - w[k] * U.v[q];
      }
    }
    /* gather L (strict lower) and U (diagonal first) */
    int has_diag = 0;
    for (int64_t p = pp[i]; p < pp[i + 1]; ++p) {
      const int32_t j = pc[p];
      if (j < i) {
        if (!rb_push(&L, j, w[j])) goto fail;
      } else {
        if (j == i) has_diag = 1;
        if (!rb_push(&U, j, w[j])) goto fail;
      }
      inrow[j] = 0;
    }
    if (!has_diag || w[i] == 0.0 || !isfinite(w[i])) {
      *status = ORC_ZERO_PIVOT;
      goto fail_nomsg;
    }
    lrow[i + 1] = L.len;
    urow[i + 1] = U.len;
    udiag[i] = urow[i];
  }
  {
    orc_lu* f = lu_from_rows(n, &L, &U, lrow, urow);
    free(w);
    free(inrow);
    free(lrow);
    free(urow);
    free(udiag);
    if (!f) {
      free(L.c);
      free(L.v);
      free(U.c);
      free(U.v);
      *status = ORC_NOMEM;
      return NULL;
    }
    *status = ORC_OK;
    return f;
  }
fail:
  *status = ORC_NOMEM;
fail_nomsg:
  free(w);
  free(inrow);
  free(lrow);
  free(urow);
  free(udiag);
  free(L.c);
  free(L.v);
  free(U.c);
  free(U.v);
  return NULL;
}

/* ILU(0): the pattern of the factors is the pattern of A (Sec. 5.1, Table dep). */
orc_lu* orc_ilu0(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, int* status) {
  if (!csr_ok(n, rp, ci) || !va) {
    *status = ORC_BADARG;
    return NULL;
  }
  return ilu_on_pattern(n, rp, ci, va, rp, ci, status);
}

/*
 * Symbolic phase of ILU(k) (Sec. 1 names ILU(k); Saad's level-of-fill):
 * lev(i,j) = 0 on the pattern of A; eliminating with pivot row k gives
 * lev(i,j) = min(lev(i,j), lev(i,k) + lev(k,j) + 1); entries with
 * lev <= k_fill are kept.  Returns the pattern (sorted) in *pp, *pc.
 */
int orc_iluk_symbolic(int64_t n, const int64_t* rp, const int32_t* ci, int kfill, int64_t** pp_out, int32_t** pc_out,
                      int32_t** plev_out) {
  if (!csr_ok(n, rp, ci) || kfill < 0) return ORC_BADARG;
  int32_t* lev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  minheap q = {(int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)), 0};
  int64_t* pp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* udiag = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  rowbuf P = {0};   /* columns in c, levels stored as doubles in v */
  if (!lev || !cols || !q.h || !pp || !udiag) goto fail;
  for (int64_t j = 0; j < n; ++j) lev[j] = -1;
  pp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ncols = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      lev[ci[p]] = 0;
      cols[ncols++] = ci[p];
      if (ci[p] < i) heap_push(&q, ci[p]);
    }
    while (q.len > 0) {
      const int32_t k = heap_pop(&q);
      const int32_t lik = lev[k];
      /* row k of U: pattern entries of row k with column > k */
      for (int64_t p = udiag[k] + 1; p < pp[k + 1]; ++p) {
        const int32_t j = P.c[p];
        const int32_t nl = lik + (int32_t)P.v[p] + 1;
        if (nl > kfill) continue;
        if (lev[j] < 0) {
          lev[j] = nl;
          cols[ncols++] = j;
          if (j < i) heap_push(&q, j);
        } else if (nl < lev[j]) {
          lev[j] = nl;
        }
      }
    }
    qsort(cols, (size_t)ncols, sizeof(int32_t), cmp_i32);
    int64_t dpos = -1;
    for (int64_t t = 0; t < ncols; ++t) {
      if (cols[t] == i) dpos = P.len;
      if (!rb_push(&P, cols[t], (double)lev[cols[t]])) goto fail;
      lev[cols[t]] = -1;
    }
    if (dpos < 0) {
      /* no diagonal in the pattern: the pivot is structurally zero */
      free(lev);
      free(cols);
      free(q.h);
      free(pp);
      free(udiag);
      free(P.c);
      free(P.v);
      return ORC_ZERO_PIVOT;
    }
    udiag[i] = dpos;
    pp[i + 1] = P.len;
  }
  {
    int64_t nnz = P.len;
    int32_t* plev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!plev) goto fail;
    for (int64_t p = 0; p < nnz; ++p) plev[p] = (int32_t)P.v[p];
    free(P.v);
    *pp_out = pp;
    *pc_out = P.c ? P.c : (int32_t*)malloc(sizeof(int32_t));
    if (plev_out)
      *plev_out = plev;
    else
      free(plev);
    free(lev);
    free(cols);
    free(q.h);
    free(udiag);
    return ORC_OK;
  }
fail:
  free(lev);
  free(cols);
  free(q.h);
  free(pp);
  free(udiag);
  free(P.c);
  free(P.v);
  return ORC_NOMEM;
}

/* ILU(k): symbolic level-of-fill pattern, then the numeric phase on it */
orc_lu* orc_iluk(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, int kfill, int* status) {
  int64_t* pp = NULL;
  int32_t* pc = NULL;
  if (!va) {
    *status = ORC_BADARG;
    return NULL;
  }
  int st = orc_iluk_symbolic(n, rp, ci, kfill, &pp, &pc, NULL);
  if (st != ORC_OK) {
    *status = st;
    return NULL;
  }
  orc_lu* f = ilu_on_pattern(n, rp, ci, va, pp, pc, status);
  free(pp);
  free(pc);
  return f;
}

/* pattern of ILU(k) for the tests: caller frees with orc_free */
int orc_iluk_pattern(int64_t n, const int64_t* rp, const int32_t* ci, int kfill, int64_t* nnz_out, int64_t** pp,
                     int32_t** pc, int32_t** plev) {
  int st = orc_iluk_symbolic(n, rp, ci, kfill, pp, pc, plev);
  if (st == ORC_OK) *nnz_out = (*pp)[n];
  return st;
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* ILUT(tau, p), Saad's dual threshold, pivoting off                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t c;
  double a;
} cand;

/* larger magnitude first; equal magnitudes: smaller column first */
static int cmp_cand(const void* x, const void* y) {
  const cand* u = (const cand*)x;
  const cand* v = (const cand*)y;
  if (u->a > v->a) return -1;
  if (u->a < v->a) return 1;
  return (u->c > v->c) - (u->c < v->c);
}

static int cmp_cand_col(const void* x, const void* y) {
  const cand* u = (const cand*)x;
  const cand* v = (const cand*)y;
  return (u->c > v->c) - (u->c < v->c);
}

/*
 * The paper uses ILUT with a drop tolerance and a fill limit per row
 * (droptol, lfill; Sec. 4.2, Sec. 6.1) without defining the rule.  Reading:
 * Saad's ILUT(tau, p) with pivoting off.  For row i:
 *   tau_i = tau * ||a_{i,:}||_2
 *   w = a_{i,:}
 *   for k < i with w_k != 0, ascending:
 *       w_k <- w_k / u_kk
 *       if |w_k| < tau_i: w_k <- 0 (dropped, no update)
 *       else w_j <- w_j - w_k * u_kj for j > k in row k of U
 *   drop off-diagonal entries with |w_j| < tau_i
 *   keep the p largest-magnitude entries of the L part and, separately, of
 *   the U part (ties: smaller column); the diagonal is always kept.
 * A zero or non-finite pivot is an error (no pivot boosting).
 */
orc_lu* orc_ilut(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, double tau, int pfill,
                 int* status) {
  if (!csr_ok(n, rp, ci) || !va || !(tau >= 0.0) || pfill < 0) {
    *status = ORC_BADARG;
    return NULL;
  }
  const size_t nn = (size_t)(n > 0 ? n : 1);
  double* w = (double*)calloc(nn, sizeof(double));
  char* inrow = (char*)calloc(nn, 1);
  int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * nn);
  cand* cl = (cand*)malloc(sizeof(cand) * nn);
  cand* cu = (cand*)malloc(sizeof(cand) * nn);
  minheap q = {(int32_t*)malloc(sizeof(int32_t) * nn), 0};
  int64_t* lrow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* urow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  rowbuf L = {0}, U = {0};
  *status = ORC_NOMEM;
  if (!w || !inrow || !cols || !cl || !cu || !q.h || !lrow || !urow) goto fail;
  lrow[0] = urow[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    double nrm2 = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) nrm2 = nrm2 + va[p] * va[p];
    const double tau_i = tau * sqrt(nrm2);
    int64_t ncols = 0, nl = 0, nu = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t j = ci[p];
      w[j] = va[p];
      inrow[j] = 1;
      cols[ncols++] = j;
      if (j < i) heap_push(&q, j);
    }
    while (q.len > 0) {
      const int32_t k = heap_pop(&q);
      w[k] = w[k] / U.v[urow[k]];
      if (fabs(w[k]) < tau_i) {
        w[k] = 0.0;
        continue;
      }
      cl[nl].c = k;
      cl[nl].a = fabs(w[k]);
      nl++;
      for (int64_t qq = urow[k] + 1; qq < urow[k + 1]; ++qq) {
        const int32_t j = U.c[qq];
        if (!inrow[j]) {
          inrow[j] = 1;
          w[j] = 0.0;
          cols[ncols++] = j;
          if (j < i) heap_push(&q, j);
        }
        w[j] = w[j] - w[k] * U.v[qq];
      }
    }
    const double piv = inrow[i] ? w[i] : 0.0;
    if (piv == 0.0 || !isfinite(piv)) {
      *status = ORC_ZERO_PIVOT;
      goto fail_nomsg;
    }
    for (int64_t t = 0; t < ncols; ++t) {
      const int32_t j = cols[t];
      if (j > i && fabs(w[j]) >= tau_i) {
        cu[nu].c = j;
        cu[nu].a = fabs(w[j]);
        nu++;
      }
    }
    qsort(cl, (size_t)nl, sizeof(cand), cmp_cand);
    qsort(cu, (size_t)nu, sizeof(cand), cmp_cand);
    if (nl > pfill) nl = pfill;
    if (nu > pfill) nu = pfill;
    qsort(cl, (size_t)nl, sizeof(cand), cmp_cand_col);
    qsort(cu, (size_t)nu, sizeof(cand), cmp_cand_col);
    for (int64_t t = 0; t < nl; ++t)
      if (!rb_push(&L, cl[t].c, w[cl[t].c])) goto fail;
    if (!rb_push(&U, (int32_t)i, piv)) goto fail;
    for (int64_t t = 0; t < nu; ++t)
      if (!rb_push(&U, cu[t].c, w[cu[t].c])) goto fail;
    for (int64_t t = 0; t < ncols; ++t) {
      inrow[cols[t]] = 0;
      w[cols[t]] = 0.0;
    }
    lrow[i + 1] = L.len;
    urow[i + 1] = U.len;
  }
  {
    orc_lu* f = lu_from_rows(n, &L, &U, lrow, urow);
    free(w);
    free(inrow);
    free(cols);
    free(cl);
    free(cu);
    free(q.h);
    free(lrow);
    free(urow);
    if (!f) {
      free(L.c);
      free(L.v);
      free(U.c);
      free(U.v);
      *status = ORC_NOMEM;
      return NULL;
    }
    *status = ORC_OK;
    return f;
  }
fail:
  *status = ORC_NOMEM;
fail_nomsg:
  free(w);
  free(inrow);
  free(cols);
  free(cl);
  free(cu);
  free(q.h);
  free(lrow);
  free(urow);
  free(L.c);
  free(L.v);
  free(U.c);
  free(U.v);
  return NULL;
}

/* ------------------------------------------------------------------------ */
/* Row scaling (Eq. extractD, Eq. newD)                                      */
/* ------------------------------------------------------------------------ */

/*
 * D = diag(U), Utilde = D^{-1} U, so Utilde_ij = u_ij / u_ii.  Writes
 * dinv_i = 1 / u_ii and the strict upper part Utilde_s (row pointer sp with
 * n+1 entries, nnz(U) - n entries).  diag(Utilde) = u_ii / u_ii = 1 exactly
 * for finite nonzero u_ii, so it is not stored.
 */
int orc_row_scale(int64_t n, const int64_t* up, const int32_t* uc, const double* uv, double* dinv, int64_t* sp,
                  int32_t* sc, double* sv) {
  int64_t q = 0;
  sp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (up[i + 1] <= up[i] || uc[up[i]] != i) return ORC_BADARG;
    const double d = uv[up[i]];
    if (d == 0.0 || !isfinite(d)) return ORC_ZERO_PIVOT;
    dinv[i] = 1.0 / d;
    for (int64_t p = up[i] + 1; p < up[i + 1]; ++p) {
      sc[q] = uc[p];
      sv[q] = uv[p] / d;
      ++q;
    }
    sp[i + 1] = q;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Residual, SpMV and the Richardson sweeps (Alg. ILUJac, Eq. richard)        */
/* ------------------------------------------------------------------------ */

/* y = A x  (sum over the row in ascending column order) */
void orc_spmv(int64_t n, int R, const int64_t* rp, const int32_t* ci, const double* va, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < R; ++r) {
      double s = 0.0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s = s + va[p] * x[(int64_t)ci[p] * R + r];
      y[i * R + r] = s;
    }
}

/* r = b - A x (Eq. ILUsplit, the residual of the splitting iteration) */
void orc_residual(int64_t n, int R, const int64_t* rp, const int32_t* ci, const double* va, const double* x,
                  const double* b, double* r) {
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < R; ++c) {
      double s = 0.0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s = s + va[p] * x[(int64_t)ci[p] * R + c];
      r[i * R + c] = b[i * R + c] - s;
    }
}

/* one sweep: out = c - T_s in */
static void sweep(int64_t n, int R, const int64_t* tp, const int32_t* tc, const double* tv, const double* c,
                  const double* in, double* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < R; ++k) {
      double s = 0.0;
      for (int64_t p = tp[i]; p < tp[i + 1]; ++p) s = s + tv[p] * in[(int64_t)tc[p] * R + k];
      out[i * R + k] = c[i * R + k] - s;
    }
}

/*
 * Richardson iteration for L y = r with L = I + L_s (Alg. ILUJac, first loop):
 *   y^0 = 0;  y^k = r - L_s y^{k-1},  k = 1..m.
 * Writes y^m.  m = 0 leaves y = 0.
 */
int orc_richardson_lower(int64_t n, int R, const int64_t* lp, const int32_t* lc, const double* lv, const double* r,
                         int m, double* y) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* prev = (double*)calloc(sz, sizeof(double));
  if (!prev) return ORC_NOMEM;
  memset(y, 0, sizeof(double) * (size_t)(n * R));
  for (int k = 1; k <= m; ++k) {
    memcpy(prev, y, sizeof(double) * (size_t)(n * R));
    sweep(n, R, lp, lc, lv, r, prev, y);
  }
  free(prev);
  return ORC_OK;
}

/*
 * Richardson iteration for Utilde v = D^{-1} y with Utilde = I + Utilde_s
 * (Alg. ILUJac, second loop; Eq. richard with b_s = D_U^{-1} b):
 *   c = dinv .* y;  v^0 = 0;  v^k = c - Utilde_s v^{k-1},  k = 1..m.
 */
int orc_richardson_upper(int64_t n, int R, const int64_t* sp, const int32_t* sc, const double* sv, const double* dinv,
                         const double* y, int m, double* v) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* c = (double*)malloc(sz * sizeof(double));
  double* prev = (double*)calloc(sz, sizeof(double));
  if (!c || !prev) {
    free(c);
    free(prev);
    return ORC_NOMEM;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < R; ++k) c[i * R + k] = dinv[i] * y[i * R + k];
  memset(v, 0, sizeof(double) * (size_t)(n * R));
  for (int k = 1; k <= m; ++k) {
    memcpy(prev, v, sizeof(double) * (size_t)(n * R));
    sweep(n, R, sp, sc, sv, c, prev, v);
  }
  free(c);
  free(prev);
  return ORC_OK;
}

/*
 * One smoother application (Eq. ILUsplit with M = L D Utilde, Alg. ILUJac):
 *   r = b - A x;  y = L^{-1} r by m_L sweeps;  v = Utilde^{-1} D^{-1} y by
 *   m_U sweeps;  x <- x + v.
 * A factor with zero sweeps is skipped (treated as the identity, with the
 * D^{-1} scaling dropped too when m_U = 0).
 */
int orc_smooth(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, const int64_t* lp,
               const int32_t* lc, const double* lv, const int64_t* sp, const int32_t* sc, const double* sv,
               const double* dinv, double* x, const double* b, int mL, int mU) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* r = (double*)malloc(sz * sizeof(double));
  double* y = (double*)malloc(sz * sizeof(double));
  double* v = (double*)malloc(sz * sizeof(double));
  int st = ORC_NOMEM;
  if (!r || !y || !v) goto done;
  orc_residual(n, R, ap, ac, av, x, b, r);
  if (mL > 0) {
    if ((st = orc_richardson_lower(n, R, lp, lc, lv, r, mL, y))) goto done;
  } else {
    memcpy(y, r, sizeof(double) * (size_t)(n * R));
  }
  if (mU > 0) {
    if ((st = orc_richardson_upper(n, R, sp, sc, sv, dinv, y, mU, v))) goto done;
  } else {
    memcpy(v, y, sizeof(double) * (size_t)(n * R));
  }
  for (int64_t t = 0; t < n * R; ++t) x[t] = x[t] + v[t];
  st = ORC_OK;
done:
  free(r);
  free(y);
  free(v);
  return st;
}

/*
 * Unscaled plain Richardson on U = D + U_s (diagonal stored first in each
 * row): v^k = y - (U - I) v^{k-1}.  Converges only if every |1 - u_ii| < 1
 * (Sec. 6.1: iterations on unscaled factors fail to converge unless
 * preconditioned).
 */
int orc_upper_unscaled_richardson(int64_t n, int R, const int64_t* up, const int32_t* uc, const double* uv,
                                  const double* y, int m, double* v) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* prev = (double*)calloc(sz, sizeof(double));
  if (!prev) return ORC_NOMEM;
  memset(v, 0, sizeof(double) * (size_t)(n * R));
  for (int k = 1; k <= m; ++k) {
    memcpy(prev, v, sizeof(double) * (size_t)(n * R));
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < R; ++c) {
        double s = 0.0;
        for (int64_t p = up[i]; p < up[i + 1]; ++p) {
          const double t = (uc[p] == i) ? uv[p] - 1.0 : uv[p];
          s = s + t * prev[(int64_t)uc[p] * R + c];
        }
        v[i * R + c] = y[i * R + c] - s;
      }
  }
  free(prev);
  return ORC_OK;
}

/*
 * Unscaled Jacobi on U (Eq. LUiterMat, G_U = I - D_U^{-1} U):
 *   v^k = v^{k-1} + D_U^{-1} (y - U v^{k-1}).
 * In exact arithmetic equal to the scaled Richardson iterates.
 */
int orc_upper_jacobi(int64_t n, int R, const int64_t* up, const int32_t* uc, const double* uv, const double* y, int m,
                     double* v) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* prev = (double*)calloc(sz, sizeof(double));
  if (!prev) return ORC_NOMEM;
  memset(v, 0, sizeof(double) * (size_t)(n * R));
  for (int k = 1; k <= m; ++k) {
    memcpy(prev, v, sizeof(double) * (size_t)(n * R));
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < R; ++c) {
        double s = 0.0;
        for (int64_t p = up[i]; p < up[i + 1]; ++p) s = s + uv[p] * prev[(int64_t)uc[p] * R + c];
        v[i * R + c] = prev[i * R + c] + (y[i * R + c] - s) / uv[up[i]];
      }
  }
  free(prev);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Direct triangular solves and level sets (Sec. 4, level-set scheduling)     */
/* ------------------------------------------------------------------------ */

/* forward substitution for (I + L_s) y = r */
void orc_forward_subst(int64_t n, int R, const int64_t* lp, const int32_t* lc, const double* lv, const double* r,
                       double* y) {
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < R; ++c) {
      double s = 0.0;
      for (int64_t p = lp[i]; p < lp[i + 1]; ++p) s = s + lv[p] * y[(int64_t)lc[p] * R + c];
      y[i * R + c] = r[i * R + c] - s;
    }
}

/* backward substitution for (I + Utilde_s) v = c */
void orc_backward_subst_unit(int64_t n, int R, const int64_t* sp, const int32_t* sc, const double* sv, const double* c,
                             double* v) {
  for (int64_t i = n - 1; i >= 0; --i)
    for (int k = 0; k < R; ++k) {
      double s = 0.0;
      for (int64_t p = sp[i]; p < sp[i + 1]; ++p) s = s + sv[p] * v[(int64_t)sc[p] * R + k];
      v[i * R + k] = c[i * R + k] - s;
    }
}

/*
 * Direct smoother application: x <- x + Utilde^{-1} D^{-1} L^{-1} (b - A x),
 * the exact solves that the sweeps approximate.
 */
int orc_direct_apply(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, const int64_t* lp,
                     const int32_t* lc, const double* lv, const int64_t* sp, const int32_t* sc, const double* sv,
                     const double* dinv, double* x, const double* b) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* r = (double*)malloc(sz * sizeof(double));
  double* y = (double*)malloc(sz * sizeof(double));
  double* v = (double*)malloc(sz * sizeof(double));
  if (!r || !y || !v) {
    free(r);
    free(y);
    free(v);
    return ORC_NOMEM;
  }
  orc_residual(n, R, ap, ac, av, x, b, r);
  orc_forward_subst(n, R, lp, lc, lv, r, y);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < R; ++k) y[i * R + k] = dinv[i] * y[i * R + k];
  orc_backward_subst_unit(n, R, sp, sc, sv, y, v);
  for (int64_t t = 0; t < n * R; ++t) x[t] = x[t] + v[t];
  free(r);
  free(y);
  free(v);
  return ORC_OK;
}

/*
 * Level sets of a strictly lower triangular pattern: lev(i) = 0 for a row
 * with no entries, else 1 + max lev(j) over its entries.  Returns the number
 * of levels (0 for n = 0).
 */
int64_t orc_levels_lower(int64_t n, const int64_t* lp, const int32_t* lc, int32_t* lev) {
  int64_t nlev = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int64_t p = lp[i]; p < lp[i + 1]; ++p)
      if (lev[lc[p]] + 1 > l) l = lev[lc[p]] + 1;
    lev[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  return nlev;
}

/* Level sets of a strictly upper triangular pattern, computed from the bottom. */
int64_t orc_levels_upper(int64_t n, const int64_t* sp, const int32_t* sc, int32_t* lev) {
  int64_t nlev = 0;
  for (int64_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int64_t p = sp[i]; p < sp[i + 1]; ++p)
      if (lev[sc[p]] + 1 > l) l = lev[sc[p]] + 1;
    lev[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  return nlev;
}

/* ------------------------------------------------------------------------ */
/* FGMRES(m) with modified Gram-Schmidt (Sec. 6: Eq. relres, FGMRES, MGS)     */
/* ------------------------------------------------------------------------ */

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

/*
 * Right-preconditioned flexible GMRES(m) for A x = b, one right-hand side.
 * x holds the initial guess on entry.  precond: 0 = the Richardson smoother
 * with (mL, mU) sweeps applied from a zero guess, 1 = direct triangular
 * solves, 2 = none.  Arnoldi by modified Gram-Schmidt, Givens rotations with
 * r = hypot(a, b).  Stops when the Arnoldi residual estimate falls to
 * tol * ||b||; then the true residual ||b - A x|| / ||b|| (Eq. relres) is
 * recomputed and the method restarts while it is above tol (the paper warns
 * of false convergence).  maxit bounds the total number of inner iterations.
 * Returns ORC_OK when the true relative residual is <= tol.
 */
int orc_fgmres(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, const int64_t* lp, const int32_t* lc,
               const double* lv, const int64_t* sp, const int32_t* sc, const double* sv, const double* dinv, double* x,
               const double* b, double tol, int m, int maxit, int mL, int mU, int precond, int* iters_out,
               double* relres_out) {
  if (n < 0 || m < 1 || maxit < 0 || precond < 0 || precond > 2) return ORC_BADARG;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  double* V = (double*)malloc(sizeof(double) * nn * (size_t)(m + 1));
  double* Z = (double*)malloc(sizeof(double) * nn * (size_t)m);
  double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* yv = (double*)malloc(sizeof(double) * (size_t)m);
  double* r = (double*)malloc(sizeof(double) * nn);
  double* w = (double*)malloc(sizeof(double) * nn);
  double* zero = (double*)calloc(nn, sizeof(double));
  int st = ORC_NOMEM;
  int its = 0;
  double relres = 0.0;
  if (!V || !Z || !H || !cs || !sn || !g || !yv || !r || !w || !zero) goto done;
  const double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    st = ORC_OK;
    goto done;
  }
#define HH(i, j) H[(size_t)(i) * (size_t)m + (size_t)(j)]
  for (;;) {
    orc_residual(n, 1, ap, ac, av, x, b, r);
    const double beta = sqrt(dot(n, r, r));
    relres = beta / bnorm;
    if (relres <= tol) {
      st = ORC_OK;
      break;
    }
    if (its >= maxit) {
      st = ORC_NOT_CONVERGED;
      break;
    }
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int t = 0; t <= m; ++t) g[t] = 0.0;
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * nn;
      double* zj = Z + (size_t)j * nn;
      /* z_j = M^{-1} v_j */
      if (precond == 0) {
        memset(zj, 0, sizeof(double) * nn);
        if ((st = orc_smooth(n, 1, ap, ac, av, lp, lc, lv, sp, sc, sv, dinv, zj, vj, mL, mU))) goto done;
      } else if (precond == 1) {
        memset(zj, 0, sizeof(double) * nn);
        if ((st = orc_direct_apply(n, 1, ap, ac, av, lp, lc, lv, sp, sc, sv, dinv, zj, vj))) goto done;
      } else {
        memcpy(zj, vj, sizeof(double) * nn);
      }
      orc_spmv(n, 1, ap, ac, av, zj, w);
      for (int i = 0; i <= j; ++i) {
        const double* vi = V + (size_t)i * nn;
        const double h = dot(n, w, vi);
        HH(i, j) = h;
        for (int64_t t = 0; t < n; ++t) w[t] = w[t] - h * vi[t];
      }
      const double hn = sqrt(dot(n, w, w));
      HH(j + 1, j) = hn;
      if (hn != 0.0) {
        double* vn = V + (size_t)(j + 1) * nn;
        for (int64_t t = 0; t < n; ++t) vn[t] = w[t] / hn;
      }
      for (int i = 0; i < j; ++i) {
        const double a = HH(i, j), bb = HH(i + 1, j);
        HH(i, j) = cs[i] * a + sn[i] * bb;
        HH(i + 1, j) = -sn[i] * a + cs[i] * bb;
      }
      const double a = HH(j, j), bb = HH(j + 1, j);
      const double den = hypot(a, bb);
      cs[j] = a / den;
      sn[j] = bb / den;
      HH(j, j) = den;
      HH(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      its++;
      jend = j + 1;
      if (fabs(g[j + 1]) <= tol * bnorm || its >= maxit || hn == 0.0) break;
    }
    /* solve the jend x jend upper triangular system and update x */
    for (int i = jend - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < jend; ++t) s = s - HH(i, t) * yv[t];
      yv[i] = s / HH(i, i);
    }
    for (int i = 0; i < jend; ++i) {
      const double* zi = Z + (size_t)i * nn;
      for (int64_t t = 0; t < n; ++t) x[t] = x[t] + yv[i] * zi[t];
    }
  }
#undef HH
done:
  if (iters_out) *iters_out = its;
  if (relres_out) *relres_out = relres;
  free(V);
  free(Z);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(yv);
  free(r);
  free(w);
  free(zero);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Eq. depB, Eq. diagDep, Eq. nbre)                              */
/* ------------------------------------------------------------------------ */

/*
 * Henrici's departure from normality dep(T) = sqrt(||T||_F^2 - ||Lambda||_F^2)
 * (Eq. depB) of a triangular T stored in CSR.  The eigenvalues of a
 * triangular matrix are its diagonal, so ||T||_F^2 - ||Lambda||_F^2 is the
 * sum of squares of the off-diagonal entries, which is what is summed (the
 * same quantity without the cancellation of the difference).  With
 * unit_diag != 0 the stored entries are the strict part of I + T_s and the
 * result is ||T_s||_F (Eq. diagDep).
 */
double orc_dep_triangular(int64_t n, const int64_t* tp, const int32_t* tc, const double* tv, int unit_diag) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = tp[i]; p < tp[i + 1]; ++p)
      if (unit_diag || tc[p] != i) s = s + tv[p] * tv[p];
  return sqrt(s);
}

/* ||A||_2 of a symmetric A estimated by `iters` power iterations from ones */
double orc_norm2_est(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, int iters) {
  if (n <= 0) return 0.0;
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double lam = 0.0;
  if (!v || !w) {
    free(v);
    free(w);
    return -1.0;
  }
  for (int64_t i = 0; i < n; ++i) v[i] = 1.0 / sqrt((double)n);
  for (int it = 0; it < iters; ++it) {
    orc_spmv(n, 1, ap, ac, av, v, w);
    lam = sqrt(dot(n, w, w));
    if (lam == 0.0) break;
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / lam;
  }
  free(v);
  free(w);
  return lam;
}

/* NRBE = ||b - A x|| / (||b|| + ||A||_2 ||x||)  (Eq. nbre) */
double orc_nrbe(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, double norm2A, const double* x,
                const double* b) {
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!r) return -1.0;
  orc_residual(n, 1, ap, ac, av, x, b, r);
  const double rn = sqrt(dot(n, r, r));
  const double out = rn / (sqrt(dot(n, b, b)) + norm2A * sqrt(dot(n, x, x)));
  free(r);
  return out;
}

/* ------------------------------------------------------------------------ */
/* Polynomial Gauss-Seidel (Sec. 3.1: the Gauss-Seidel splitting M = D + L   */
/* with (D + L)^{-1} written as (I + D^{-1} L)^{-1} D^{-1} and the inverse   */
/* replaced by a truncated Neumann series)                                   */
/* ------------------------------------------------------------------------ */

/*
 * z = sum_{j=0}^{p} (-D^{-1} T)^j s, where D = diag(A), T is the strictly
 * lower (upper = 0) or strictly upper (upper != 0) part of A, and
 * s = D^{-1} r (scale_first != 0) or s = r.  The terms are formed one after
 * another, t_0 = s and t_j = -D^{-1} (T t_{j-1}), and summed in order
 * j = 0..p.  p = -1 gives z = 0.  A zero or non-finite diagonal entry gives
 * ORC_ZERO_PIVOT.
 */
static int poly_gs_terms(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, const double* r,
                         int p, int upper, int scale_first, double* z) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* t = (double*)malloc(sz * sizeof(double));
  double* u = (double*)malloc(sz * sizeof(double));
  int st = ORC_NOMEM;
  if (!d || !t || !u) goto done;
  st = ORC_ZERO_PIVOT;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int64_t q = ap[i]; q < ap[i + 1]; ++q)
      if (ac[q] == i) d[i] = d[i] + av[q];
    if (d[i] == 0.0 || !isfinite(d[i])) goto done;
  }
  memset(z, 0, sizeof(double) * (size_t)(n * R));
  if (p >= 0) {
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < R; ++k) t[i * R + k] = scale_first ? r[i * R + k] / d[i] : r[i * R + k];
    for (int64_t e = 0; e < n * R; ++e) z[e] = z[e] + t[e];
  }
  for (int j = 1; j <= p; ++j) {
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < R; ++k) {
        double s = 0.0;
        for (int64_t q = ap[i]; q < ap[i + 1]; ++q) {
          const int in_part = upper ? (ac[q] > i) : (ac[q] < i);
          if (in_part) s = s + av[q] * t[(int64_t)ac[q] * R + k];
        }
        u[i * R + k] = -(s / d[i]);
      }
    memcpy(t, u, sizeof(double) * (size_t)(n * R));
    for (int64_t e = 0; e < n * R; ++e) z[e] = z[e] + t[e];
  }
  st = ORC_OK;
done:
  free(d);
  free(t);
  free(u);
  return st;
}

/* z = sum_{j=0}^{p} (-D^{-1} L)^j D^{-1} r: the forward Gauss-Seidel solve
 * (D + L) z = r with its inverse truncated after p + 1 Neumann terms. */
int orc_poly_gs_lower(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, const double* r,
                      int p, double* z) {
  return poly_gs_terms(n, R, ap, ac, av, r, p, 0, 1, z);
}

/* w = sum_{j=0}^{q} (-D^{-1} U)^j z: (I + D^{-1} U)^{-1} z truncated after q + 1
 * terms, the backward half of symmetric Gauss-Seidel, whose splitting matrix
 * is (D + L) D^{-1} (D + U), so that M^{-1} r = (I + D^{-1} U)^{-1} (D + L)^{-1} r. */
int orc_poly_gs_upper_unit(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av,
                           const double* z, int q, double* w) {
  return poly_gs_terms(n, R, ap, ac, av, z, q, 1, 0, w);
}

/*
 * One polynomial Gauss-Seidel smoothing step (Eq. ILUsplit with M = D + L,
 * or M = (D + L) D^{-1} (D + U) when symmetric != 0):
 *   r = b - A x;  z = sum_{j<=pL} (-D^{-1} L)^j D^{-1} r;
 *   symmetric: w = sum_{j<=pU} (-D^{-1} U)^j z, else w = z;  x <- x + w.
 */
int orc_poly_gs_smooth(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, double* x,
                       const double* b, int pL, int pU, int symmetric) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* r = (double*)malloc(sz * sizeof(double));
  double* z = (double*)malloc(sz * sizeof(double));
  double* w = (double*)malloc(sz * sizeof(double));
  int st = ORC_NOMEM;
  if (!r || !z || !w) goto done;
  orc_residual(n, R, ap, ac, av, x, b, r);
  if ((st = orc_poly_gs_lower(n, R, ap, ac, av, r, pL, z))) goto done;
  if (symmetric) {
    if ((st = orc_poly_gs_upper_unit(n, R, ap, ac, av, z, pU, w))) goto done;
  } else {
    memcpy(w, z, sizeof(double) * (size_t)(n * R));
  }
  for (int64_t e = 0; e < n * R; ++e) x[e] = x[e] + w[e];
  st = ORC_OK;
done:
  free(r);
  free(z);
  free(w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Row/column scaling of U (Sec. 5.1, Eq. rowcolScale: Richardson on the     */
/* unit-diagonal D_r U D_c)                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Ruiz equilibration of U (diagonal first in each row), then the unit
 * diagonal.  Step k: with B = diag(rs) U diag(cs) (rs = cs = 1 at the start),
 * every row i is divided by sqrt(max_j |b_ij|) and every column j by
 * sqrt(max_i |b_ij|), both maxima taken on the same B; stop after `maxit`
 * steps or when every row and column maximum of B lies within `tol` of 1.
 * The column scaling is then dc = cs, and the row scaling is the one that
 * makes the diagonal of D_r U D_c exactly one: dr_i = 1 / (u_ii dc_i).
 * Writes dr, dc and Uhat_s = strict part of D_r U D_c (n+1 row pointers,
 * nnz(U) - n entries): uhat_ij = (dr_i u_ij) dc_j.  Returns the number of
 * Ruiz steps taken, or -ORC_ZERO_PIVOT / -ORC_NOMEM.
 */
int orc_ruiz_rowcol(int64_t n, const int64_t* up, const int32_t* uc, const double* uv, int maxit, double tol,
                    double* dr, double* dc, int64_t* sp, int32_t* sc, double* sv) {
  double* rs = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* rmax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* cmax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int steps = 0;
  if (!rs || !rmax || !cmax) {
    steps = -ORC_NOMEM;
    goto done;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (up[i + 1] <= up[i] || uc[up[i]] != i || uv[up[i]] == 0.0 || !isfinite(uv[up[i]])) {
      steps = -ORC_ZERO_PIVOT;
      goto done;
    }
    rs[i] = 1.0;
    dc[i] = 1.0;
  }
  for (;;) {
    for (int64_t i = 0; i < n; ++i) {
      rmax[i] = 0.0;
      cmax[i] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = up[i]; p < up[i + 1]; ++p) {
        const double b = fabs(rs[i] * uv[p] * dc[uc[p]]);
        if (b > rmax[i]) rmax[i] = b;
        if (b > cmax[uc[p]]) cmax[uc[p]] = b;
      }
    int equilibrated = 1;
    for (int64_t i = 0; i < n; ++i)
      if (fabs(1.0 - rmax[i]) > tol || fabs(1.0 - cmax[i]) > tol) equilibrated = 0;
    if (equilibrated || steps >= maxit) break;
    for (int64_t i = 0; i < n; ++i) {
      rs[i] = rs[i] / sqrt(rmax[i]);
      dc[i] = dc[i] / sqrt(cmax[i]);
    }
    ++steps;
  }
  sp[0] = 0;
  for (int64_t i = 0, q = 0; i < n; ++i) {
    dr[i] = 1.0 / (uv[up[i]] * dc[i]);
    for (int64_t p = up[i] + 1; p < up[i + 1]; ++p) {
      sc[q] = uc[p];
      sv[q] = (dr[i] * uv[p]) * dc[uc[p]];
      ++q;
    }
    sp[i + 1] = q;
  }
done:
  free(rs);
  free(rmax);
  free(cmax);
  return steps;
}

/*
 * One smoother application with row/column scaling (Alg. ILUJac with
 * Uhat = D_r U D_c, Eq. rowcolScale):  r = b - A x;  y = L^{-1} r by m_L
 * sweeps;  w^k = D_r y - Uhat_s w^{k-1} for m_U sweeps from w^0 = 0;
 * x <- x + D_c w (the final multiply of Alg. ILUJac).  m_U = 0 skips the
 * upper factor (x <- x + y).
 */
int orc_smooth_rowcol(int64_t n, int R, const int64_t* ap, const int32_t* ac, const double* av, const int64_t* lp,
                      const int32_t* lc, const double* lv, const int64_t* sp, const int32_t* sc, const double* sv,
                      const double* dr, const double* dc, double* x, const double* b, int mL, int mU) {
  const size_t sz = (size_t)(n * R > 0 ? n * R : 1);
  double* r = (double*)malloc(sz * sizeof(double));
  double* y = (double*)malloc(sz * sizeof(double));
  double* w = (double*)malloc(sz * sizeof(double));
  int st = ORC_NOMEM;
  if (!r || !y || !w) goto done;
  orc_residual(n, R, ap, ac, av, x, b, r);
  if (mL > 0) {
    if ((st = orc_richardson_lower(n, R, lp, lc, lv, r, mL, y))) goto done;
  } else {
    memcpy(y, r, sizeof(double) * (size_t)(n * R));
  }
  if (mU > 0) {
    if ((st = orc_richardson_upper(n, R, sp, sc, sv, dr, y, mU, w))) goto done;
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < R; ++k) x[i * R + k] = x[i * R + k] + dc[i] * w[i * R + k];
  } else {
    for (int64_t e = 0; e < n * R; ++e) x[e] = x[e] + y[e];
  }
  st = ORC_OK;
done:
  free(r);
  free(y);
  free(w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Numerical nilpotence: ||T_s^p||_2 (Sec. 5.2, Fig. Up)                      */
/* ------------------------------------------------------------------------ */

/*
 * Estimates of the spectral norms ||T^p||_2, p = 1..pmax, of a strictly
 * triangular T (CSR) by power iteration on (T^p)^T T^p.  For each p, from
 * v = v0 / ||v0||: `iters` times, w = T^p v (p products), s = ||w||,
 * z = (T^T)^p w (p products with the transpose, formed by scattering
 * t_ij w_i into z_j), v = z / ||z||.  out[p-1] = s of the last iteration
 * (the norm of T^p on a unit vector: a lower bound that rises to ||T^p||_2).
 * When T^p v vanishes (T nilpotent of index <= p on that vector) s = 0 and
 * the iteration for that p stops.
 */
int orc_power_norms(int64_t n, const int64_t* tp, const int32_t* tc, const double* tv, int pmax, int iters,
                    const double* v0, double* out) {
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* a = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!v || !a || !b) {
    free(v);
    free(a);
    free(b);
    return ORC_NOMEM;
  }
  const double n0 = sqrt(dot(n, v0, v0));
  for (int p = 1; p <= pmax; ++p) {
    for (int64_t i = 0; i < n; ++i) v[i] = v0[i] / n0;
    double s = 0.0;
    for (int it = 0; it < iters; ++it) {
      memcpy(a, v, sizeof(double) * (size_t)n);
      for (int k = 0; k < p; ++k) { /* a <- T a */
        orc_spmv(n, 1, tp, tc, tv, a, b);
        memcpy(a, b, sizeof(double) * (size_t)n);
      }
      s = sqrt(dot(n, a, a));
      if (s == 0.0) break;
      for (int k = 0; k < p; ++k) { /* a <- T^T a */
        for (int64_t j = 0; j < n; ++j) b[j] = 0.0;
        for (int64_t i = 0; i < n; ++i)
          for (int64_t q = tp[i]; q < tp[i + 1]; ++q) b[tc[q]] = b[tc[q]] + tv[q] * a[i];
        memcpy(a, b, sizeof(double) * (size_t)n);
      }
      const double z = sqrt(dot(n, a, a));
      if (z == 0.0) break;
      for (int64_t i = 0; i < n; ++i) v[i] = a[i] / z;
    }
    out[p - 1] = s;
  }
  free(v);
  free(a);
  free(b);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algebraic multigrid (Sec. 3: Ruge-Stueben coarsening with the strength    */
/* threshold theta, Galerkin coarse operators A_{l+1} = P^T A_l P, and the   */
/* V-cycle of Alg. mgcycle with the ILU smoother on the finest level)        */
/* ------------------------------------------------------------------------ */

#define ORC_AMG_MAXLEV 32

typedef struct {
  int64_t n, nc;
  int64_t* ap; /* A_l */
  int32_t* ac;
  double* av;
  int64_t* pp; /* P_l: n x nc (NULL on the coarsest level) */
  int32_t* pc;
  double* pv;
  int32_t* cf; /* 1 = coarse point, 0 = fine point */
} orc_amg_level;

typedef struct {
  int nlev;
  orc_amg_level lev[ORC_AMG_MAXLEV];
} orc_amg;

void orc_amg_free(orc_amg* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) {
    free(h->lev[l].ap);
    free(h->lev[l].ac);
    free(h->lev[l].av);
    free(h->lev[l].pp);
    free(h->lev[l].pc);
    free(h->lev[l].pv);
    free(h->lev[l].cf);
  }
  free(h);
}

/*
 * Strength of connection (Sec. 3): j != i strongly influences i when
 * |a_ij| >= theta * max_{k != i} |a_ik|.  s[p] = 1 marks such an entry p of
 * row i; a row without off-diagonal entries has none.
 */
static void amg_strength(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, double theta,
                         char* s) {
  for (int64_t i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int64_t p = ap[i]; p < ap[i + 1]; ++p)
      if (ac[p] != i && fabs(av[p]) > mx) mx = fabs(av[p]);
    for (int64_t p = ap[i]; p < ap[i + 1]; ++p)
      s[p] = (char)(ac[p] != i && mx > 0.0 && fabs(av[p]) >= theta * mx);
  }
}

/*
 * Ruge-Stueben first pass.  lambda_i = number of points that i strongly
 * influences.  Repeatedly the undecided point of largest lambda (smallest
 * index among equals) becomes C; every undecided point it strongly
 * influences becomes F, and each undecided point that strongly influences
 * a new F point gains one in lambda.  When the largest lambda left is zero,
 * the remaining undecided points become F.  The scan for the largest lambda
 * is a plain loop over all points.
 */
static void amg_split(int64_t n, const int64_t* ap, const int32_t* ac, const char* s, int32_t* cf) {
  int64_t* lam = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  char* und = (char*)malloc((size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    und[i] = 1;
    cf[i] = 0;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = ap[i]; p < ap[i + 1]; ++p)
      if (s[p]) lam[ac[p]]++;
  /* S^T: for each point k the rows j with k in S_j, in ascending j */
  int64_t* stp = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
  int64_t* stj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ap[n] + 1));
  for (int64_t k = 0; k < n; ++k) stp[k + 1] = stp[k] + lam[k];
  {
    int64_t* f = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t k = 0; k < n; ++k) f[k] = stp[k];
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = ap[j]; p < ap[j + 1]; ++p)
        if (s[p]) stj[f[ac[p]]++] = j;
    free(f);
  }
  for (;;) {
    int64_t best = -1;
    for (int64_t i = 0; i < n; ++i)
      if (und[i] && (best < 0 || lam[i] > lam[best])) best = i;
    if (best < 0) break;
    if (lam[best] == 0) {
      for (int64_t i = 0; i < n; ++i) und[i] = 0; /* the rest become F */
      break;
    }
    cf[best] = 1;
    und[best] = 0;
    /* points j that best strongly influences (best in S_j), ascending j */
    for (int64_t t = stp[best]; t < stp[best + 1]; ++t) {
      const int64_t j = stj[t];
      if (!und[j]) continue;
      und[j] = 0; /* F */
      for (int64_t p = ap[j]; p < ap[j + 1]; ++p)
        if (s[p] && und[ac[p]]) lam[ac[p]]++;
    }
  }
  free(lam);
  free(und);
  free(stp);
  free(stj);
}

/*
 * Direct interpolation (Stueben's, the classical choice of Ruge and
 * Stueben).  For a C point, its own coarse value.  For an F point i with
 * strong coarse neighbours C_i:  with sneg / spos the sums of the negative /
 * positive off-diagonal entries of row i and cneg / cpos the same over C_i,
 * d = a_ii, plus spos when cpos = 0 and plus sneg when cneg = 0, and
 * w_ij = -(alpha a_ij) / d, alpha = sneg / cneg for a_ij < 0, spos / cpos for
 * a_ij > 0.  An F point without strong coarse neighbours gets an empty row.
 */
static int amg_interp(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, const char* s,
                      const int32_t* cf, int64_t** pp_o, int32_t** pc_o, double** pv_o, int64_t* nc_o) {
  int64_t* cidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) cidx[i] = cf[i] ? nc++ : -1;
  int64_t* pp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t cap = ap[n] + n + 1;
  int32_t* pc = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  double* pv = (double*)malloc(sizeof(double) * (size_t)cap);
  int64_t q = 0;
  pp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i]) {
      pc[q] = (int32_t)cidx[i];
      pv[q] = 1.0;
      ++q;
    } else {
      double aii = 0.0, sneg = 0.0, spos = 0.0, cneg = 0.0, cpos = 0.0;
      for (int64_t p = ap[i]; p < ap[i + 1]; ++p) {
        const int32_t j = ac[p];
        if (j == i) {
          aii = aii + av[p];
          continue;
        }
        if (av[p] < 0.0) sneg = sneg + av[p];
        if (av[p] > 0.0) spos = spos + av[p];
        if (s[p] && cf[j]) {
          if (av[p] < 0.0) cneg = cneg + av[p];
          if (av[p] > 0.0) cpos = cpos + av[p];
        }
      }
      double d = aii;
      if (cpos == 0.0) d = d + spos;
      if (cneg == 0.0) d = d + sneg;
      const double alpha = (cneg != 0.0) ? sneg / cneg : 0.0;
      const double beta = (cpos != 0.0) ? spos / cpos : 0.0;
      for (int64_t p = ap[i]; p < ap[i + 1]; ++p) {
        const int32_t j = ac[p];
        if (j == i || !s[p] || !cf[j]) continue;
        const double f = av[p] < 0.0 ? alpha : beta;
        pc[q] = (int32_t)cidx[j];
        pv[q] = -(f * av[p]) / d;
        ++q;
      }
    }
    pp[i + 1] = q;
  }
  free(cidx);
  *pp_o = pp;
  *pc_o = pc;
  *pv_o = pv;
  *nc_o = nc;
  return ORC_OK;
}

/*
 * Galerkin product A_c = P^T A P (Sec. 3): entry (I, J) is the sum over fine
 * i with p_iI != 0 (ascending), then over j in row i of A (ascending), then
 * over J in row j of P, of (p_iI a_ij) p_jJ, added in that order.  Every
 * entry that receives a contribution is stored (columns ascending).
 */
static void amg_galerkin(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, const int64_t* pp,
                         const int32_t* pc, const double* pv, int64_t nc, int64_t** cp_o, int32_t** cc_o,
                         double** cv_o) {
  /* rows of P^T: for each coarse I the fine i with p_iI != 0, ascending */
  int64_t* tp = (int64_t*)calloc((size_t)(nc + 1), sizeof(int64_t));
  for (int64_t q = 0; q < pp[n]; ++q) tp[pc[q] + 1]++;
  for (int64_t I = 0; I < nc; ++I) tp[I + 1] += tp[I];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  int32_t* ti = (int32_t*)malloc(sizeof(int32_t) * (size_t)(pp[n] + 1));
  double* tv = (double*)malloc(sizeof(double) * (size_t)(pp[n] + 1));
  for (int64_t I = 0; I < nc; ++I) fill[I] = tp[I];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = pp[i]; q < pp[i + 1]; ++q) {
      ti[fill[pc[q]]] = (int32_t)i;
      tv[fill[pc[q]]] = pv[q];
      fill[pc[q]]++;
    }
  double* acc = (double*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
  char* hit = (char*)calloc((size_t)(nc > 0 ? nc : 1), 1);
  int64_t cap = 16, len = 0;
  int64_t* cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  int32_t* cc = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  double* cv = (double*)malloc(sizeof(double) * (size_t)cap);
  cp[0] = 0;
  for (int64_t I = 0; I < nc; ++I) {
    for (int64_t t = tp[I]; t < tp[I + 1]; ++t) {
      const int64_t i = ti[t];
      const double piI = tv[t];
      for (int64_t p = ap[i]; p < ap[i + 1]; ++p) {
        const int64_t j = ac[p];
        const double w = piI * av[p];
        for (int64_t q = pp[j]; q < pp[j + 1]; ++q) {
          acc[pc[q]] = acc[pc[q]] + w * pv[q];
          hit[pc[q]] = 1;
        }
      }
    }
    for (int64_t J = 0; J < nc; ++J) { /* plain scan of the dense accumulator */
      if (!hit[J]) continue;
      if (len == cap) {
        cap *= 2;
        cc = (int32_t*)realloc(cc, sizeof(int32_t) * (size_t)cap);
        cv = (double*)realloc(cv, sizeof(double) * (size_t)cap);
      }
      cc[len] = (int32_t)J;
      cv[len] = acc[J];
      ++len;
      acc[J] = 0.0;
      hit[J] = 0;
    }
    cp[I + 1] = len;
  }
  free(tp);
  free(fill);
  free(ti);
  free(tv);
  free(acc);
  free(hit);
  *cp_o = cp;
  *cc_o = cc;
  *cv_o = cv;
}

/*
 * AMG setup: levels are coarsened while the level has more than
 * coarse_size rows and fewer than max_levels levels exist; a level whose
 * split gives no C point, or only C points, ends the hierarchy.  The input
 * matrix is copied as level 0.
 */
orc_amg* orc_amg_setup(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, double theta,
                       int max_levels, int64_t coarse_size, int* status) {
  orc_amg* h = (orc_amg*)calloc(1, sizeof(orc_amg));
  *status = ORC_OK;
  if (max_levels > ORC_AMG_MAXLEV) max_levels = ORC_AMG_MAXLEV;
  if (max_levels < 1) max_levels = 1;
  orc_amg_level* L0 = &h->lev[0];
  L0->n = n;
  L0->ap = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  L0->ac = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ap[n] + 1));
  L0->av = (double*)malloc(sizeof(double) * (size_t)(ap[n] + 1));
  memcpy(L0->ap, ap, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(L0->ac, ac, sizeof(int32_t) * (size_t)ap[n]);
  memcpy(L0->av, av, sizeof(double) * (size_t)ap[n]);
  h->nlev = 1;
  while (h->nlev < max_levels) {
    orc_amg_level* L = &h->lev[h->nlev - 1];
    if (L->n <= coarse_size) break;
    char* s = (char*)malloc((size_t)(L->ap[L->n] + 1));
    int32_t* cf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L->n + 1));
    amg_strength(L->n, L->ap, L->ac, L->av, theta, s);
    amg_split(L->n, L->ap, L->ac, s, cf);
    int64_t nc = 0;
    for (int64_t i = 0; i < L->n; ++i) nc += cf[i];
    if (nc == 0 || nc == L->n) {
      free(s);
      free(cf);
      break;
    }
    amg_interp(L->n, L->ap, L->ac, L->av, s, cf, &L->pp, &L->pc, &L->pv, &L->nc);
    L->cf = cf;
    free(s);
    orc_amg_level* C = &h->lev[h->nlev];
    C->n = nc;
    amg_galerkin(L->n, L->ap, L->ac, L->av, L->pp, L->pc, L->pv, nc, &C->ap, &C->ac, &C->av);
    h->nlev++;
  }
  return h;
}

int orc_amg_nlev(const orc_amg* h) { return h->nlev; }

/* Sizes of level l: rows, entries of A_l, coarse points and entries of P_l (0 on the coarsest). */
void orc_amg_level_sizes(const orc_amg* h, int l, int64_t* n, int64_t* nnz, int64_t* nc, int64_t* pnnz) {
  const orc_amg_level* L = &h->lev[l];
  *n = L->n;
  *nnz = L->ap[L->n];
  *nc = L->pp ? L->nc : 0;
  *pnnz = L->pp ? L->pp[L->n] : 0;
}

/* Copy level l out (any pointer may be NULL; P and cf only below the coarsest level). */
void orc_amg_level_copy(const orc_amg* h, int l, int64_t* ap, int32_t* ac, double* av, int64_t* pp, int32_t* pc,
                        double* pv, int32_t* cf) {
  const orc_amg_level* L = &h->lev[l];
  if (ap) memcpy(ap, L->ap, sizeof(int64_t) * (size_t)(L->n + 1));
  if (ac) memcpy(ac, L->ac, sizeof(int32_t) * (size_t)L->ap[L->n]);
  if (av) memcpy(av, L->av, sizeof(double) * (size_t)L->ap[L->n]);
  if (L->pp) {
    if (pp) memcpy(pp, L->pp, sizeof(int64_t) * (size_t)(L->n + 1));
    if (pc) memcpy(pc, L->pc, sizeof(int32_t) * (size_t)L->pp[L->n]);
    if (pv) memcpy(pv, L->pv, sizeof(double) * (size_t)L->pp[L->n]);
    if (cf) memcpy(cf, L->cf, sizeof(int32_t) * (size_t)L->n);
  }
}

/* x = A^{-1} b for a small dense copy of A: Gaussian elimination with partial pivoting. */
static int dense_solve(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, const double* b,
                       double* x) {
  double* M = (double*)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!M || !y) {
    free(M);
    free(y);
    return ORC_NOMEM;
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = ap[i]; p < ap[i + 1]; ++p) M[i * n + ac[p]] = M[i * n + ac[p]] + av[p];
    y[i] = b[i];
  }
  for (int64_t k = 0; k < n; ++k) {
    int64_t piv = k;
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(M[i * n + k]) > fabs(M[piv * n + k])) piv = i;
    if (M[piv * n + k] == 0.0) {
      free(M);
      free(y);
      return ORC_ZERO_PIVOT;
    }
    if (piv != k) {
      for (int64_t j = 0; j < n; ++j) {
        const double t = M[k * n + j];
        M[k * n + j] = M[piv * n + j];
        M[piv * n + j] = t;
      }
      const double t = y[k];
      y[k] = y[piv];
      y[piv] = t;
    }
    for (int64_t i = k + 1; i < n; ++i) {
      const double f = M[i * n + k] / M[k * n + k];
      if (f == 0.0) continue;
      for (int64_t j = k; j < n; ++j) M[i * n + j] = M[i * n + j] - f * M[k * n + j];
      y[i] = y[i] - f * y[k];
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t j = i + 1; j < n; ++j) s = s - M[i * n + j] * x[j];
    x[i] = s / M[i * n + i];
  }
  free(M);
  free(y);
  return ORC_OK;
}

/* nu sweeps of l1-Jacobi on level L: x <- x + (b - A x) / d, d_i = sum_j |a_ij|. */
static void l1_jacobi(const orc_amg_level* L, const double* b, double* x, int nu) {
  const int64_t n = L->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int k = 0; k < nu; ++k) {
    orc_residual(n, 1, L->ap, L->ac, L->av, x, b, r);
    for (int64_t i = 0; i < n; ++i) {
      double d = 0.0;
      for (int64_t p = L->ap[i]; p < L->ap[i + 1]; ++p) d = d + fabs(L->av[p]);
      x[i] = x[i] + r[i] / d;
    }
  }
  free(r);
}

/* nu steps of polynomial Gauss-Seidel on level L (Sec. 3.1):
 * x <- x + sum_{j<terms} (-D^{-1} L)^j D^{-1} (b - A x). */
static int poly_gs_steps(const orc_amg_level* L, const double* b, double* x, int nu, int terms) {
  const int64_t n = L->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int st = ORC_OK;
  for (int k = 0; k < nu && !st; ++k) {
    orc_residual(n, 1, L->ap, L->ac, L->av, x, b, r);
    st = orc_poly_gs_lower(n, 1, L->ap, L->ac, L->av, r, terms - 1, z);
    for (int64_t i = 0; i < n && !st; ++i) x[i] = x[i] + z[i];
  }
  free(r);
  free(z);
  return st;
}

/* the ILU smoother of one level below the finest: row-scaled factors of A_l
   and its sweep counts */
typedef struct {
  const int64_t *lp, *sp;
  const int32_t *lc, *sc;
  const double *lv, *sv, *dinv;
  int mL, mU;
} level_ilu;

typedef struct {
  const int64_t *lp, *sp;
  const int32_t *lc, *sc;
  const double *lv, *sv, *dinv;
  int mL, mU, nu;
  int coarse; /* 0: l1-Jacobi, 1: polynomial Gauss-Seidel with `terms` terms */
  int terms;
  /* the finest level's smoother: the ILU smoother on (lp.., sp.., dinv), or,
     when schur_parts > 0, the ILUT Schur complement smoother over that many
     row blocks (ILUT(schur_tau, schur_fill) of each block, m_L + m_U sweeps) */
  int schur_parts;
  double schur_tau;
  int schur_fill;
  int schur_prec; /* interface iteration preconditioned by diag(C) (orc_schur_apply_prec) */
  /* levels 1 .. ilu_levels - 1 (above the coarsest) are smoothed by the ILU
     smoother on ilu[l] instead of the coarse smoother */
  int ilu_levels;
  const level_ilu* ilu;
} amg_smoother;

int orc_schur_apply_prec(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, int parts, double tau,
                         int fill, int mL, int mU, int iface_prec, const double* r, double* z);

/* x = x + M^{-1} (b - A_0 x) with the finest level's smoother. */
static int fine_smooth(const orc_amg_level* L, const amg_smoother* sm, const double* b, double* x) {
  const int64_t n = L->n;
  if (sm->schur_parts <= 0)
    return orc_smooth(n, 1, L->ap, L->ac, L->av, sm->lp, sm->lc, sm->lv, sm->sp, sm->sc, sm->sv, sm->dinv, x, b,
                      sm->mL, sm->mU);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  orc_residual(n, 1, L->ap, L->ac, L->av, x, b, r);
  const int st = orc_schur_apply_prec(n, L->ap, L->ac, L->av, sm->schur_parts, sm->schur_tau, sm->schur_fill,
                                      sm->mL, sm->mU, sm->schur_prec, r, z);
  if (!st)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + z[i];
  free(r);
  free(z);
  return st;
}

static int coarse_smooth(const orc_amg_level* L, const amg_smoother* sm, const double* b, double* x) {
  if (sm->coarse == 1) return poly_gs_steps(L, b, x, sm->nu, sm->terms);
  l1_jacobi(L, b, x, sm->nu);
  return ORC_OK;
}

/* The smoother of level l >= 0 (not the coarsest): the finest level's, the
   ILU smoother x = x + M_l^{-1} (b - A_l x) on level l's own factors where
   the cycle asks for ILU on that level, else the coarse smoother. */
static int level_smooth(int l, const orc_amg_level* L, const amg_smoother* sm, const double* b, double* x) {
  if (l == 0) return fine_smooth(L, sm, b, x);
  if (l < sm->ilu_levels) {
    const level_ilu* f = &sm->ilu[l];
    return orc_smooth(L->n, 1, L->ap, L->ac, L->av, f->lp, f->lc, f->lv, f->sp, f->sc, f->sv, f->dinv, x, b, f->mL,
                      f->mU);
  }
  return coarse_smooth(L, sm, b, x);
}

/* Alg. mgcycle, Multilevel(A_l, b, x, l) with nu = 1 (V-cycle). */
static int multilevel(const orc_amg* h, int l, const amg_smoother* sm, const double* b, double* x) {
  const orc_amg_level* L = &h->lev[l];
  const int64_t n = L->n;
  if (l == h->nlev - 1) /* coarsest level: direct solve */
    return dense_solve(n, L->ap, L->ac, L->av, b, x);
  int st;
  if ((st = level_smooth(l, L, sm, b, x))) return st; /* pre-smoothing */
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* bc = (double*)calloc((size_t)(L->nc > 0 ? L->nc : 1), sizeof(double));
  double* v = (double*)calloc((size_t)(L->nc > 0 ? L->nc : 1), sizeof(double));
  orc_residual(n, 1, L->ap, L->ac, L->av, x, b, r);
  /* r_{l+1} = R_l r with R_l = P_l^T: scatter row by row */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = L->pp[i]; q < L->pp[i + 1]; ++q) bc[L->pc[q]] = bc[L->pc[q]] + L->pv[q] * r[i];
  st = multilevel(h, l + 1, sm, bc, v);
  if (!st) {
    for (int64_t i = 0; i < n; ++i) { /* x = x + P_l v */
      double s = 0.0;
      for (int64_t q = L->pp[i]; q < L->pp[i + 1]; ++q) s = s + L->pv[q] * v[L->pc[q]];
      x[i] = x[i] + s;
    }
    st = level_smooth(l, L, sm, b, x); /* post-smoothing */
  }
  free(r);
  free(bc);
  free(v);
  return st;
}

/*
 * One V-cycle (Alg. mgcycle, nu = 1) on A_0 x = b, updating x in place:
 * the finest level is smoothed before and after the coarse-grid correction
 * by the ILU smoother (m_L + m_U Richardson sweeps on the row-scaled factors
 * L_s, Utilde_s, dinv), every coarser level by nu steps of l1-Jacobi
 * (coarse = 0) or of polynomial Gauss-Seidel with `terms` Neumann terms
 * (coarse = 1; Sec. 6.3's mixed V-cycle), and the coarsest level is solved
 * directly.  A single-level hierarchy is one
 * direct solve.
 */
int orc_amg_vcycle(const orc_amg* h, const int64_t* lp, const int32_t* lc, const double* lv, const int64_t* sp,
                   const int32_t* sc, const double* sv, const double* dinv, int mL, int mU, int nu, int coarse,
                   int terms, double* x, const double* b) {
  amg_smoother sm = {lp, sp, lc, sc, lv, sv, dinv, mL, mU, nu, coarse, terms, 0, 0.0, 0, 0, 1, NULL};
  return multilevel(h, 0, &sm, b, x);
}

/*
 * The V-cycle with the ILU smoother on the first `nilu` levels (Sec. 6: the
 * ILU smoother applied on any number of levels from the finest down, up to
 * all levels above the coarsest direct solve): level l < nilu is smoothed
 * before and after its coarse-grid correction by m_L[l] + m_U[l] Richardson
 * sweeps on its own row-scaled factors (lp[l] .. dinv[l]: L_s, Utilde_s and
 * D^{-1} of an incomplete factorisation of A_l); the levels below by the
 * coarse smoother as in orc_amg_vcycle.  Entries at l >= nlev - 1 are not
 * used.  nilu >= 1 (level 0's factors are entry 0).  With schur_parts > 0
 * the finest level is smoothed by the ILUT Schur complement smoother instead
 * (as in orc_amg_vcycle_schur, with m_L[0] + m_U[0] sweeps in its blocks and
 * its interface iteration preconditioned by diag(C) when schur_prec = 1;
 * entry 0's factors are then not read).
 */
int orc_amg_vcycle_ilu(const orc_amg* h, int nilu, const int64_t* const* lp, const int32_t* const* lc,
                       const double* const* lv, const int64_t* const* sp, const int32_t* const* sc,
                       const double* const* sv, const double* const* dinv, const int* mL, const int* mU, int nu,
                       int coarse, int terms, int schur_parts, double schur_tau, int schur_fill, int schur_prec,
                       double* x, const double* b) {
  if (nilu < 1 || schur_parts < 0) return ORC_BADARG;
  level_ilu* f = (level_ilu*)malloc(sizeof(level_ilu) * (size_t)nilu);
  if (!f) return ORC_NOMEM;
  for (int l = 0; l < nilu; ++l) {
    level_ilu e = {lp[l], sp[l], lc[l], sc[l], lv[l], sv[l], dinv[l], mL[l], mU[l]};
    f[l] = e;
  }
  amg_smoother sm = {lp[0], sp[0], lc[0], sc[0], lv[0], sv[0], dinv[0], mL[0], mU[0], nu, coarse, terms,
                     schur_parts, schur_tau, schur_fill, schur_prec, nilu, f};
  const int st = multilevel(h, 0, &sm, b, x);
  free(f);
  return st;
}

/*
 * The same V-cycle with the finest level smoothed, before and after the
 * coarse-grid correction, by one application of the ILUT Schur complement
 * smoother (Sec. 3.1: the smoother of one level of the V-cycle; orc_schur_apply
 * over `parts` row blocks, ILUT(tau, fill) of each block, m_L + m_U sweeps;
 * iface_prec as in orc_schur_apply_prec) instead of the ILU smoother.
 */
int orc_amg_vcycle_schur(const orc_amg* h, int parts, double tau, int fill, int iface_prec, int mL, int mU, int nu,
                         int coarse, int terms, double* x, const double* b) {
  if (parts <= 0) return ORC_BADARG;
  amg_smoother sm = {NULL, NULL, NULL, NULL, NULL, NULL, NULL, mL, mU, nu, coarse, terms, parts, tau, fill,
                     iface_prec, 1, NULL};
  return multilevel(h, 0, &sm, b, x);
}

/* ------------------------------------------------------------------------ */
/* ILUT Schur complement smoother (Sec. 3.1, Eq. schur)                       */
/* ------------------------------------------------------------------------ */

/*
 * Interface of a `parts`-way partition into contiguous row blocks (block k
 * holds rows [k n / parts, (k+1) n / parts)), the stand-in for the paper's
 * MPI ranks: row i is an interface row when it has an entry in a column of
 * another block.  iface[i] = 1 for interface rows.  Returns their number.
 */
int64_t orc_schur_interface(int64_t n, const int64_t* ap, const int32_t* ac, int parts, int32_t* iface) {
  int64_t ni = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t bi = (i * parts) / n;
    int32_t f = 0;
    for (int64_t p = ap[i]; p < ap[i + 1]; ++p) {
      /* block of column j: the k with k n / parts <= j < (k+1) n / parts */
      int64_t bj = 0;
      while ((bj + 1) * n / parts <= ac[p]) ++bj;
      if (bj != bi) f = 1;
    }
    iface[i] = f;
    ni += f;
  }
  return ni;
}

/* submatrix of A with rows `rows` (count nr) and columns mapped by cmap (-1 = dropped) */
static void submatrix(const int64_t* ap, const int32_t* ac, const double* av, const int64_t* rows, int64_t nr,
                      const int64_t* cmap, int64_t** sp_o, int32_t** sc_o, double** sv_o) {
  int64_t cnt = 0;
  for (int64_t t = 0; t < nr; ++t)
    for (int64_t p = ap[rows[t]]; p < ap[rows[t] + 1]; ++p)
      if (cmap[ac[p]] >= 0) ++cnt;
  int64_t* sp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nr + 1));
  int32_t* sc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt + 1));
  double* sv = (double*)malloc(sizeof(double) * (size_t)(cnt + 1));
  int64_t q = 0;
  sp[0] = 0;
  for (int64_t t = 0; t < nr; ++t) {
    for (int64_t p = ap[rows[t]]; p < ap[rows[t] + 1]; ++p)
      if (cmap[ac[p]] >= 0) {
        sc[q] = (int32_t)cmap[ac[p]];
        sv[q] = av[p];
        ++q;
      }
    sp[t + 1] = q;
  }
  *sp_o = sp;
  *sc_o = sc;
  *sv_o = sv;
}

typedef struct {
  int64_t nI, nG;
  int64_t *rowsI, *rowsG;     /* original row numbers, ascending */
  int64_t *bp, *ep, *fp, *cp; /* B = A_II, E = A_IG, F = A_GI, C = A_GG */
  int32_t *bc, *ec, *fc, *cc;
  double *bv, *ev, *fv, *cv;
  int64_t *lp, *sp; /* row-scaled ILUT factors of B */
  int32_t *lc, *sc;
  double *lv, *sv, *dinv;
} schur_parts;

static void schur_free(schur_parts* S) {
  void* ptrs[] = {S->rowsI, S->rowsG, S->bp, S->ep, S->fp, S->cp, S->bc, S->ec, S->fc, S->cc, S->bv, S->ev,
                  S->fv, S->cv, S->lp, S->sp, S->lc, S->sc, S->lv, S->sv, S->dinv};
  for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
}

static int schur_build(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, int parts, double tau,
                       int fill, schur_parts* S) {
  memset(S, 0, sizeof(*S));
  int32_t* iface = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  S->nG = orc_schur_interface(n, ap, ac, parts, iface);
  S->nI = n - S->nG;
  S->rowsI = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->nI + 1));
  S->rowsG = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->nG + 1));
  int64_t* mapI = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* mapG = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t a = 0, g = 0;
  for (int64_t i = 0; i < n; ++i) {
    mapI[i] = iface[i] ? -1 : a;
    mapG[i] = iface[i] ? g : -1;
    if (iface[i])
      S->rowsG[g++] = i;
    else
      S->rowsI[a++] = i;
  }
  submatrix(ap, ac, av, S->rowsI, S->nI, mapI, &S->bp, &S->bc, &S->bv);
  submatrix(ap, ac, av, S->rowsI, S->nI, mapG, &S->ep, &S->ec, &S->ev);
  submatrix(ap, ac, av, S->rowsG, S->nG, mapI, &S->fp, &S->fc, &S->fv);
  submatrix(ap, ac, av, S->rowsG, S->nG, mapG, &S->cp, &S->cc, &S->cv);
  free(iface);
  free(mapI);
  free(mapG);
  int st = ORC_OK;
  orc_lu* lu = orc_ilut(S->nI, S->bp, S->bc, S->bv, tau, fill, &st);
  if (!lu) return st ? st : ORC_NOMEM;
  int64_t nl, nu;
  orc_lu_nnz(lu, &nl, &nu);
  S->lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->nI + 1));
  S->lc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl + 1));
  S->lv = (double*)malloc(sizeof(double) * (size_t)(nl + 1));
  int64_t* up = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->nI + 1));
  int32_t* uc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nu + 1));
  double* uv = (double*)malloc(sizeof(double) * (size_t)(nu + 1));
  orc_lu_copy(lu, S->lp, S->lc, S->lv, up, uc, uv);
  orc_lu_free(lu);
  S->sp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->nI + 1));
  S->sc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nu + 1));
  S->sv = (double*)malloc(sizeof(double) * (size_t)(nu + 1));
  S->dinv = (double*)malloc(sizeof(double) * (size_t)(S->nI + 1));
  st = orc_row_scale(S->nI, up, uc, uv, S->dinv, S->sp, S->sc, S->sv);
  free(up);
  free(uc);
  free(uv);
  return st;
}

/* u = B^{-1} f approximated by the ILU smoother from zero (m_L + m_U sweeps) */
static int schur_binv(const schur_parts* S, const double* f, int mL, int mU, double* u) {
  const int64_t m = S->nI;
  double* x = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  int st = orc_smooth(m, 1, S->bp, S->bc, S->bv, S->lp, S->lc, S->lv, S->sp, S->sc, S->sv, S->dinv, x, f, mL, mU);
  memcpy(u, x, sizeof(double) * (size_t)m);
  free(x);
  return st;
}

/*
 * z = M^{-1} r for the Schur complement smoother, in the paper's order, with
 * A permuted to [B E; F C] (interior rows first, interface rows last, each
 * in ascending original order) and B ~ L D Utilde from ILUT(tau, fill)
 * (row-scaled, the triangular solves replaced by m_L + m_U sweeps):
 *   f = r_I, g = r_G;  s = g - F B^{-1} f  (right-hand side of Eq. schur);
 *   one GMRES iteration on S y = s, S = C - F B^{-1} E, from y = 0:
 *     beta = ||s||, v = s / beta, w = S v, h11 = v.w, h21 = ||w - h11 v||,
 *     Givens rho = hypot(h11, h21), y = (beta h11 / rho^2) v
 *   (no residual of the full system is formed); with iface_prec = 1 the
 *   iteration is right-preconditioned by M = diag(C) (not in the paper, which
 *   leaves the interface iteration unpreconditioned): w = S M^{-1} v and
 *   y = (beta h11 / rho^2) M^{-1} v; a zero c_kk gives ORC_ZERO_PIVOT;
 *   x_I = B^{-1} (f - E y);  z = [x_I; y] in the original order.
 */
int orc_schur_apply_prec(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, int parts, double tau,
                         int fill, int mL, int mU, int iface_prec, const double* r, double* z) {
  if (iface_prec != 0 && iface_prec != 1) return ORC_BADARG;
  schur_parts S;
  int st = schur_build(n, ap, ac, av, parts, tau, fill, &S);
  const int64_t nI = S.nI, nG = S.nG;
  const size_t mi = (size_t)(nI > 0 ? nI : 1), mg = (size_t)(nG > 0 ? nG : 1);
  double* f = (double*)malloc(sizeof(double) * mi);
  double* u = (double*)malloc(sizeof(double) * mi);
  double* t = (double*)malloc(sizeof(double) * mi);
  double* s = (double*)malloc(sizeof(double) * mg);
  double* v = (double*)malloc(sizeof(double) * mg);
  double* w = (double*)malloc(sizeof(double) * mg);
  double* y = (double*)calloc(mg, sizeof(double));
  double* q = (double*)malloc(sizeof(double) * mg);
  if (st) goto done;
  for (int64_t k = 0; k < nI; ++k) f[k] = r[S.rowsI[k]];
  /* s = g - F B^{-1} f */
  if ((st = schur_binv(&S, f, mL, mU, u))) goto done;
  orc_spmv(nG, 1, S.fp, S.fc, S.fv, u, w);
  for (int64_t k = 0; k < nG; ++k) s[k] = r[S.rowsG[k]] - w[k];
  /* one GMRES iteration on S y = s, right-preconditioned by M = diag(C) when
     iface_prec = 1 (M = I otherwise): Arnoldi on S M^{-1}, y = M^{-1} (coef v) */
  {
    const double beta = sqrt(dot(nG, s, s));
    if (beta > 0.0) {
      for (int64_t k = 0; k < nG; ++k) v[k] = s[k] / beta;
      for (int64_t k = 0; k < nG; ++k) q[k] = v[k];
      if (iface_prec == 1)
        for (int64_t k = 0; k < nG; ++k) {
          double d = 0.0; /* c_kk */
          for (int64_t p = S.cp[k]; p < S.cp[k + 1]; ++p)
            if (S.cc[p] == k) d = S.cv[p];
          if (d == 0.0) {
            st = ORC_ZERO_PIVOT;
            goto done;
          }
          q[k] = v[k] / d;                                     /* q = M^{-1} v */
        }
      orc_spmv(nI, 1, S.ep, S.ec, S.ev, q, t);                 /* E q */
      if ((st = schur_binv(&S, t, mL, mU, u))) goto done;      /* B^{-1} E q */
      orc_spmv(nG, 1, S.fp, S.fc, S.fv, u, w);                 /* F B^{-1} E q */
      double* cvv = (double*)malloc(sizeof(double) * mg);
      orc_spmv(nG, 1, S.cp, S.cc, S.cv, q, cvv);               /* C q */
      for (int64_t k = 0; k < nG; ++k) w[k] = cvv[k] - w[k];   /* w = S M^{-1} v */
      free(cvv);
      const double h11 = dot(nG, v, w);
      for (int64_t k = 0; k < nG; ++k) w[k] = w[k] - h11 * v[k];
      const double h21 = sqrt(dot(nG, w, w));
      const double rho = hypot(h11, h21);
      const double coef = rho > 0.0 ? (beta * h11) / (rho * rho) : 0.0;
      for (int64_t k = 0; k < nG; ++k) y[k] = coef * q[k];
    }
  }
  /* x_I = B^{-1} (f - E y) */
  orc_spmv(nI, 1, S.ep, S.ec, S.ev, y, t);
  for (int64_t k = 0; k < nI; ++k) t[k] = f[k] - t[k];
  if ((st = schur_binv(&S, t, mL, mU, u))) goto done;
  for (int64_t k = 0; k < nI; ++k) z[S.rowsI[k]] = u[k];
  for (int64_t k = 0; k < nG; ++k) z[S.rowsG[k]] = y[k];
done:
  schur_free(&S);
  free(f);
  free(u);
  free(t);
  free(s);
  free(v);
  free(w);
  free(y);
  free(q);
  return st;
}

int orc_schur_apply(int64_t n, const int64_t* ap, const int32_t* ac, const double* av, int parts, double tau,
                    int fill, int mL, int mU, const double* r, double* z) {
  return orc_schur_apply_prec(n, ap, ac, av, parts, tau, fill, mL, mU, 0, r, z);
}
