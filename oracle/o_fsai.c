/*
 * Oracle: the adaptive FSAI smoother S = I - omega G^T G A (Sec. 3.1), the
 * aFSAI factor aFSAI(A, G_s, k, rho, eps) (adaptive Factorized Sparse
 * Approximate Inverse, reference [JanFerSarGam15] of the paper), the Lanczos
 * estimate of lambda_1(G A G^T) and the set-up loop of Algorithm 3.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * aFSAI, as computed here.  G is lower triangular with G^T G ~ A^{-1}.  Row i
 * of G is g_i = gt_i / sqrt(psi_i) where gt_i has a unit entry at i and its
 * other entries gh on the pattern Q_i (indices < i) solve
 *     A[Q,Q] gh = -A[Q,i],          psi_i = a_ii + A[i,Q] gh,
 * which minimises gt^T A gt = psi_i (the row's Kaporin functional) over the
 * pattern and gives (G A G^T)_ii = 1.  The pattern grows in k steps: the
 * gradient of gt^T A gt with respect to an entry j outside the pattern is
 * 2 (A gt)_j; the rho entries with the largest gradient are added, the row is
 * re-solved, and the row stops early when psi decreased by no more than eps
 * relative to its previous value.
 *
 * Order of the row system (the method does not fix it): the pattern nodes in
 * the order they were added -- the starting pattern (a row of G_s) in
 * ascending order, then each step's nodes in the order they were picked --
 * so every step only appends to the system (the factor of the earlier nodes
 * stays valid, and the GPU factors only the new rows); the gradient and psi
 * sums run over the pattern in the same order; G is written with its pattern
 * in ascending order.
 *
 * Block form (b = 3).  The pattern is kept per node: node row I holds a set of
 * nodes J < I, and each dof row c of node I uses all dofs of those nodes plus
 * the dofs of I below c (so the diagonal block is lower triangular).  A
 * candidate node J is scored by the sum of squares of the gradient entries of
 * its b dofs over the b rows of I; rho counts nodes; the early stop needs
 * every one of the b rows to have stalled.  At b = 1 all three rules are the
 * scalar rules above.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

static double a_entry(const obsr *A, int r, int c) {
  const int b = A->b;
  const double *blk = or_bsr_find(A, r / b, c / b);
  return blk ? blk[(r % b) * b + (c % b)] : 0.0;
}

/* Solve the b dof rows of node I for the node pattern pat[0..np-1]. gh[c] has
 * room for b*np + b entries. */
static int solve_rows(const obsr *A, int I, const int *pat, int np,
                      double **gh, double *psi, double *M, double *L,
                      double *rhs, int *Q) {
  const int b = A->b;
  for (int c = 0; c < b; ++c) {
    const int i = b * I + c;
    int m = 0;
    for (int j = 0; j < np; ++j)
      for (int e = 0; e < b; ++e) Q[m++] = b * pat[j] + e;
    for (int e = 0; e < c; ++e) Q[m++] = b * I + e;
    for (int a = 0; a < m; ++a) {
      for (int a2 = 0; a2 < m; ++a2) M[a * m + a2] = a_entry(A, Q[a], Q[a2]);
      rhs[a] = -a_entry(A, Q[a], i);
    }
    if (m > 0) {
      int rc = or_chol(m, M, L);
      if (rc) return rc;
      or_chol_solve(m, L, rhs, gh[c]);
    }
    double s = a_entry(A, i, i);
    for (int a = 0; a < m; ++a) s = fma(a_entry(A, i, Q[a]), gh[c][a], s);
    if (!(s > 0.0)) return OR_ERR_NOT_SPD;
    psi[c] = s;
  }
  return OR_OK;
}

static int cmp_int(const void *a, const void *b) {
  const int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* Per-thread work space of one aFSAI row. */
typedef struct {
  int *pat, *Q, *cand;
  double *ghbuf, *M, *L, *rhs, *score;
  long *mark; /* per node: the row-and-step stamp that last marked it */
  long stamp;
} afsai_ws;

/* Row I of aFSAI: its pattern nodes (ascending, *np_out of them, into
 * pat_out) and its np+1 blocks (pattern blocks, then the diagonal block) into
 * val_out. */
static int afsai_row(const obsr *A, const obsr *Gs, int I, int ksteps, int rho, double eps,
                     int max_nodes, afsai_ws *w, int *np_out, int *pat_out, double *val_out) {
  const int b = A->b;
  const int mmax = b * max_nodes + b;
  int *pat = w->pat, *cand = w->cand;
  double *score = w->score;
  double *gh[3];
  for (int c = 0; c < b; ++c) gh[c] = w->ghbuf + (size_t)c * mmax;
  double psi[3], psi_old[3];
  int np = 0;
  if (Gs)
    for (int k = Gs->rowptr[I]; k < Gs->rowptr[I + 1]; ++k)
      if (Gs->col[k] != I && np < max_nodes) pat[np++] = Gs->col[k];
  int rc = solve_rows(A, I, pat, np, gh, psi, w->M, w->L, w->rhs, w->Q);
  for (int step = 0; step < ksteps && rc == OR_OK; ++step) {
    if (np >= max_nodes) break;
    /* candidates: nodes J < I, outside the pattern, adjacent in A to the
     * pattern or to I */
    int nc = 0;
    ++w->stamp; /* fresh mark for this row and step */
    const long stamp = w->stamp;
    for (int j = 0; j < np; ++j) w->mark[pat[j]] = stamp;
    for (int j = 0; j <= np; ++j) {
      const int K = (j < np) ? pat[j] : I;
      for (int k = A->rowptr[K]; k < A->rowptr[K + 1]; ++k) {
        const int J = A->col[k];
        if (J < I && w->mark[J] != stamp) {
          w->mark[J] = stamp;
          cand[nc++] = J;
        }
      }
    }
    qsort(cand, nc, sizeof(int), cmp_int);
    for (int t = 0; t < nc; ++t) {
      const int J = cand[t];
      double s = 0.0;
      for (int c = 0; c < b; ++c)
        for (int d = 0; d < b; ++d) {
          double g = 0.0;
          for (int j = 0; j < np; ++j) {
            const double *blk = or_bsr_find(A, J, pat[j]);
            if (blk)
              for (int e = 0; e < b; ++e) g = fma(blk[d * b + e], gh[c][b * j + e], g);
          }
          const double *blk = or_bsr_find(A, J, I);
          if (blk) {
            for (int e = 0; e < c; ++e) g = fma(blk[d * b + e], gh[c][b * np + e], g);
            g = g + blk[d * b + c] * 1.0;
          }
          s = fma(g, g, s);
        }
      score[t] = s;
    }
    /* take up to rho best (score > 0, ties to the smaller node) */
    int want = rho < max_nodes - np ? rho : max_nodes - np, got = 0;
    for (int p = 0; p < want; ++p) {
      int best = -1;
      for (int t = 0; t < nc; ++t)
        if (score[t] > 0.0 && (best < 0 || score[t] > score[best])) best = t;
      if (best < 0) break;
      pat[np + got++] = cand[best];
      score[best] = -1.0;
    }
    if (got == 0) break;
    np += got; /* the new nodes stay after the old ones (insertion order) */
    for (int c = 0; c < b; ++c) psi_old[c] = psi[c];
    rc = solve_rows(A, I, pat, np, gh, psi, w->M, w->L, w->rhs, w->Q);
    if (rc) break;
    int stalled = 1;
    for (int c = 0; c < b; ++c)
      if (psi_old[c] - psi[c] > eps * psi_old[c]) stalled = 0;
    if (stalled) break;
  }
  if (rc) return rc;
  /* row I: pattern blocks in ascending node order, then the diagonal block;
   * ord[j] = position in the row system of the j-th smallest pattern node */
  int *ord = w->cand; /* the candidate list is free once the row is done */
  for (int j = 0; j < np; ++j) ord[j] = j;
  for (int u = 1; u < np; ++u) {
    const int v = ord[u];
    int w = u - 1;
    while (w >= 0 && pat[ord[w]] > pat[v]) {
      ord[w + 1] = ord[w];
      --w;
    }
    ord[w + 1] = v;
  }
  for (int j = 0; j <= np; ++j) {
    double *blk = val_out + (size_t)j * b * b;
    const int q = j < np ? ord[j] : np;
    if (j < np) pat_out[j] = pat[q];
    for (int c = 0; c < b; ++c) {
      const double rs = 1.0 / sqrt(psi[c]); /* g / sqrt(psi) as g times 1 / sqrt(psi) */
      for (int d = 0; d < b; ++d) {
        double g;
        if (j < np) g = gh[c][b * q + d];
        else g = (d < c) ? gh[c][b * np + d] : (d == c ? 1.0 : 0.0);
        blk[c * b + d] = (j < np || d <= c) ? g * rs : 0.0;
      }
    }
  }
  *np_out = np;
  return OR_OK;
}

/* aFSAI of A continuing from the pattern of Gs (NULL: from the identity).
 * Rows are independent: with OpenMP a batch of rows is computed by several
 * threads (each row exactly as in a single thread, into its own slot), and
 * the batch is appended to G in row order. */
int or_afsai(const obsr *A, const obsr *Gs, int ksteps, int rho, double eps,
             int max_nodes, obsr *G) {
  const int b = A->b, n = A->nr, bb = b * b;
  const int mmax = b * max_nodes + b;
  const int batch = 8192;
  int rc = OR_OK;
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  afsai_ws *ws = (afsai_ws *)calloc((size_t)nthr, sizeof(afsai_ws));
  for (int t = 0; t < nthr; ++t) {
    ws[t].pat = (int *)malloc((size_t)(max_nodes + 1) * sizeof(int));
    ws[t].ghbuf = (double *)calloc((size_t)b * mmax, sizeof(double));
    ws[t].M = (double *)malloc((size_t)mmax * mmax * sizeof(double));
    ws[t].L = (double *)malloc((size_t)mmax * mmax * sizeof(double));
    ws[t].rhs = (double *)malloc((size_t)mmax * sizeof(double));
    ws[t].Q = (int *)malloc((size_t)mmax * sizeof(int));
    ws[t].mark = (long *)malloc((size_t)n * sizeof(long));
    ws[t].cand = (int *)malloc((size_t)n * sizeof(int));
    ws[t].score = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) ws[t].mark[i] = -1;
    ws[t].stamp = -1;
  }
  int *bnp = (int *)malloc((size_t)batch * sizeof(int));
  int *bpat = (int *)malloc((size_t)batch * max_nodes * sizeof(int));
  double *bval = (double *)malloc((size_t)batch * (max_nodes + 1) * bb * sizeof(double));
  int *brc = (int *)malloc((size_t)batch * sizeof(int));
  /* output rows, grown as needed */
  size_t cap = (size_t)n * 4 + 16, used = 0;
  int *gcol = (int *)malloc(cap * sizeof(int));
  double *gval = (double *)malloc(cap * bb * sizeof(double));
  int *growptr = (int *)malloc(((size_t)n + 1) * sizeof(int));
  growptr[0] = 0;

  for (int I0 = 0; I0 < n && rc == OR_OK; I0 += batch) {
    const int nb = n - I0 < batch ? n - I0 : batch;
#pragma omp parallel for schedule(dynamic, 16)
    for (int q = 0; q < nb; ++q) {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      brc[q] = afsai_row(A, Gs, I0 + q, ksteps, rho, eps, max_nodes, &ws[t], &bnp[q],
                         bpat + (size_t)q * max_nodes, bval + (size_t)q * (max_nodes + 1) * bb);
    }
    for (int q = 0; q < nb; ++q) {
      if (brc[q]) {
        rc = brc[q];
        break;
      }
      const int I = I0 + q, np = bnp[q];
      if (used + np + 1 > cap) {
        while (used + np + 1 > cap) cap *= 2;
        gcol = (int *)realloc(gcol, cap * sizeof(int));
        gval = (double *)realloc(gval, cap * bb * sizeof(double));
      }
      for (int j = 0; j < np; ++j) gcol[used + j] = bpat[(size_t)q * max_nodes + j];
      gcol[used + np] = I;
      memcpy(gval + used * bb, bval + (size_t)q * (max_nodes + 1) * bb, (size_t)(np + 1) * bb * sizeof(double));
      used += np + 1;
      growptr[I + 1] = (int)used;
    }
  }
  if (rc == OR_OK) {
    or_bsr_alloc(G, n, n, b, (int)used);
    memcpy(G->rowptr, growptr, ((size_t)n + 1) * sizeof(int));
    memcpy(G->col, gcol, used * sizeof(int));
    memcpy(G->val, gval, used * bb * sizeof(double));
  }
  for (int t = 0; t < nthr; ++t) {
    free(ws[t].pat); free(ws[t].ghbuf); free(ws[t].M); free(ws[t].L); free(ws[t].rhs);
    free(ws[t].Q); free(ws[t].mark); free(ws[t].cand); free(ws[t].score);
  }
  free(ws); free(bnp); free(bpat); free(bval); free(brc);
  free(gcol); free(gval); free(growptr);
  return rc;
}

/* Sturm count: number of eigenvalues of the symmetric tridiagonal matrix
 * (alpha, beta) that are smaller than x, as the number of sign changes in the
 * sequence of leading principal minors of T - x I:
 *   q_0 = 1, q_1 = a_0 - x, q_{i+1} = (a_i - x) q_i - b_{i-1}^2 q_{i-1}
 * (each product and difference rounded once, in that order).  The recurrence
 * needs no division (on the GPU a division costs about ten products).  A minor
 * that is exactly zero is replaced by q_{i-1} 2^-200 (the sign of the one
 * before it: the next minor then records the change); when a minor's binary
 * exponent leaves [-512, 511] it and its predecessor are multiplied by 2^-512
 * or 2^512, which is exact and keeps every sign. */
static int bexp(double v) {
  uint64_t u;
  memcpy(&u, &v, sizeof u);
  return (int)((u >> 52) & 0x7ff) - 1023;
}

static int sturm_count(int m, const double *al, const double *be, double x) {
  int cnt = 0;
  double qp = 1.0, q = 1.0;
  for (int i = 0; i < m; ++i) {
    double qn = (i == 0) ? (al[0] - x) : (al[i] - x) * q - (be[i - 1] * be[i - 1]) * qp;
    if (qn == 0.0) qn = q * 0x1p-200;
    if ((qn < 0.0) != (q < 0.0)) ++cnt;
    qp = q;
    q = qn;
    const int e = bexp(q);
    if (e > 511) {
      q = q * 0x1p-512;
      qp = qp * 0x1p-512;
    } else if (e < -512) {
      q = q * 0x1p512;
      qp = qp * 0x1p512;
    }
  }
  return cnt;
}

/* Largest eigenvalue of G A G^T estimated by m Lanczos steps with full
 * re-orthogonalisation (one classical Gram-Schmidt pass against all previous
 * vectors; the paper says only "a few Lanczos passes"; every multiply-add of
 * the vector updates is one fused multiply-add and the normalisations multiply
 * by the reciprocal of the norm),
 * from the start vector of level `level` of the counter generator; the
 * largest Ritz value is found by bisection on Sturm counts. */
double or_lanczos_lmax(const obsr *A, const obsr *G, const obsr *GT, int m,
                       uint64_t seed, int level) {
  const int n = A->nr * A->b;
  if (m > n) m = n;
  if (m > 64) m = 64;
  double *Vs = (double *)malloc((size_t)m * n * sizeof(double));
  double *w = (double *)malloc((size_t)n * sizeof(double));
  double *t1 = (double *)malloc((size_t)n * sizeof(double));
  double *t2 = (double *)malloc((size_t)n * sizeof(double));
  double al[64], be[64], hk[64];
  for (int i = 0; i < n; ++i)
    Vs[i] = or_uniform_pm1(seed, (1ull << 62) | ((uint64_t)level << 40) | (uint64_t)i);
  double nr = sqrt(or_dot(n, Vs, Vs));
  {
    const double rn = 1.0 / nr;
    for (int i = 0; i < n; ++i) Vs[i] = Vs[i] * rn;
  }
  int mm = m;
  for (int j = 0; j < m; ++j) {
    double *v = Vs + (size_t)j * n;
    or_spmv(GT, v, t1);
    or_spmv(A, t1, t2);
    or_spmv(G, t2, w);
    al[j] = or_dot(n, w, v);
#pragma omp parallel for schedule(static) if (n > 65536)
    for (int i = 0; i < n; ++i) w[i] = fma(-al[j], v[i], w[i]);
    if (j > 0) {
      const double *vp = Vs + (size_t)(j - 1) * n;
#pragma omp parallel for schedule(static) if (n > 65536)
      for (int i = 0; i < n; ++i) w[i] = fma(-be[j - 1], vp[i], w[i]);
    }
    /* one classical Gram-Schmidt pass against v_0..v_j: all coefficients
     * from the same w, then w_i - sum_k h_k v_k,i with k ascending */
    for (int k = 0; k <= j; ++k) hk[k] = or_dot(n, w, Vs + (size_t)k * n);
#pragma omp parallel for schedule(static) if (n > 65536)
    for (int i = 0; i < n; ++i) {
      double s = w[i];
      for (int k = 0; k <= j; ++k) s = fma(-hk[k], Vs[(size_t)k * n + i], s);
      w[i] = s;
    }
    be[j] = sqrt(or_dot(n, w, w));
    if (j == m - 1) break;
    if (!(be[j] > 1e-12 * fabs(al[j]))) {
      mm = j + 1;
      break;
    }
    double *vn = Vs + (size_t)(j + 1) * n;
    const double rb = 1.0 / be[j];
    for (int i = 0; i < n; ++i) vn[i] = w[i] * rb;
  }
  double lo = al[0], hi = al[0];
  for (int i = 0; i < mm; ++i) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < mm - 1 ? fabs(be[i]) : 0.0);
    if (al[i] - r < lo) lo = al[i] - r;
    if (al[i] + r > hi) hi = al[i] + r;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm_count(mm, al, be, mid) >= mm) hi = mid; else lo = mid;
  }
  free(Vs); free(w); free(t1); free(t2);
  return hi;
}

/* Algorithm 3 (Smoother_SetUp): G from scratch with (k_g, rho_g, eps_g), then
 * refined with (k_i, rho_i, eps_i) while 2/lambda_1 < omega_bar and the
 * average number of blocks per block row of G is below rho_bar (at most
 * max_refine passes).  The smoother's omega obeys omega < min(1, 2/lambda_1)
 * (Sec. 3.1): it is min(1, omega_safety * 2/lambda_1), the safety factor
 * covering the Lanczos under-estimate of lambda_1. */
int or_smoother_setup(const obsr *A, const or_params *p, int level, obsr *G,
                      obsr *GT, double *omega, double *lmax, int *npasses) {
  int rc = or_afsai(A, NULL, p->k_g, p->rho_g, p->eps_g, p->max_g_nodes, G);
  if (rc) return rc;
  or_transpose(G, GT);
  double lam = or_lanczos_lmax(A, G, GT, p->lanczos_m, p->seed, level);
  double w = 2.0 / lam;
  int passes = 0;
  while (w < p->omega_bar &&
         (double)G->rowptr[G->nr] / (double)G->nr < p->rho_bar &&
         passes < p->max_refine) {
    obsr G2;
    rc = or_afsai(A, G, p->k_i, p->rho_i, p->eps_i, p->max_g_nodes, &G2);
    if (rc) return rc;
    or_bsr_free(G);
    or_bsr_free(GT);
    *G = G2;
    or_transpose(G, GT);
    lam = or_lanczos_lmax(A, G, GT, p->lanczos_m, p->seed, level);
    w = 2.0 / lam;
    ++passes;
  }
  double om = p->omega_safety * w;
  if (om > 1.0) om = 1.0;
  *omega = om;
  *lmax = lam;
  *npasses = passes;
  return OR_OK;
}
