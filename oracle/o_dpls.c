/*
 * Oracle: Dynamic Pattern Least Squares prolongation, DPLS (Sec. 3.4,
 * Algorithm 5).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * For a fine node i the weights w minimise || v_i - V_{c,i} w || (eq. minDPLS)
 * where v_i is the test-space row of i and the columns of V_{c,i} are the rows
 * of the coarse nodes chosen so far.  The set J_i of admissible coarse nodes
 * holds the coarse nodes reachable from i by a path of at most d_p edges of
 * the filtered (strong) graph.  Coarse nodes are added greedily: the next one
 * is the candidate with maximal affinity to the current least-squares residual,
 * both taken in the trailing rows left after the Householder reflections of
 * the columns already chosen.  Its column is reduced by Householder QR; the
 * condition number of V_{c,i} is monitored through the diagonal of R
 * (max |R_kk| / min |R_kk|) and a node that would push it above kappa_p is not
 * taken and ends the loop (the paper stops "whenever cond > kappa_p" to avoid
 * large weights, so the offending node is not kept).  The loop also ends when
 * n_max nodes are chosen, when the next node would not fit in the n_tv rows,
 * when J_i is exhausted, or when the residual is exactly zero.  Finally
 * w = R^{-1} r (back substitution, inner sums from the last column down).
 * Coarse rows of P are the identity (injection); a fine node without an
 * admissible coarse node gets an empty row.
 *
 * Block form (b = 3): v_i becomes the n_tv x b block of node i's b rows (b
 * right-hand sides sharing one pattern), a candidate adds b columns, and the
 * affinity between residual block X and candidate block Y is
 * ||X^T Y||_F^2 / (||X^T X||_F ||Y^T Y||_F), the scalar affinity at b = 1.
 * The P block (i, J_m) is the transpose of rows b*m..b*m+b-1 of w.
 *
 * Householder step on column x (rows p..t-1): sigma = sqrt(sum x_k^2),
 * alpha = -sigma if x_p >= 0 else sigma, v = x with v_p = x_p - alpha,
 * vv = sum v_k^2, R_pp = alpha; a column y becomes y - ((2 v^T y) (1 / vv)) v
 * (the reciprocal of vv, not a division per column).
 * All sums ascend; each multiply-add of a sum, of the update y - f v and of
 * the back substitution is one fused multiply-add.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define TMAX 64

/* apply reflection (v from row p, vv) to column y (stride b):
 * y <- y - ((2 v.y) (1 / vv)) v */
static void reflect(int t, int p, const double *v, double vv, double *y,
                    int stride) {
  double s = 0.0;
  for (int k = p; k < t; ++k) s = fma(v[k], y[k * stride], s);
  const double f = (2.0 * s) * (1.0 / vv);
  for (int k = p; k < t; ++k) y[k * stride] = fma(-f, v[k], y[k * stride]);
}

static double affinity(int t, int p, int b, const double *X, const double *Y) {
  double xy = 0.0, xx = 0.0, yy = 0.0;
  for (int a = 0; a < b; ++a)
    for (int c = 0; c < b; ++c) {
      double sxy = 0.0, sxx = 0.0, syy = 0.0;
      for (int k = p; k < t; ++k) {
        sxy = fma(X[k * b + a], Y[k * b + c], sxy);
        sxx = fma(X[k * b + a], X[k * b + c], sxx);
        syy = fma(Y[k * b + a], Y[k * b + c], syy);
      }
      xy = fma(sxy, sxy, xy);
      xx = fma(sxx, sxx, xx);
      yy = fma(syy, syy, yy);
    }
  const double den = sqrt(xx) * sqrt(yy);
  return den > 0.0 ? xy / den : -1.0;
}

typedef struct {
  int col;
  double blk[9];
} pent;

static int cmp_pent(const void *a, const void *b) {
  const int x = ((const pent *)a)->col, y = ((const pent *)b)->col;
  return (x > y) - (x < y);
}

int or_dpls(const obsr *A, const unsigned char *strong, const int *cf,
            int t, const double *V, int n_max, int d_p, double kappa_p,
            obsr *P) {
  const int b = A->b, nn = A->nr, n = nn * b;
  if (t > TMAX || b > 3) return OR_ERR_ARG;
  int *cidx = (int *)malloc((size_t)nn * sizeof(int));
  int nc = 0;
  for (int I = 0; I < nn; ++I) cidx[I] = cf[I] == 1 ? nc++ : -1;
  int *dist = (int *)malloc((size_t)nn * sizeof(int));
  for (int I = 0; I < nn; ++I) dist[I] = -1;
  int *front = (int *)malloc((size_t)nn * sizeof(int));
  int *cand = (int *)malloc((size_t)nn * sizeof(int));
  unsigned char *taken = (unsigned char *)malloc((size_t)nn + 1);
  size_t cap = (size_t)nn * 4 + 16, used = 0;
  pent *ent = (pent *)malloc(cap * sizeof(pent));
  int *rowptr = (int *)malloc(((size_t)nn + 1) * sizeof(int));
  double *Vt = NULL;
  size_t vt_cap = 0;
  rowptr[0] = 0;
  for (int I = 0; I < nn; ++I) {
    pent row[TMAX];
    int nrow = 0;
    if (cf[I] == 1) {
      row[0].col = cidx[I];
      for (int r = 0; r < b * b; ++r) row[0].blk[r] = (r % (b + 1) == 0) ? 1.0 : 0.0;
      nrow = 1;
    } else {
      /* J_i: coarse nodes within d_p strong edges */
      int nf = 1, ncand = 0;
      front[0] = I;
      dist[I] = 0;
      for (int q = 0; q < nf; ++q) {
        const int K = front[q];
        if (dist[K] >= d_p) continue;
        for (int k = A->rowptr[K]; k < A->rowptr[K + 1]; ++k) {
          const int J = A->col[k];
          if (!strong[k] || J == K || dist[J] >= 0) continue;
          dist[J] = dist[K] + 1;
          front[nf++] = J;
          if (cf[J] == 1) cand[ncand++] = J;
        }
      }
      for (int q = 0; q < nf; ++q) dist[front[q]] = -1;
      /* sort candidates ascending */
      for (int i = 1; i < ncand; ++i) {
        const int x = cand[i];
        int j = i - 1;
        while (j >= 0 && cand[j] > x) {
          cand[j + 1] = cand[j];
          --j;
        }
        cand[j + 1] = x;
      }
      /* working copies: residual r (t x b) and candidates (t x b each) */
      double r[TMAX * 3], R[TMAX * TMAX], Y[TMAX * 3], hv[3][TMAX], hvv[3];
      memset(R, 0, sizeof R);
      for (int k = 0; k < t; ++k)
        for (int c = 0; c < b; ++c) r[k * b + c] = V[(size_t)k * n + (size_t)b * I + c];
      if ((size_t)ncand * t * b > vt_cap) {
        vt_cap = (size_t)ncand * t * b;
        Vt = (double *)realloc(Vt, vt_cap * sizeof(double));
      }
      for (int j = 0; j < ncand; ++j)
        for (int k = 0; k < t; ++k)
          for (int c = 0; c < b; ++c)
            Vt[((size_t)j * t + k) * b + c] = V[(size_t)k * n + (size_t)b * cand[j] + c];
      int sel[TMAX], nsel = 0, p = 0;
      memset(taken, 0, (size_t)(ncand > 0 ? ncand : 1));
      double rdmax = 0.0, rdmin = 0.0;
      for (;;) {
        if (nsel >= n_max || p + b > t) break;
        double rr = 0.0;
        for (int k = p; k < t; ++k)
          for (int c = 0; c < b; ++c) rr = fma(r[k * b + c], r[k * b + c], rr);
        if (rr == 0.0) break;
        int best = -1;
        double baff = 0.0;
        for (int j = 0; j < ncand; ++j) {
          if (taken[j]) continue;
          const double a = affinity(t, p, b, r, Vt + (size_t)j * t * b);
          if (a < 0.0) continue;
          if (best < 0 || a > baff) {
            best = j;
            baff = a;
          }
        }
        if (best < 0) break;
        /* tentative QR of the candidate's b columns */
        memcpy(Y, Vt + (size_t)best * t * b, (size_t)t * b * sizeof(double));
        int ok = 1;
        double dmax = rdmax, dmin = rdmin;
        for (int c = 0; c < b && ok; ++c) {
          const int pc = p + c;
          double sg = 0.0;
          for (int k = pc; k < t; ++k) sg = fma(Y[k * b + c], Y[k * b + c], sg);
          sg = sqrt(sg);
          if (!(sg > 0.0)) {
            ok = 0;
            break;
          }
          const double alpha = Y[pc * b + c] >= 0.0 ? -sg : sg;
          for (int k = 0; k < t; ++k) hv[c][k] = (k >= pc) ? Y[k * b + c] : 0.0;
          hv[c][pc] = Y[pc * b + c] - alpha;
          double vv = 0.0;
          for (int k = pc; k < t; ++k) vv = fma(hv[c][k], hv[c][k], vv);
          hvv[c] = vv;
          for (int c2 = c + 1; c2 < b; ++c2) reflect(t, pc, hv[c], vv, Y + c2, b);
          Y[pc * b + c] = alpha;
          for (int k = pc + 1; k < t; ++k) Y[k * b + c] = 0.0;
          const double ad = fabs(alpha);
          if (pc == 0) {
            dmax = ad;
            dmin = ad;
          } else {
            if (ad > dmax) dmax = ad;
            if (ad < dmin) dmin = ad;
          }
        }
        if (!ok || !(dmin > 0.0) || dmax / dmin > kappa_p) break;
        /* accept: R columns, then reflect the residual and remaining candidates */
        for (int c = 0; c < b; ++c)
          for (int k = 0; k <= p + c; ++k) R[k * TMAX + p + c] = Y[k * b + c];
        for (int c = 0; c < b; ++c) {
          for (int c2 = 0; c2 < b; ++c2) reflect(t, p + c, hv[c], hvv[c], r + c2, b);
          for (int j = 0; j < ncand; ++j) {
            if (taken[j] || j == best) continue;
            for (int c2 = 0; c2 < b; ++c2)
              reflect(t, p + c, hv[c], hvv[c], Vt + (size_t)j * t * b + c2, b);
          }
        }
        taken[best] = 1;
        sel[nsel++] = cand[best];
        p += b;
        rdmax = dmax;
        rdmin = dmin;
      }
      /* w = R^{-1} r[0:p], per right-hand side */
      double w[TMAX * 3];
      for (int c = 0; c < b; ++c)
        for (int i = p - 1; i >= 0; --i) {
          double s = r[i * b + c];
          for (int k = p - 1; k > i; --k) s = fma(-R[i * TMAX + k], w[k * b + c], s);
          w[i * b + c] = s / R[i * TMAX + i];
        }
      for (int m = 0; m < nsel; ++m) {
        row[nrow].col = cidx[sel[m]];
        for (int c = 0; c < b; ++c)
          for (int d = 0; d < b; ++d) row[nrow].blk[c * b + d] = w[(b * m + d) * b + c];
        ++nrow;
      }
      qsort(row, nrow, sizeof(pent), cmp_pent);
    }
    if (used + nrow > cap) {
      while (used + nrow > cap) cap *= 2;
      ent = (pent *)realloc(ent, cap * sizeof(pent));
    }
    memcpy(ent + used, row, (size_t)nrow * sizeof(pent));
    used += nrow;
    rowptr[I + 1] = (int)used;
  }
  or_bsr_alloc(P, nn, nc, b, (int)used);
  memcpy(P->rowptr, rowptr, ((size_t)nn + 1) * sizeof(int));
  for (size_t k = 0; k < used; ++k) {
    P->col[k] = ent[k].col;
    memcpy(P->val + k * b * b, ent[k].blk, (size_t)b * b * sizeof(double));
  }
  free(cidx); free(dist); free(front); free(cand); free(taken); free(ent); free(rowptr); free(Vt);
  return OR_OK;
}
