/*
 * Oracle: Galerkin coarse matrix A_{k+1} = P_k^T A_k P_k (Sec. 2; Algorithm 1,
 * "compute the new coarse level matrix").  TEST INFRASTRUCTURE ONLY.
 *
 * Computed as R (A P) with R = P^T.  Row i of AP: for each block A_ik of row i
 * (ascending k) and each block P_kc of row k (ascending c), the block product
 * A_ik P_kc is added to the accumulator of column c; likewise row I of the
 * result adds R_Ii (AP)_ic over i ascending.  A block product entry (r,c) is
 * sum_d X(r,d) Y(d,c) with d ascending from 0; it is then added to the
 * accumulator, which starts at 0.  The pattern is the structural one (no
 * dropping); columns ascend.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static int spgemm(const obsr *X, const obsr *Y, obsr *Z) {
  const int b = X->b, bb = b * b, nr = X->nr, nc = Y->nc;
  int *mark = (int *)malloc((size_t)nc * sizeof(int));
  int *cols = (int *)malloc((size_t)nc * sizeof(int));
  double *acc = (double *)malloc((size_t)nc * bb * sizeof(double));
  for (int c = 0; c < nc; ++c) mark[c] = -1;
  size_t cap = (size_t)nr * 8 + 16, used = 0;
  int *zc = (int *)malloc(cap * sizeof(int));
  double *zv = (double *)malloc(cap * bb * sizeof(double));
  int *zr = (int *)malloc(((size_t)nr + 1) * sizeof(int));
  zr[0] = 0;
  for (int i = 0; i < nr; ++i) {
    int ncol = 0;
    for (int kx = X->rowptr[i]; kx < X->rowptr[i + 1]; ++kx) {
      const int k = X->col[kx];
      const double *x = X->val + (size_t)kx * bb;
      for (int ky = Y->rowptr[k]; ky < Y->rowptr[k + 1]; ++ky) {
        const int c = Y->col[ky];
        const double *y = Y->val + (size_t)ky * bb;
        if (mark[c] != i) {
          mark[c] = i;
          cols[ncol++] = c;
          memset(acc + (size_t)c * bb, 0, bb * sizeof(double));
        }
        double *a = acc + (size_t)c * bb;
        for (int r = 0; r < b; ++r)
          for (int q = 0; q < b; ++q) {
            double s = 0.0;
            for (int d = 0; d < b; ++d) s = fma(x[r * b + d], y[d * b + q], s);
            a[r * b + q] = a[r * b + q] + s;
          }
      }
    }
    /* ascending columns */
    for (int u = 1; u < ncol; ++u) {
      const int v = cols[u];
      int w = u - 1;
      while (w >= 0 && cols[w] > v) {
        cols[w + 1] = cols[w];
        --w;
      }
      cols[w + 1] = v;
    }
    if (used + ncol > cap) {
      while (used + ncol > cap) cap *= 2;
      zc = (int *)realloc(zc, cap * sizeof(int));
      zv = (double *)realloc(zv, cap * bb * sizeof(double));
    }
    for (int u = 0; u < ncol; ++u) {
      zc[used + u] = cols[u];
      memcpy(zv + (used + u) * bb, acc + (size_t)cols[u] * bb, bb * sizeof(double));
    }
    used += ncol;
    zr[i + 1] = (int)used;
  }
  or_bsr_alloc(Z, nr, nc, b, (int)used);
  memcpy(Z->rowptr, zr, ((size_t)nr + 1) * sizeof(int));
  memcpy(Z->col, zc, used * sizeof(int));
  memcpy(Z->val, zv, used * bb * sizeof(double));
  free(mark); free(cols); free(acc); free(zc); free(zv); free(zr);
  return OR_OK;
}

int or_rap(const obsr *A, const obsr *P, obsr *Ac) {
  obsr AP, R;
  int rc = spgemm(A, P, &AP);
  if (rc) return rc;
  or_transpose(P, &R);
  rc = spgemm(&R, &AP, Ac);
  or_bsr_free(&AP);
  or_bsr_free(&R);
  return rc;
}
