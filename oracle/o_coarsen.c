/*
 * Oracle: coarsening (Sec. 3.3): affinity strength of connection on the
 * pattern of A, filtering to about theta connections per node, and coarse
 * nodes chosen as a maximal independent set of the filtered graph.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * SoC.  For adjacent dofs i, j with test-space rows v_i, v_j the paper's
 * affinity is (v_i^T v_j)^2 / ((v_i^T v_i)(v_j^T v_j)) (eq. SoCdef).  For
 * nodal blocks (b = 3) with V_I the b x n_tv rows of node I it is
 *     || V_I V_J^T ||_F^2 / ( ||V_I V_I^T||_F ||V_J V_J^T||_F ),
 * which is the scalar formula at b = 1 and equals 1 when V_J = Q V_I for an
 * orthogonal Q.  It is evaluated once per unordered pair with the smaller
 * node first, so SoC is exactly symmetric; a zero denominator gives 0.
 *
 * Filter.  The paper fixes theta, the average number of connections kept per
 * node, without the rule; here every node keeps its theta largest positive
 * connections (ties to the smaller node index) and the kept graph is made
 * symmetric by union.
 *
 * MIS.  "Maximum" independent set in the paper is read as a maximal one:
 * nodes are visited by decreasing strong degree, ties by increasing index; a
 * visited node that is still undecided becomes coarse and its strong
 * neighbours fine.  Nodes without strong connections end up coarse.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static void node_gram(int n, int b, int t, const double *V, int I, int J,
                      double *M) {
  for (int r = 0; r < b; ++r)
    for (int c = 0; c < b; ++c) {
      double s = 0.0;
      for (int k = 0; k < t; ++k)
        s = fma(V[(size_t)k * n + (size_t)b * I + r], V[(size_t)k * n + (size_t)b * J + c], s);
      M[r * b + c] = s;
    }
}

static double fro2(int b, const double *M) {
  double s = 0.0;
  for (int i = 0; i < b * b; ++i) s = fma(M[i], M[i], s);
  return s;
}

int or_soc(const obsr *A, int t, const double *V, double *soc) {
  const int b = A->b, nn = A->nr, n = nn * b;
  double *nrm = (double *)malloc((size_t)nn * sizeof(double));
  /* rows are independent (OpenMP may split them; each value is formed by
   * the same operations) */
#pragma omp parallel for schedule(static) if (nn > 4096)
  for (int I = 0; I < nn; ++I) {
    double M[9];
    node_gram(n, b, t, V, I, I, M);
    nrm[I] = sqrt(fro2(b, M));
  }
#pragma omp parallel for schedule(static) if (nn > 4096)
  for (int I = 0; I < nn; ++I)
    for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k) {
      double M[9];
      const int J = A->col[k];
      if (J == I) {
        soc[k] = 0.0;
        continue;
      }
      const int lo = I < J ? I : J, hi = I < J ? J : I;
      node_gram(n, b, t, V, lo, hi, M);
      const double num = fro2(b, M), den = nrm[lo] * nrm[hi];
      soc[k] = den > 0.0 ? num / den : 0.0;
    }
  free(nrm);
  return OR_OK;
}

static int find_pos(const obsr *A, int i, int j) {
  int lo = A->rowptr[i], hi = A->rowptr[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) / 2;
    if (A->col[mid] == j) return mid;
    if (A->col[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int or_filter(const obsr *A, const double *soc, int theta, unsigned char *kept,
              unsigned char *strong) {
  const int nn = A->nr, nnzb = A->rowptr[nn];
  memset(kept, 0, (size_t)nnzb);
  for (int I = 0; I < nn; ++I)
    for (int p = 0; p < theta; ++p) {
      int best = -1;
      for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k)
        if (!kept[k] && A->col[k] != I && soc[k] > 0.0 && (best < 0 || soc[k] > soc[best]))
          best = k;
      if (best < 0) break;
      kept[best] = 1;
    }
  for (int I = 0; I < nn; ++I)
    for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k) {
      const int J = A->col[k];
      const int kt = find_pos(A, J, I);
      strong[k] = (unsigned char)(kept[k] || (kt >= 0 && kept[kt]));
    }
  return OR_OK;
}

int or_mis(const obsr *A, const unsigned char *strong, int *cf) {
  const int nn = A->nr;
  int *deg = (int *)calloc((size_t)nn, sizeof(int));
  int *order = (int *)malloc((size_t)nn * sizeof(int));
  int maxdeg = 0;
  for (int I = 0; I < nn; ++I) {
    for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k)
      if (strong[k] && A->col[k] != I) deg[I]++;
    if (deg[I] > maxdeg) maxdeg = deg[I];
  }
  /* visiting order: degree descending, index ascending (counting sort) */
  int pos = 0;
  for (int d = maxdeg; d >= 0; --d)
    for (int I = 0; I < nn; ++I)
      if (deg[I] == d) order[pos++] = I;
  for (int I = 0; I < nn; ++I) cf[I] = -1;
  for (int q = 0; q < nn; ++q) {
    const int I = order[q];
    if (cf[I] != -1) continue;
    cf[I] = 1;
    for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k) {
      const int J = A->col[k];
      if (strong[k] && J != I && cf[J] == -1) cf[J] = 0;
    }
  }
  free(deg);
  free(order);
  return OR_OK;
}
