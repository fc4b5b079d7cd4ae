/*
 * Oracle utilities: counter-based random numbers, the fixed-order dot product,
 * block sparse matrix-vector products, transposition and small dense Cholesky.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * OpenMP (when compiled in) only splits loops whose iterations write disjoint
 * outputs (matrix rows, dot-product chunks, Cholesky entries of one column);
 * every value is formed by the same operations in the same order as in a
 * single thread.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the output for state seed + (counter+1)*gamma,
 * gamma = 0x9E3779B97F4A7C15, mixed by the published finaliser. */
uint64_t or_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Uniform in [-1, 1): the top 53 bits as a fraction, doubled, minus one.  All
 * three steps are exact in binary64. */
double or_uniform_pm1(uint64_t seed, uint64_t counter) {
  uint64_t m = or_splitmix64(seed, counter) >> 11;
  return ((double)m * 0x1.0p-53) * 2.0 - 1.0;
}

/* Dot product in the fixed order used for every quantity that decides
 * structure.  The vector is cut into chunks of 1024 entries.  Inside a chunk,
 * lane l (0..31) accumulates entries l, l+32, l+64, ... in increasing order
 * (s <- fma(x_i, y_i, s) from 0), and the 32 lane sums are combined by five
 * exchange steps (lane l adds lane l^16, then l^8, l^4, l^2, l^1), leaving the
 * chunk sum in every lane.  The chunk sums are combined the same way one level
 * up: lane l adds chunk sums l, l+32, l+64, ... in increasing order (from 0),
 * and five exchange steps give the total. */
static void exchange32(double *v) {
  double tmp[32];
  for (int off = 16; off >= 1; off >>= 1) {
    for (int l = 0; l < 32; ++l) tmp[l] = v[l] + v[l ^ off];
    memcpy(v, tmp, sizeof tmp);
  }
}

static double chunk_sum(int n, const double *x, const double *y, int base) {
  double lane[32];
  for (int l = 0; l < 32; ++l) {
    double s = 0.0;
    for (int i = base + l; i < base + 1024 && i < n; i += 32) s = fma(x[i], y[i], s);
    lane[l] = s;
  }
  exchange32(lane);
  return lane[0];
}

/* The chunk sums are independent of each other; with OpenMP they are formed
 * by several threads (each one exactly as above) and then combined in chunk
 * order, so the result does not depend on the number of threads. */
double or_dot(int n, const double *x, const double *y) {
  double top[32];
  for (int l = 0; l < 32; ++l) top[l] = 0.0;
  const int nch = (n + 1023) / 1024;
  if (nch <= 64) {
    for (int c = 0; c < nch; ++c) top[c % 32] = top[c % 32] + chunk_sum(n, x, y, c * 1024);
  } else {
    double *cs = (double *)malloc((size_t)nch * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nch; ++c) cs[c] = chunk_sum(n, x, y, c * 1024);
    for (int c = 0; c < nch; ++c) top[c % 32] = top[c % 32] + cs[c];
    free(cs);
  }
  exchange32(top);
  return top[0];
}

/* y = A x.  Row r of block row I: sum over the blocks of row I in stored
 * (ascending column) order, and inside a block over its columns, starting
 * from 0. */
void or_spmv(const obsr *A, const double *x, double *y) {
  const int b = A->b;
#pragma omp parallel for schedule(static) if (A->nr > 4096)
  for (int I = 0; I < A->nr; ++I) {
    for (int r = 0; r < b; ++r) {
      double s = 0.0;
      for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k) {
        const double *blk = A->val + (size_t)k * b * b;
        const int J = A->col[k];
        for (int c = 0; c < b; ++c) s = fma(blk[r * b + c], x[(size_t)J * b + c], s);
      }
      y[(size_t)I * b + r] = s;
    }
  }
}

int or_bsr_alloc(obsr *A, int nr, int nc, int b, int nnzb) {
  A->nr = nr;
  A->nc = nc;
  A->b = b;
  A->rowptr = (int *)calloc((size_t)nr + 1, sizeof(int));
  A->col = (int *)malloc(((size_t)nnzb + 1) * sizeof(int));
  A->val = (double *)calloc(((size_t)nnzb + 1) * b * b, sizeof(double));
  if (!A->rowptr || !A->col || !A->val) return OR_ERR_MEM;
  return OR_OK;
}

void or_bsr_free(obsr *A) {
  free(A->rowptr);
  free(A->col);
  free(A->val);
  memset(A, 0, sizeof *A);
}

/* Transpose: block (I,J) of A becomes block (J,I) of T, transposed.  Rows of
 * T list their columns in ascending order because A's rows are visited in
 * ascending order. */
int or_transpose(const obsr *A, obsr *T) {
  const int b = A->b, nnzb = A->rowptr[A->nr];
  if (or_bsr_alloc(T, A->nc, A->nr, b, nnzb)) return OR_ERR_MEM;
  for (int k = 0; k < nnzb; ++k) T->rowptr[A->col[k] + 1]++;
  for (int i = 0; i < A->nc; ++i) T->rowptr[i + 1] += T->rowptr[i];
  int *next = (int *)malloc(((size_t)A->nc + 1) * sizeof(int));
  if (!next) return OR_ERR_MEM;
  memcpy(next, T->rowptr, (size_t)A->nc * sizeof(int));
  for (int I = 0; I < A->nr; ++I)
    for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k) {
      const int J = A->col[k], dst = next[J]++;
      T->col[dst] = I;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c)
          T->val[(size_t)dst * b * b + c * b + r] = A->val[(size_t)k * b * b + r * b + c];
    }
  free(next);
  return OR_OK;
}

const double *or_bsr_find(const obsr *A, int i, int j) {
  int lo = A->rowptr[i], hi = A->rowptr[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) / 2, c = A->col[mid];
    if (c == j) return A->val + (size_t)mid * A->b * A->b;
    if (c < j) lo = mid + 1; else hi = mid - 1;
  }
  return NULL;
}

/* Dense Cholesky M = L L^T of an m x m row-major matrix (only the lower
 * triangle of M is read).  Entry (i,j), i >= j:
 *   s = M[i][j] - sum_{k<j} L[i][k] L[j][k]   (k ascending)
 *   L[j][j] = sqrt(s) for i = j, else L[i][j] = s * rho_j with the
 * reciprocal rho_j = 1 / L[j][j] (one correctly rounded division per column,
 * then products: a division costs many times a product on the GPU).  */
int or_chol(int m, const double *M, double *L) {
  memset(L, 0, (size_t)m * m * sizeof(double));
  for (int j = 0; j < m; ++j) {
    double s = M[j * m + j];
    for (int k = 0; k < j; ++k) s = fma(-L[j * m + k], L[j * m + k], s);
    if (!(s > 0.0)) return OR_ERR_NOT_SPD;
    const double d = sqrt(s), rho = 1.0 / d;
    L[j * m + j] = d;
#pragma omp parallel for schedule(static) if (m - j > 512)
    for (int i = j + 1; i < m; ++i) {
      double t = M[i * m + j];
      for (int k = 0; k < j; ++k) t = fma(-L[i * m + k], L[j * m + k], t);
      L[i * m + j] = t * rho;
    }
  }
  return OR_OK;
}

/* Solve L L^T x = rhs: forward substitution with k ascending, then backward
 * substitution with k descending (from m-1 down to i+1); each unknown is its
 * reduced right-hand side times 1 / L[i][i]. */
void or_chol_solve(int m, const double *L, const double *rhs, double *x) {
  double *y = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  for (int i = 0; i < m; ++i) {
    double s = rhs[i];
    for (int k = 0; k < i; ++k) s = fma(-L[i * m + k], y[k], s);
    y[i] = s * (1.0 / L[i * m + i]);
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = m - 1; k > i; --k) s = fma(-L[k * m + i], x[k], s);
    x[i] = s * (1.0 / L[i * m + i]);
  }
  free(y);
}
