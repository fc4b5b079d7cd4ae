/*
 * Oracle: recursive AMG set-up (Algorithm 1), the V(1,1)-cycle (Algorithm 2,
 * with the post-smoother M^{-T} of Sec. 2 so the cycle is symmetric) and PCG
 * with x0 = 0 stopping at ||r||_2 <= rtol ||b||_2 (Sec. 4).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Levels.  Level k gets the smoother of Algorithm 3, the test space of
 * Algorithm 4, the C/F split of Sec. 3.3, the prolongation of Algorithm 5 and
 * A_{k+1} = P^T A P.  The first level's test space starts from the given
 * near-null space (rigid-body modes for elasticity) padded to n_tv columns
 * with counter-generator vectors uniform in [-1, 1) (Sec. 3.2: padding "with
 * random vectors"); a coarser level starts from the finer level's test space
 * restricted to its coarse nodes (the paper does not say; this is injection).
 * Coarsening stops at a level with at most n_coarse dofs, at max_levels, or
 * when a split keeps more than max_coarse_ratio of the nodes; the last level
 * is factorised by dense Cholesky.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

void or_default_params(or_params *p, int b) {
  memset(p, 0, sizeof *p);
  p->b = b;
  p->k_g = 4;
  p->rho_g = (b == 3) ? 2 : 4;
  p->eps_g = 1e-3;
  p->k_i = p->k_g;
  p->rho_i = p->rho_g;
  p->eps_i = p->eps_g;
  p->omega_bar = 0.8;
  p->rho_bar = 2.0 * (1.0 + (double)(p->k_g * p->rho_g));
  p->max_refine = 2;
  p->max_g_nodes = (b == 3) ? 24 : 64;
  p->lanczos_m = 20;
  p->omega_safety = 0.95;
  p->n_tv = 10;
  p->n_rq = 10;
  p->k_ritz = 1;
  p->theta = 5;
  p->n_max = 5;
  p->d_p = 2;
  p->kappa_p = 50.0;
  p->n_coarse = 1536;
  p->max_levels = 20;
  p->max_coarse_ratio = 0.9;
  p->seed = 20190205ull;
}

static int copy_bsr(const obsr *A, obsr *B) {
  const int nnzb = A->rowptr[A->nr], bb = A->b * A->b;
  if (or_bsr_alloc(B, A->nr, A->nc, A->b, nnzb)) return OR_ERR_MEM;
  memcpy(B->rowptr, A->rowptr, ((size_t)A->nr + 1) * sizeof(int));
  memcpy(B->col, A->col, (size_t)nnzb * sizeof(int));
  memcpy(B->val, A->val, (size_t)nnzb * bb * sizeof(double));
  return OR_OK;
}

int or_setup(const or_params *p, const obsr *K, int t0, const double *V0,
             or_hier **out) {
  if (!p || !K || K->b != p->b || (p->b != 1 && p->b != 3) || t0 > p->n_tv ||
      p->n_tv > 64)
    return OR_ERR_ARG;
  or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
  h->prm = *p;
  const int b = p->b, t = p->n_tv;
  int rc = copy_bsr(K, &h->lev[0].A);
  if (rc) return rc;
  int n = K->nr * b;
  double *Vin = (double *)malloc((size_t)n * t * sizeof(double));
  for (int j = 0; j < t; ++j)
    for (int i = 0; i < n; ++i)
      Vin[(size_t)j * n + i] = (j < t0) ? V0[(size_t)j * n + i]
                                        : or_uniform_pm1(p->seed, ((uint64_t)j << 40) | (uint64_t)i);
  int k = 0;
  for (;; ++k) {
    or_level *L = &h->lev[k];
    n = L->A.nr * b;
    if (n <= p->n_coarse || k == p->max_levels - 1 || k == 31) break;
    rc = or_smoother_setup(&L->A, p, k, &L->G, &L->GT, &L->omega, &L->lmax, &L->npasses);
    if (rc) break;
    L->V = (double *)malloc((size_t)n * t * sizeof(double));
    rc = or_srqcg(&L->A, &L->G, &L->GT, p->n_rq, p->k_ritz, t, Vin, L->V);
    if (rc) break;
    const int nnzb = L->A.rowptr[L->A.nr];
    double *soc = (double *)malloc((size_t)nnzb * sizeof(double));
    unsigned char *kept = (unsigned char *)malloc((size_t)nnzb + 1);
    unsigned char *strong = (unsigned char *)malloc((size_t)nnzb + 1);
    L->cf = (int *)malloc((size_t)L->A.nr * sizeof(int));
    or_soc(&L->A, t, L->V, soc);
    or_filter(&L->A, soc, p->theta, kept, strong);
    or_mis(&L->A, strong, L->cf);
    int nc = 0;
    for (int I = 0; I < L->A.nr; ++I) nc += (L->cf[I] == 1);
    if (nc == 0 || (double)nc > p->max_coarse_ratio * (double)L->A.nr) {
      free(soc); free(kept); free(strong);
      or_bsr_free(&L->G);
      or_bsr_free(&L->GT);
      free(L->cf); L->cf = NULL;
      free(L->V); L->V = NULL;
      break;
    }
    rc = or_dpls(&L->A, strong, L->cf, t, L->V, p->n_max, p->d_p, p->kappa_p, &L->P);
    free(soc); free(kept); free(strong);
    if (rc) break;
    or_transpose(&L->P, &L->R);
    rc = or_rap(&L->A, &L->P, &h->lev[k + 1].A);
    if (rc) break;
    /* next level's starting test space: rows of the coarse nodes */
    const int ncd = nc * b;
    free(Vin);
    Vin = (double *)malloc((size_t)ncd * t * sizeof(double));
    for (int j = 0; j < t; ++j) {
      int q = 0;
      for (int I = 0; I < L->A.nr; ++I)
        if (L->cf[I] == 1)
          for (int c = 0; c < b; ++c) Vin[(size_t)j * ncd + q++] = L->V[(size_t)j * n + (size_t)b * I + c];
    }
  }
  free(Vin);
  if (rc) {
    h->nlev = k + 1;
    or_free(h);
    return rc;
  }
  h->nlev = k + 1;
  /* last level: dense Cholesky */
  const obsr *Al = &h->lev[k].A;
  const int m = Al->nr * b;
  if (m > 20000) {
    or_free(h);
    return OR_ERR_COARSENING;
  }
  double *D = (double *)calloc((size_t)m * m, sizeof(double));
  for (int I = 0; I < Al->nr; ++I)
    for (int q = Al->rowptr[I]; q < Al->rowptr[I + 1]; ++q)
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c)
          D[(size_t)(b * I + r) * m + b * Al->col[q] + c] = Al->val[(size_t)q * b * b + r * b + c];
  h->Lc = (double *)malloc((size_t)m * m * sizeof(double));
  h->nc_dof = m;
  rc = (m > 0) ? or_chol(m, D, h->Lc) : OR_OK;
  free(D);
  if (rc) {
    or_free(h);
    return rc;
  }
  *out = h;
  return OR_OK;
}

void or_free(or_hier *h) {
  if (!h) return;
  for (int k = 0; k < h->nlev; ++k) {
    or_level *L = &h->lev[k];
    if (L->A.rowptr) or_bsr_free(&L->A);
    if (L->G.rowptr) or_bsr_free(&L->G);
    if (L->GT.rowptr) or_bsr_free(&L->GT);
    if (L->P.rowptr) or_bsr_free(&L->P);
    if (L->R.rowptr) or_bsr_free(&L->R);
    free(L->cf);
    free(L->V);
  }
  free(h->Lc);
  free(h);
}

/* AMG_Apply of Algorithm 2 with nu1 = nu2 = 1 and M^{-1} = omega G^T G:
 *   s = omega G^T G y            (one smoothing step from s = 0)
 *   r = y - A s; r_c = P^T r; z_c = AMG_Apply(r_c); s = s + P z_c
 *   z = s + omega G^T G (y - A s)  (post-smoothing with M^{-T} = M^{-1})
 * and the forward/backward Cholesky solve on the last level. */
static void vcycle_level(const or_hier *h, int k, const double *y, double *z) {
  const or_level *L = &h->lev[k];
  const int b = h->prm.b;
  if (k == h->nlev - 1) {
    if (h->nc_dof > 0) or_chol_solve(h->nc_dof, h->Lc, y, z);
    return;
  }
  const int n = L->A.nr * b, nc = L->P.nc * b;
  double *t = (double *)malloc((size_t)n * sizeof(double));
  double *s = (double *)malloc((size_t)n * sizeof(double));
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *yc = (double *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
  double *zc = (double *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
  or_spmv(&L->G, y, t);
  or_spmv(&L->GT, t, s);
  #pragma omp parallel for schedule(static) if (n > 65536)
  for (int i = 0; i < n; ++i) s[i] = L->omega * s[i];
  or_spmv(&L->A, s, r);
  #pragma omp parallel for schedule(static) if (n > 65536)
  for (int i = 0; i < n; ++i) r[i] = y[i] - r[i];
  or_spmv(&L->R, r, yc);
  vcycle_level(h, k + 1, yc, zc);
  or_spmv(&L->P, zc, u);
  #pragma omp parallel for schedule(static) if (n > 65536)
  for (int i = 0; i < n; ++i) s[i] = s[i] + u[i];
  or_spmv(&L->A, s, r);
  #pragma omp parallel for schedule(static) if (n > 65536)
  for (int i = 0; i < n; ++i) r[i] = y[i] - r[i];
  or_spmv(&L->G, r, t);
  or_spmv(&L->GT, t, u);
  #pragma omp parallel for schedule(static) if (n > 65536)
  for (int i = 0; i < n; ++i) z[i] = s[i] + L->omega * u[i];
  free(t); free(s); free(r); free(u); free(yc); free(zc);
}

int or_vcycle(const or_hier *h, const double *y, double *z) {
  vcycle_level(h, 0, y, z);
  return OR_OK;
}

static double dot_seq(int n, const double *x, const double *y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = s + x[i] * y[i];
  return s;
}

/* Preconditioned conjugate gradients, x0 = 0, one V-cycle per iteration;
 * iters counts products with A; convergence when ||r||_2 <= rtol ||b||_2 on
 * the recurrence residual. */
int or_pcg(const or_hier *h, const double *b, double *x, double rtol,
           int maxit, int *iters, double *relres) {
  const obsr *A = &h->lev[0].A;
  const int n = A->nr * A->b;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *q = (double *)malloc((size_t)n * sizeof(double));
  for (int i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
  }
  const double bn = sqrt(dot_seq(n, b, b));
  int it = 0, rc = OR_OK;
  double rn = bn;
  if (bn > 0.0) {
    or_vcycle(h, r, z);
    memcpy(p, z, (size_t)n * sizeof(double));
    double rz = dot_seq(n, r, z);
    for (;;) {
      if (it >= maxit) {
        rc = OR_ERR_NOT_CONVERGED;
        break;
      }
      or_spmv(A, p, q);
      const double pq = dot_seq(n, p, q);
      if (!(pq > 0.0)) {
        rc = OR_ERR_BREAKDOWN;
        break;
      }
      const double alpha = rz / pq;
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int i = 0; i < n; ++i) {
        x[i] = x[i] + alpha * p[i];
        r[i] = r[i] - alpha * q[i];
      }
      ++it;
      rn = sqrt(dot_seq(n, r, r));
      if (rn <= rtol * bn) break;
      or_vcycle(h, r, z);
      const double rz2 = dot_seq(n, r, z);
      const double beta = rz2 / rz;
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rz = rz2;
    }
  }
  *iters = it;
  *relres = bn > 0.0 ? rn / bn : 0.0;
  free(r); free(z); free(p); free(q);
  return rc;
}

/* ---- accessors for the Python wrapper ---- */
int or_h_nlev(const or_hier *h) { return h->nlev; }

/* info: nr, nnzb(A), nnzb(G), nnzb(P), nc (coarse nodes), npasses */
void or_h_level_info(const or_hier *h, int k, int *info, double *omega,
                     double *lmax) {
  const or_level *L = &h->lev[k];
  info[0] = L->A.nr;
  info[1] = L->A.rowptr[L->A.nr];
  info[2] = L->G.rowptr ? L->G.rowptr[L->G.nr] : 0;
  info[3] = L->P.rowptr ? L->P.rowptr[L->P.nr] : 0;
  info[4] = L->P.rowptr ? L->P.nc : 0;
  info[5] = L->npasses;
  *omega = L->omega;
  *lmax = L->lmax;
}

static const obsr *pick(const or_hier *h, int k, int which) {
  const or_level *L = &h->lev[k];
  switch (which) {
    case 0: return &L->A;
    case 1: return &L->G;
    case 2: return &L->GT;
    case 3: return &L->P;
    default: return &L->R;
  }
}

int or_h_bsr_size(const or_hier *h, int k, int which, int *nr, int *nc, int *nnzb) {
  const obsr *M = pick(h, k, which);
  if (!M->rowptr) return OR_ERR_ARG;
  *nr = M->nr;
  *nc = M->nc;
  *nnzb = M->rowptr[M->nr];
  return OR_OK;
}

int or_h_bsr_copy(const or_hier *h, int k, int which, int *rowptr, int *col, double *val) {
  const obsr *M = pick(h, k, which);
  if (!M->rowptr) return OR_ERR_ARG;
  const int nnzb = M->rowptr[M->nr];
  memcpy(rowptr, M->rowptr, ((size_t)M->nr + 1) * sizeof(int));
  memcpy(col, M->col, (size_t)nnzb * sizeof(int));
  memcpy(val, M->val, (size_t)nnzb * M->b * M->b * sizeof(double));
  return OR_OK;
}

int or_h_cf(const or_hier *h, int k, int *cf) {
  const or_level *L = &h->lev[k];
  if (!L->cf) return OR_ERR_ARG;
  memcpy(cf, L->cf, (size_t)L->A.nr * sizeof(int));
  return OR_OK;
}

int or_h_V(const or_hier *h, int k, double *V) {
  const or_level *L = &h->lev[k];
  if (!L->V) return OR_ERR_ARG;
  memcpy(V, L->V, (size_t)L->A.nr * h->prm.b * h->prm.n_tv * sizeof(double));
  return OR_OK;
}

int or_h_coarse_factor(const or_hier *h, double *Lc) {
  memcpy(Lc, h->Lc, (size_t)h->nc_dof * h->nc_dof * sizeof(double));
  return h->nc_dof;
}

/* Scalar (b = 1) copy of a block matrix: every block entry becomes a scalar
 * entry, explicit zeros of a stored block included (the structural pattern). */
int or_bsr_to_scalar(const obsr *A, obsr *S) {
  const int b = A->b, nnz = A->rowptr[A->nr] * b * b;
  if (or_bsr_alloc(S, A->nr * b, A->nc * b, 1, nnz)) return OR_ERR_MEM;
  int q = 0;
  for (int I = 0; I < A->nr; ++I)
    for (int r = 0; r < b; ++r) {
      for (int k = A->rowptr[I]; k < A->rowptr[I + 1]; ++k)
        for (int c = 0; c < b; ++c) {
          S->col[q] = A->col[k] * b + c;
          S->val[q] = A->val[(size_t)k * b * b + r * b + c];
          ++q;
        }
      S->rowptr[I * b + r + 1] = q;
    }
  return OR_OK;
}
