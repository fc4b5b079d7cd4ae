/*
 * Oracle for aSP-AMG (Franceschini, Paludetto Magri, Mazzucco, Spiezia, Janna,
 * "A robust adaptive algebraic multigrid linear solver for structural mechanics",
 * arXiv 1902.01715).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * implementation of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may build, load or call
 * it.  It shares no code, header or table with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Everything is generic in the block size b: b = 1 is the paper's scalar
 * (per-dof) algorithm, b = 3 groups the x, y, z dofs of a mesh node, the
 * extension the paper names as future work (Sec. 5).  Every b = 3 rule below
 * reduces to the paper's rule at b = 1.
 *
 * Floating point: the oracle is compiled with -ffp-contract=off (the
 * compiler fuses nothing) and without -ffast-math.  Every sum that decides
 * structure (FSAI candidate ranking, Lanczos omega, SRQCG, SoC, DPLS
 * selection) is taken in a fixed, documented order, so that an independent
 * implementation that follows the same order reproduces it bit for bit.  The
 * accumulations of the inner product (or_dot), the block sparse product
 * (or_spmv), the dense Cholesky factor and its triangular solves
 * (or_chol, or_chol_solve), the aFSAI row functional and candidate gradients
 * and the Galerkin block product are written as explicit C99 fma() calls,
 * s <- fma(a, b, s): one rounding per term, as IEEE 754 fusedMultiplyAdd
 * defines it on every conforming machine.  All other arithmetic rounds each
 * product and each sum separately.
 */
#ifndef ASPAMG_ORACLE_H
#define ASPAMG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_SPD (-2)
#define OR_ERR_BREAKDOWN (-3)
#define OR_ERR_NOT_CONVERGED (-4)
#define OR_ERR_MEM (-5)
#define OR_ERR_COARSENING (-6)

/* Block compressed sparse row matrix: nr block rows, nc block columns, block
 * size b, blocks stored row-major (b*b doubles each), column indices ascending
 * inside each row. */
typedef struct {
  int nr, nc, b;
  int *rowptr; /* nr+1 */
  int *col;    /* nnzb */
  double *val; /* nnzb*b*b */
} obsr;

/* Parameters.  Defaults (or_default_params) follow Table "TestParam" of the
 * paper (k_g=4, rho_g=4, eps_g=1e-3, n_tv=10, n_rq=10, theta=5, n_max=5,
 * kappa_p=50); the values the paper leaves open are documented at each use. */
typedef struct {
  int b;            /* block size: 1 (paper) or 3 (nodal blocks) */
  int k_g, rho_g;   /* aFSAI steps and nodes added per step (Sec. 3.1) */
  double eps_g;     /* aFSAI exit tolerance */
  int k_i, rho_i;   /* refinement aFSAI calls in Alg. 3 */
  double eps_i;
  double omega_bar; /* Alg. 3: refine while omega < omega_bar ... */
  double rho_bar;   /* ... and nnz_r(G) (blocks per block row) < rho_bar */
  int max_refine;   /* cap on Alg. 3 refinement passes */
  int max_g_nodes;  /* cap on off-diagonal pattern nodes in a G row */
  int lanczos_m;    /* Lanczos steps for lambda_1(G A G^T) */
  double omega_safety; /* omega used in the smoother = min(1, safety*2/lambda) */
  int n_tv, n_rq, k_ritz; /* test space (Sec. 3.2, Alg. 4) */
  int theta;        /* SoC connections kept per node (Sec. 3.3) */
  int n_max, d_p;   /* DPLS: max interpolation nodes, path length (Sec. 3.4) */
  double kappa_p;   /* DPLS conditioning bound */
  int n_coarse;     /* direct solve when the level has <= n_coarse dofs */
  int max_levels;
  double max_coarse_ratio; /* stop when n_{k+1} / n_k exceeds this */
  uint64_t seed;    /* counter-based generator seed (padding, Lanczos start) */
} or_params;

void or_default_params(or_params *p, int b);

/* ---- utilities (o_util.c) ---- */
uint64_t or_splitmix64(uint64_t seed, uint64_t counter);
double or_uniform_pm1(uint64_t seed, uint64_t counter);
double or_dot(int n, const double *x, const double *y); /* fixed-order sum */
void or_spmv(const obsr *A, const double *x, double *y);  /* fixed-order rows */
int or_transpose(const obsr *A, obsr *T);
int or_bsr_alloc(obsr *A, int nr, int nc, int b, int nnzb);
void or_bsr_free(obsr *A);
const double *or_bsr_find(const obsr *A, int i, int j); /* block or NULL */
int or_chol(int m, const double *M, double *L);           /* lower Cholesky */
void or_chol_solve(int m, const double *L, const double *rhs, double *x);

/* ---- finite elements (o_fe.c) ---- */
int or_ke0(double nu, double hx, double hy, double hz, double *Ke);
/* clamp_axis: -1 none, 0 x=0 face, 2 z=0 face.  node_map[global node] = free
 * node index or -1.  K is assembled as sum_e E[e] * Ke0. */
int or_assemble(int nx, int ny, int nz, double hx, double hy, double hz,
                double nu, const double *E, int clamp_axis, obsr *K,
                int *node_map);
int or_rbm(int nx, int ny, int nz, double hx, double hy, double hz,
           const int *node_map, int nfree, double *V);
int or_load_body(int nx, int ny, int nz, double hx, double hy, double hz,
                 const double *g, const int *node_map, double *f);
int or_load_top_pressure(int nx, int ny, int nz, double hx, double hy,
                         double hz, const double *p, const int *node_map,
                         double *f);
int or_load_end_shear(int nx, int ny, int nz, double hx, double hy, double hz,
                      double total, const int *node_map, double *f);

/* ---- smoother (o_fsai.c) ---- */
int or_afsai(const obsr *A, const obsr *Gs, int ksteps, int rho, double eps,
             int max_nodes, obsr *G);
double or_lanczos_lmax(const obsr *A, const obsr *G, const obsr *GT, int m,
                       uint64_t seed, int level);
int or_smoother_setup(const obsr *A, const or_params *p, int level, obsr *G,
                      obsr *GT, double *omega, double *lmax, int *npasses);

/* ---- test space (o_srqcg.c) ---- */
int or_srqcg(const obsr *A, const obsr *G, const obsr *GT, int kmax,
             int k_ritz, int t, const double *V0, double *V);
int or_gen_eig(int t, const double *H, const double *M, double *U,
               double *lam);
void or_mgs(int n, int t, double *V);
double or_rq_line_min(double a, double b, double c, double d, double e,
                      double f);

/* ---- coarsening (o_coarsen.c) ---- */
int or_soc(const obsr *A, int t, const double *V, double *soc);
int or_filter(const obsr *A, const double *soc, int theta, unsigned char *kept,
              unsigned char *strong);
int or_mis(const obsr *A, const unsigned char *strong, int *cf);

/* ---- prolongation (o_dpls.c) ---- */
int or_dpls(const obsr *A, const unsigned char *strong, const int *cf,
            int t, const double *V, int n_max, int d_p, double kappa_p,
            obsr *P);

/* ---- Galerkin product (o_rap.c) ---- */
int or_rap(const obsr *A, const obsr *P, obsr *Ac);

/* ---- hierarchy, V-cycle, PCG (o_amg.c) ---- */
typedef struct {
  obsr A, G, GT, P, R;
  double omega, lmax;
  int npasses;
  int *cf;     /* 1 = coarse node */
  double *V;   /* test space of this level, n_dof x n_tv column-major */
} or_level;

typedef struct {
  or_params prm;
  int nlev;
  or_level lev[32];
  double *Lc;  /* dense Cholesky factor of the last level, row-major */
  int nc_dof;
} or_hier;

int or_setup(const or_params *p, const obsr *K, int t0, const double *V0,
             or_hier **out);
void or_free(or_hier *h);
int or_vcycle(const or_hier *h, const double *y, double *z);
int or_pcg(const or_hier *h, const double *b, double *x, double rtol,
           int maxit, int *iters, double *relres);

#ifdef __cplusplus
}
#endif
#endif
