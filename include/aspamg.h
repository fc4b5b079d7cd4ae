/*
 * aspamg.h -- C ABI of the GB300 library for the adaptive AMG solver aSP-AMG
 * (Franceschini, Paludetto Magri, Mazzucco, Spiezia, Janna, "A robust adaptive
 * algebraic multigrid linear solver for structural mechanics", arXiv
 * 1902.01715), with 3x3 nodal blocks, or, with amg_params.block = 1, in
 * the paper's own scalar (per-dof) form.
 *
 * Conventions shared by every entry point
 *  - Matrices are block CSR with b x b blocks, b = amg_params.block: b = 3
 *    ("BSR3", the default) groups the 3 dofs of a mesh node, b = 1 is plain
 *    scalar CSR (one row per dof, the paper's algorithm as printed).
 *    rowptr[nnodes+1], colind[nnzb] (ascending inside a row), vals[nnzb*b*b]
 *    with each block row-major; nnodes counts block rows (nodes for b = 3,
 *    dofs for b = 1).  Vectors have b*nnodes entries, dof b*I+c = component c
 *    of block row I.  Several right-hand sides are stored column-major (n x k).
 *  - Pointers are device pointers unless the argument says "host" or a
 *    `mem` argument selects AMG_MEM_HOST.  Device pointers must be usable on
 *    the handle's stream; the library never frees caller memory.
 *  - Every function returns 0 (AMG_OK) or a negative AMG_ERR_* code and never
 *    aborts or throws.  amg_last_error() gives a one-line description of the
 *    last failure on the calling thread.
 *  - The handle owns all hierarchy storage (device) and frees it in amg_free.
 *    Calls on one handle must not run concurrently.  Device storage and
 *    temporaries come from the device's default stream-ordered memory pool
 *    (cudaMallocAsync on the handle's stream); the first allocation raises
 *    that pool's release threshold so that freed memory stays in the pool
 *    for the process instead of being returned at each synchronisation.
 */
#ifndef ASPAMG_H
#define ASPAMG_H

#ifdef __cplusplus
extern "C" {
#endif

#define AMG_OK 0
#define AMG_ERR_ARG (-1)           /* invalid argument or unsupported size */
#define AMG_ERR_NOT_SPD (-2)       /* non-positive pivot (FSAI row, Ritz pencil, coarse inverse) */
#define AMG_ERR_BREAKDOWN (-3)     /* p^T A p <= 0 or a NaN/Inf in PCG */
#define AMG_ERR_NOT_CONVERGED (-4) /* maxit reached; X holds the last iterate */
#define AMG_ERR_CUDA (-5)          /* a CUDA runtime call failed */
#define AMG_ERR_COARSENING (-6)    /* coarsening stalled on a large level */
#define AMG_ERR_MEM (-7)           /* allocation failed */

#define AMG_MEM_DEVICE 0
#define AMG_MEM_HOST 1

/* precision of the V-cycle (smoother, transfers, level matrices).  The outer
 * CG recurrence, its dot products, the true residual and the coarse solve
 * are FP64 in every mode. */
#define AMG_FP64 0
#define AMG_FP32 1        /* all V-cycle data and arithmetic FP32 */
#define AMG_FP32_BF16GP 2 /* FP32, with G, G^T, P, R stored as bf16 */

typedef struct amg_handle_s *amg_handle;

/* Parameters.  amg_default_params fills the defaults of the paper's Table
 * "TestParam" (Sec. 4.1): k_g = 4, eps_g = 1e-3, n_tv = 10, n_rq = 10,
 * theta = 5, n_max = 5, kappa_p = 50, with rho_g counted in nodes (2 per
 * step) for the nodal-block form; the other defaults are the library's
 * readings of values the paper leaves open. */
typedef struct {
  int k_g, rho_g;         /* aFSAI adaptive steps, nodes added per step (Sec. 3.1) */
  double eps_g;           /* aFSAI exit tolerance */
  int k_i, rho_i;         /* refinement calls of Algorithm 3 */
  double eps_i;
  double omega_bar;       /* Algorithm 3: refine while omega < omega_bar ... */
  double rho_bar;         /* ... and blocks per block row of G < rho_bar */
  int max_refine;         /* at most this many refinement calls */
  int max_g_nodes;        /* cap on off-diagonal nodes of a G row (<= 64) */
  int lanczos_m;          /* Lanczos steps for lambda_1(G A G^T) (<= 64) */
  double omega_safety;    /* omega = min(1, omega_safety * 2 / lambda_1) */
  int n_tv, n_rq, k_ritz; /* test space size, SRQCG iterations, Ritz period (Alg. 4) */
  int theta;              /* SoC connections kept per node (Sec. 3.3) */
  int n_max, d_p;         /* DPLS: interpolation nodes, path length (Alg. 5) */
  double kappa_p;         /* DPLS conditioning bound */
  int n_coarse;           /* dense direct solve once a level has <= n_coarse dofs */
  int max_levels;
  double max_coarse_ratio;/* stop coarsening when n_{k+1}/n_k exceeds this */
  int vcycle_prec;        /* AMG_FP64 | AMG_FP32 | AMG_FP32_BF16GP */
  int maxit;              /* PCG iteration limit (1000, as in Sec. 4.2) */
  unsigned long long seed;/* counter generator: test-space padding, Lanczos start */
  int block;              /* 3: nodal 3x3 blocks (default); 1: scalar, the paper's
                           * form (its Table "TestParam" then counts rho_g in dofs:
                           * rho_g = rho_i = 4, rho_bar = 34, max_g_nodes = 64) */
} amg_params;

typedef struct {
  int nlev;
  int n_it;               /* PCG iterations of the last solve (max over columns) */
  double C_gd, C_op, C_fs;/* grid, operator and FSAI complexity (Sec. 4.1) */
  double T_sm, T_ts, T_cs, T_pl, T_rap, T_p; /* set-up phase times, seconds */
  double T_s;             /* last solve, seconds */
  int level_nodes[32];
  int level_nnzb[32];
  int level_g_nnzb[32];
  double level_omega[32];
  /* last solve, largest over its columns: the recurrence residual
   * ||r||/||b|| the CG iteration stopped on, the FP64 true residual
   * ||b - K x||/||b||, and the number of true-residual restarts */
  double relres_rec, relres_true;
  int restarts;
  int vcycle_fused_level; /* levels from this one down run as one persistent
                           * kernel (-1: every product is its own launch, the
                           * default; the environment variable
                           * AMG_VTAIL_LEVEL=<k> asks for the fused form from
                           * level k >= 1, FP64 and FP32 V-cycles only) */
} amg_stats;

/* Fill *p with the defaults.  Returns AMG_ERR_ARG for p == NULL. */
int amg_default_params(amg_params *p);

/* Build the hierarchy of Algorithm 1 (Sec. 2) for the SPD matrix K:
 * per level the aFSAI smoother of Algorithm 3, the SRQCG test space of
 * Algorithm 4 started from the near-null space V0 (padded to n_tv columns by
 * the counter generator, Sec. 3.2), the affinity C/F split of Sec. 3.3, the
 * DPLS prolongation of Algorithm 5 and A_{k+1} = P^T A P; on the last level
 * its dense explicit inverse (blocked symmetric sweeps, pivot blocks of 32; the
 * paper's Algorithm 1 uses a dense Cholesky factor, and both give the exact
 * coarse solve up to rounding).
 *   K: rowptr, colind, vals as described above, in `mem` memory; copied.
 *   V0: 3*nnodes x ntv0 column-major near-null space (e.g. the 6 rigid-body
 *       modes), ntv0 <= n_tv, in `mem` memory; copied.
 *   stream: cudaStream_t to run on (NULL: the legacy default stream).
 * Errors: AMG_ERR_ARG (bad sizes/params, or a pattern whose row pointers do
 * not start at 0, decrease or exceed rowptr[nnodes], or whose column indices
 * leave [0, nnodes) or do not increase along a row -- checked on the GPU
 * before anything else reads the pattern -- or a pattern that is not
 * symmetric: K is symmetric, and a block (i, j) stored without (j, i) is
 * refused), AMG_ERR_NOT_SPD,
 * AMG_ERR_COARSENING, AMG_ERR_CUDA, AMG_ERR_MEM.  On error *out is NULL. */
int amg_setup(const amg_params *p, int nnodes, int nnzb, const int *rowptr,
              const int *colind, const double *vals, int ntv0,
              const double *V0, int mem, void *stream, amg_handle *out);

/* K changed values on the same pattern: rebuild the whole hierarchy (the
 * adaptive set-up depends on the values).  vals in `mem` memory. */
int amg_update_values(amg_handle h, const double *vals, int mem);

/* Solve K X = B by PCG with one V(1,1)-cycle per iteration, x0 = 0, stopping
 * column j when ||r_j||_2 <= rtol ||b_j||_2 on the recurrence residual
 * (Sec. 4).  When the recurrence stops, the true residual b_j - K x_j is
 * formed in FP64 with the level-0 K on the GPU; if ||b_j - K x_j||_2 >
 * rtol ||b_j||_2 (rounding of an FP32 or bf16 V-cycle, or the recurrence and
 * true residuals straddling rtol) the recurrence restarts from the true
 * residual, keeping x_j and its iteration count: at most 8 restarts, within
 * maxit, and only while each restart halves the true residual (a smaller
 * rtol than FP64 attains on K, about eps cond(K), stops there).  B and X are
 * 3*nnodes x k column-major in `mem` memory (host buffers are staged through
 * the device inside the call).  iters[k] and relres[k] (host) receive each
 * column's iteration count (restarts included) and final FP64 true residual
 * ||b - K x||/||b||; amg_get_stats gives the largest recurrence residual too.
 * k > 1 runs the batched (block SpMM) path with per-column convergence masks.
 * The status follows the recurrence rule: AMG_ERR_NOT_CONVERGED if a column
 * hit maxit (X holds its last iterate), AMG_ERR_BREAKDOWN on p^T K p <= 0 or
 * a NaN/Inf, else AMG_OK (relres then is <= rtol unless rtol is below the
 * attainable accuracy). */
int amg_solve(amg_handle h, int k, const double *B, double *X, double rtol,
              int *iters, double *relres, int mem);

/* Adjoint solve K Lambda = G reusing the hierarchy (K is symmetric), i.e.
 * dL/df = K^{-1} dL/du.  Same arguments and errors as amg_solve. */
int amg_adjoint(amg_handle h, int k, const double *G, double *Lambda,
                double rtol, int *iters, double *relres, int mem);

/* Element sensitivities on a structured Q1-hex mesh (device pointers):
 *   grad[e] = -dEdp[e] * lam_e^T Ke0 u_e,
 * the derivative of a functional L with adjoint Lam (K Lam = dL/du) with
 * respect to an element parameter p_e when K_e = E_e(p_e) Ke0.
 * conn: ne x 8 free-node indices (-1 for a clamped node), local node
 * a = dx + 2 dy + 4 dz; Ke0: 24 x 24 row-major element matrix for E = 1;
 * U, Lam: 3*nnodes vectors.  No handle needed. */
int amg_elem_grad(int ne, const int *conn, const double *Ke0,
                  const double *dEdp, const double *U, const double *Lam,
                  double *grad, void *stream);

int amg_get_stats(amg_handle h, amg_stats *s);
void amg_free(amg_handle h);
const char *amg_strerror(int code);
const char *amg_last_error(void);

/* ---- inspection (used by the parity tests) ---- */
/* info[0..5] = nodes, nnzb(A), nnzb(G), nnzb(P), coarse nodes, refinement
 * passes of level `lev`; dbl[0..1] = omega, lambda_1 estimate. */
int amg_level_info(amg_handle h, int lev, int *info, double *dbl);
/* Host copies of level matrices: which = 0 A, 1 G, 2 G^T, 3 P, 4 R; arrays
 * sized from amg_level_info (rowptr nodes+1 / coarse nodes+1 for R). */
int amg_level_matrix(amg_handle h, int lev, int which, int *rowptr, int *col,
                     double *val);
int amg_level_cf(amg_handle h, int lev, int *cf);          /* host, 1 = C */
int amg_level_testspace(amg_handle h, int lev, double *V); /* host, n x n_tv */
/* One V-cycle z = B(y) in the handle's precision (device vectors). */
int amg_vcycle(amg_handle h, const double *y, double *z);
/* Time the solve-phase sparse product of level `lev` (which = 0 A, 1 G,
 * 2 G^T, 3 P, 4 R; storage of the handle's V-cycle precision, FP64 for the
 * level-0 A of the CG recurrence when prec_a64 != 0) over `reps` back-to-back
 * launches with CUDA events on the handle's stream.  which = 5 times instead
 * the set-up's FP64 product of A_lev with n_tv columns (the kernel the
 * test-space iteration of Algorithm 4 applies S = G A G^T with; 18 nnzb n_tv
 * flops per launch).  which = 6 times the first aFSAI pass of Algorithm 3
 * on A_lev (k_g steps from the identity pattern; *bytes = 0), lev below the
 * last level.  *ms = average launch time, *bytes = algorithmic bytes of one
 * launch (values, column indices and row pointers once, x and y once
 * each). */
int amg_bench_spmv(amg_handle h, int lev, int which, int prec_a64, int reps,
                   double *ms, double *bytes);
/* Kernel launches the library has issued in this process (graph replays
 * count each kernel node). */
long long amg_launch_count(void);

/* amg_vcycle without any memory allocation.  The paper has no counterpart:
 * this is a library service for callers that cannot allocate while they run
 * the preconditioner, for instance an outer Krylov solver of another code
 * whose device memory is all held by its own pool (a device allocation inside
 * the call would fail or fragment it), or one that keeps every allocation out of
 * its iteration loop.  Same arguments, result and precision as amg_vcycle;
 * y and z are device vectors of block*nnodes entries (the handle's rows) owned
 * by the caller.
 * Scratch: a file-scope device array of 256 bytes in the library (a flag
 * block), held by every GPU that loads the library until the process exits.
 * The first call on a device looks up the array's device address (with that
 * device current), so make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents (the call clears what
 * must start at zero); calls that overlap on the GPU, on any handles, race on
 * it and must be serialised by the caller.  No device allocation or free
 * (pool or otherwise) and no allocating library routine is called. */
int amg_vcycle_noalloc(amg_handle h, const double *y, double *z);

/* ---- row-partitioned solve (one process per GPU; the orchestration,
 * halo exchange and all-reduces are in paper_1902_01715_gb300/dist.py) ----
 * Every rank builds the same hierarchy and applies the products of its own
 * block rows.  Vectors are device arrays of the level's full length on every
 * rank; the calls run on the handle's stream and return without waiting. */
/* y = epilogue(M x) on block rows [row0, row1) of matrix `which` (0 A, 1 G,
 * 2 G^T, 3 P, 4 R) of level `lev`, FP64 storage (a handle with an FP64
 * V-cycle, or the level-0 A of any handle): ep 0 y = Mx, 1 y = w Mx,
 * 2 y = aux - Mx, 3 y = aux + w Mx, 4 y += Mx, on those rows only.  Entries
 * of x outside the rank's rows must already hold the owners' values (the
 * halo).  Errors: AMG_ERR_ARG (bad level, matrix, rows, or no FP64 copy). */
int amg_level_apply(amg_handle h, int lev, int which, int ep, int row0,
                    int row1, const double *x, double *y, const double *aux,
                    double w);
/* z = A_L^{-1} y on the last level (its explicit inverse, FP64, all rows). */
int amg_coarse_apply(amg_handle h, const double *y, double *z);
/* *out (device) = sum over i in [n0, n1) of x_i y_i in a fixed order (one
 * block: thread j sums i = n0 + j, n0 + j + 256, ..., then a binary tree). */
int amg_range_dot(long long n0, long long n1, const double *x, const double *y,
                  double *out, void *stream);
/* y_i = a x_i + b y_i for i in [n0, n1) (device vectors). */
int amg_range_axpby(long long n0, long long n1, double a, const double *x,
                    double b, double *y, void *stream);
/* out[i] = x[idx[i]] and x[idx[i]] = in[i], i < m (device arrays; idx int64):
 * packing and unpacking of halo exchanges. */
int amg_gather(long long m, const long long *idx, const double *x, double *out,
               void *stream);
int amg_scatter(long long m, const long long *idx, const double *in, double *x,
                void *stream);

/* ---- structured Q1-hex elasticity problems (problem generation) ----
 * Mesh: nodes (ix,iy,iz) with global id ix + (nx+1)(iy + (ny+1) iz) at
 * (ix hx, iy hy, iz hz); element (ex,ey,ez) id ex + nx (ey + ny ez); clamp
 * 0: nodes with ix = 0, 2: nodes with iz = 0, -1: none; free nodes keep
 * increasing global id.  K = sum_e E_e Ke0 (Sec. 1: K integrates B^T D B;
 * D is linear in E), Ke0 by 2x2x2 Gauss quadrature. */
int amg_fe_size(int nx, int ny, int nz, int clamp, int *nfree, int *nnzb);
/* node_map (host, (nx+1)(ny+1)(nz+1)) = free index or -1; rowptr/colind
 * (device) receive the 27-point block pattern; vals (device) the values for
 * the element moduli E (device, ne).  Ke0 (device, 576) receives the
 * element matrix for E = 1. */
int amg_fe_assemble(int nx, int ny, int nz, double hx, double hy, double hz,
                    double nu, const double *E, int clamp, int *node_map,
                    int *rowptr, int *colind, double *vals, double *Ke0,
                    void *stream);
/* Load vectors (device, 3*nfree, accumulated into f):
 * kind 0 body force g[3] per unit volume; kind 1 pressure p[nx*ny] on the top
 * face pushing -z; kind 2 end shear of resultant g[0] in z on the x = nx*hx
 * face; kind 3 nodal forces p[(nx+1)(ny+1)*3] on the top-face nodes. */
int amg_fe_load(int nx, int ny, int nz, double hx, double hy, double hz,
                int clamp, int kind, const double *g, const double *p,
                double *f, void *stream);
/* Scalar CSR form (b = 1) of a 3x3-block matrix (device arrays): row 3I+r
 * holds, for each block of block row I in order, its entries (3I+r, 3J+c),
 * c = 0..2, stored zeros included.  srowptr[3*nr+1], scolind[9*nnzb],
 * svals[9*nnzb] are the caller's.  Feeds amg_setup with block = 1 from the
 * structured-hex assembly. */
int amg_bsr_to_scalar(int nr, int nnzb, const int *rowptr, const int *colind,
                      const double *vals, int *srowptr, int *scolind,
                      double *svals, void *stream);

/* Rigid-body modes (device, 3*nfree x 6 column-major) about the mesh centre. */
int amg_fe_rbm(int nx, int ny, int nz, double hx, double hy, double hz,
               int clamp, double *V, void *stream);
/* Element connectivity in free-node numbering (device, ne x 8). */
int amg_fe_conn(int nx, int ny, int nz, int clamp, int *conn, void *stream);

#ifdef __cplusplus
}
#endif
#endif
