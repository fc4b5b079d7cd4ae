// Internal declarations of the aSP-AMG GB300 library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "../../include/aspamg.h"

namespace amg {

void set_error(const char *fmt, ...);

#define AMG_CU(x)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      ::amg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
      return AMG_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)

#define AMG_TRY(x)            \
  do {                        \
    int rc_ = (x);            \
    if (rc_) return rc_;      \
  } while (0)

#define AMG_LAUNCH_CHECK() AMG_CU(cudaGetLastError())

// Every kernel launch site is prefixed with AMG_KCOUNT (a comma expression),
// so the library can report how many kernels it issued.
void count_launches(long long n);
#define AMG_KCOUNT ::amg::count_launches(1),

// Device memory comes from the device's stream-ordered pool: a buffer is
// taken and given back in the order of the stream that is current for the
// calling thread when it is allocated (the entry points make the handle's
// stream current).  The set-up allocates and frees hundreds of temporaries;
// cudaFree would synchronise the device each time, and the pool keeps freed
// memory for reuse instead of returning it to the driver.
cudaStream_t current_stream();
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s);
  ~StreamScope();
};
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);

// Programmatic dependent launch.  While a PdlScope(true) lives on the
// calling thread (the hierarchy set-up, a solve, a V-cycle), launch_k issues
// kernels with programmatic stream serialisation: a kernel may be scheduled
// while the kernel before it in the stream is still running, once every CTA
// of that kernel has issued pdl_trigger() (or exited), so its launch and
// prologue overlap the end of the one before it.  pdl_wait() returns when
// the preceding grid has completed and its memory operations are visible.
// Every kernel launched through launch_k calls it before touching memory
// that kernels write -- the set-up kernels as their first statement; the
// solve-phase kernels first load their row data and first matrix blocks
// (the solve layout, written by the set-up, which ends with a stream
// synchronisation before any solve) and write nothing before it.  The
// solve-phase kernels issue pdl_trigger() after their main loop: issued at
// the start, it let the next kernel's CTAs crowd onto the SMs that freed
// first, and the solve became slower than without programmatic launch.
// A PdlScope(false) (building the solve layout and timing its mappings,
// whose kernels read a layout that the kernel just before may be writing)
// and no scope at all (the timing entry points) give plain launches, where
// pdl_wait() returns at once; AMG_NO_PDL in the environment makes every
// launch plain.
bool pdl_enabled();
struct PdlScope {
  bool prev;
  explicit PdlScope(bool on = true);
  ~PdlScope();
};
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t shm, cudaStream_t s, A... args) {
  count_launches(1);
  if (!pdl_enabled()) {
    k<<<grid, block, shm, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = shm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);  // a failure is left for the caller's launch check
}

// Owning device buffer (pool allocation on the current stream; freed on the
// same stream).
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  int alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    s = current_stream();
    cudaError_t e = pool_alloc((void **)&p, count * sizeof(T), s);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return AMG_ERR_MEM;
    }
    n = count;
    return AMG_OK;
  }
  int zero(cudaStream_t s) {
    if (!p) return AMG_OK;
    AMG_CU(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    return AMG_OK;
  }
};

// Block CSR matrix with b x b blocks (b = 3: nodal blocks; b = 1: the
// scalar matrix of the paper's per-dof method; b = 0: a pattern without
// values), values row-major per block ("AoS"), all on the device.
struct DevBsr {
  int nr = 0, nc = 0, nnzb = 0, b = 3;
  DBuf<int> rowptr, col;
  DBuf<double> val;
  mutable int maxlen = -1;  // longest row, once known
  int alloc(int nr_, int nc_, int nnzb_, int b_) {
    nr = nr_; nc = nc_; nnzb = nnzb_; b = b_;
    maxlen = -1;
    AMG_TRY(rowptr.alloc(nr + 1));
    AMG_TRY(col.alloc(nnzb));
    AMG_TRY(val.alloc((size_t)nnzb * b * b));
    return AMG_OK;
  }
  // longest row (a device reduction the first time, then kept)
  int row_max(cudaStream_t s, int *out) const;
  // blocking copy of the pattern to host arrays (rowptr: nr + 1, col: nnzb)
  int copy_pattern(int *h_rowptr, int *h_col) const {
    if (h_rowptr) AMG_CU(cudaMemcpy(h_rowptr, rowptr.p, (nr + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    if (h_col && nnzb) AMG_CU(cudaMemcpy(h_col, col.p, (size_t)nnzb * sizeof(int), cudaMemcpyDeviceToHost));
    return AMG_OK;
  }
};

// Solve-phase copy of a level matrix in the sliced layout of spmv.cu: block
// rows in slices of 32, slice s owning slots [slp[s], slp[s+1]); slot
// slp[s] + 32 j + l holds block j of the row at position 32 s + l (row
// prow[32 s + l], or 32 s + l when prow is empty; column scol[slot], entry e
// at b*b (slp[s] + 32 j) + 32 e + l of a value array).
struct SolveMat {
  int nr = 0, nc = 0, nnzb = 0, b = 3;
  int ns = 0;      // slices
  long nslot = 0;  // slots, including padding
  const int *rowptr = nullptr, *col = nullptr;
  DBuf<int> slp, scol;
  DBuf<int> prow;  // position -> block row (rows sorted by length in windows); empty: identity
  DBuf<double> v64;
  DBuf<float> v32;
  DBuf<__nv_bfloat16> v16;
  int map = 0;    // warp mapping, FP32/bf16 storage (set by the autotuner)
  int map64 = 0;  // warp mapping, FP64 storage
  // one-warp-CTA mappings: partial row sums of the warps of a slice (ns x
  // WPS x 2B x 32 values of the vector type) and one arrival counter per
  // slice (zero between launches)
  int wps_rule = 1;
  DBuf<double> wpart;
  DBuf<unsigned> wtick;
  // batched product (k columns): mapping per storage (FP64, FP32, bf16) and
  // the k it was tuned for
  int bmap[3] = {1, 1, 1};
  int bmap_k[3] = {0, 0, 0};
};

// Row accumulator of the solve-phase block products.  FP64: every product is one FMA into the running sum.
// FP32: the 3 products of a block are fused into a block partial, which is
// added to the running sum with an error-free two-sum (Knuth), the rounding
// errors being collected in a second word.  Stiffness rows cancel strongly
// (K applied to a smooth vector), and an FP32 V-cycle whose residual
// y - A s carries the rounding of a plain 81-term FP32 sum preconditions
// visibly worse; the compensated sum costs a few FP32 additions, which this
// HBM-bound product has to spare.
template <typename TX> struct RowAcc;
template <> struct RowAcc<double> {
  double s[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void add(int r, double m0, double m1, double m2, double x0, double x1, double x2) {
    s[r] = fma(m0, x0, s[r]);
    s[r] = fma(m1, x1, s[r]);
    s[r] = fma(m2, x2, s[r]);
  }
  // scalar (1x1) block
  __device__ __forceinline__ void add1(int r, double m0, double x0) { s[r] = fma(m0, x0, s[r]); }
  __device__ __forceinline__ void merge(int r, double hi, double) { s[r] += hi; }
  __device__ __forceinline__ void set(int r, double hi, double) { s[r] = hi; }
  __device__ __forceinline__ double hi(int r) const { return s[r]; }
  __device__ __forceinline__ double lo(int) const { return 0.0; }
  __device__ __forceinline__ double get(int r) const { return s[r]; }
};
template <> struct RowAcc<float> {
  float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void two_sum(int r, float t) {
    const float a = s[r], u = __fadd_rn(a, t);
    const float bp = __fsub_rn(u, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(u, bp)), __fsub_rn(t, bp));
    s[r] = u;
    c[r] = __fadd_rn(c[r], err);
  }
  __device__ __forceinline__ void add(int r, float m0, float m1, float m2, float x0, float x1, float x2) {
    two_sum(r, fmaf(m2, x2, fmaf(m1, x1, __fmul_rn(m0, x0))));
  }
  // scalar (1x1) block: the product is the block partial
  __device__ __forceinline__ void add1(int r, float m0, float x0) { two_sum(r, __fmul_rn(m0, x0)); }
  __device__ __forceinline__ void merge(int r, float hi, float lo) {
    two_sum(r, hi);
    c[r] = __fadd_rn(c[r], lo);
  }
  __device__ __forceinline__ void set(int r, float hi, float lo) {
    s[r] = hi;
    c[r] = lo;
  }
  __device__ __forceinline__ float hi(int r) const { return s[r]; }
  __device__ __forceinline__ float lo(int r) const { return c[r]; }
  __device__ __forceinline__ float get(int r) const { return __fadd_rn(s[r], c[r]); }
};

// y = epilogue(A x): EP_SET y = Ax; EP_SCALE y = w Ax; EP_RESID y = aux - Ax;
// EP_SADD y = aux + w Ax; EP_ACC y += Ax.
enum { EP_SET = 0, EP_SCALE = 1, EP_RESID = 2, EP_SADD = 3, EP_ACC = 4 };
template <typename TM, typename TX>
void bsrmv(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w, const int *done,
           cudaStream_t s);
// y = epilogue(A x) on block rows [r0, r1) only, FP64 storage
void bsrmv_rows(int ep, const SolveMat &M, const double *x, double *y, const double *aux, double w, int r0, int r1,
                cudaStream_t s);
// one matrix's sliced layout to build, with the storage types it needs
struct SolveJob {
  const DevBsr *A;
  SolveMat *M;
  bool f64, f32, b16;
};
int make_solvemats(const std::vector<SolveJob> &jobs, cudaStream_t s);
int tune_solvemat(SolveMat &M, int kind, cudaStream_t s);  // kind 0 FP64, 1 FP32, 2 bf16
const char *mapping_name(const SolveMat &M, bool f64);
int mapping_wps(const SolveMat &M, bool f64);  // warps per slice of the chosen mapping
int bulk_copy_error();  // AMG_ERR_CUDA (and clears it) if a bulk-copy stage timed out

struct Level {
  int n = 0;  // nodes
  DevBsr A, G, GT, P, R;
  SolveMat sA, sG, sGT, sP, sR;
  double omega = 0.0, lmax = 0.0;
  int npasses = 0;
  int nc = 0;
  DBuf<int> cf;         // 1 = coarse, 0 = fine (levels that were coarsened)
  DBuf<double> V;       // test space, 3n x n_tv column-major
  // V-cycle work vectors (3n x kcap, node-major with the k columns interleaved)
  DBuf<double> y64, s64, r64, t64, z64;
  DBuf<float> y32, s32, r32, t32, z32;
};

struct Batch;  // batched-solve state (batch.cu)

struct Handle {
  amg_params prm{};
  cudaStream_t stream = nullptr;
  int dev = -1;  // device current at amg_setup
  int b = 3;     // block size: 3 (nodal blocks) or 1 (scalar, the paper's form)
  int n = 0;  // fine nodes (block rows)
  int nlev = 0;
  std::vector<std::unique_ptr<Level>> lev;
  // last level: explicit inverse of its matrix (dense, row-major, symmetric)
  int nL = 0;
  DBuf<double> Cinv;
  // PCG state (FP64), sized for kcap columns
  int kcap = 0;
  DBuf<double> x, r, z, p, q, zold, bvec, scal;
  DBuf<int> flags;
  DBuf<double> red;  // reduction partials
  amg_stats stats{};
  DBuf<double> V0keep;  // starting near-null space given to amg_setup
  int ntv0 = 0;
  // CUDA graph of one PCG iteration per (k) configuration
  cudaGraphExec_t graph_exec = nullptr;
  int graph_k = -1;
  int graph_prec = -1;
  bool own_stream = false;  // created because the caller passed the legacy stream
  long long graph_nodes = 0;
  int *pinned = nullptr;    // host flag for polling the PCG state
  Batch *batch = nullptr;   // k > 1 right-hand sides
  // second stream of the set-up: the Lanczos estimate of a level runs there
  // while the test space of the same level is generated
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_main = nullptr, ev_aux = nullptr;
  // fused coarse end of the V-cycle (vtail.cu): start level (-1: off), its
  // program, grid barrier words, a set "done" flag for the trial capture
  int vt_level = -1, vt_grid = 0;
  void *vt_func = nullptr;
  DBuf<unsigned char> vt_prog;
  DBuf<unsigned> vt_bar;
  DBuf<int> vt_flag;
  ~Handle();
};

// ---- set-up (setup.cu) ----
// keep_pattern: take the level-0 pattern the handle already holds (rowptr and
// col unused) and replace only the values
int build_hierarchy(Handle *h, const int *rowptr, const int *col, const double *vals, int mem,
                    int ntv0, const double *V0, int memV, bool keep_pattern = false);
void free_hierarchy(Handle *h);

// ---- solve (solve.cu) ----
int prepare_solve(Handle *h);
int solve(Handle *h, int k, const double *B, double *X, double rtol, int *iters, double *relres);
int vcycle_apply(Handle *h, const double *y, double *z);
int bench_spmv(Handle *h, int lev, int which, int a64, int reps, double *ms, double *bytes);
int vcycle_apply_noalloc(Handle *h, const double *y, double *z);
// ---- fused coarse end of the V-cycle (vtail.cu) ----
int vtail_prepare(Handle *h);
int vtail_run(Handle *h, const int *done, cudaStream_t s);
int vtail_error();  // AMG_ERR_CUDA (and clears it) if a grid barrier wait ran out
int bench_fsai(Handle *h, int lev, int reps, double *ms);
// ---- batched solve (batch.cu) ----
int solve_batched(Handle *h, int k, const double *B, double *X, double rtol, int *iters, double *relres);
void free_batch(Handle *h);
long long launch_count();

// ---- deterministic set-up kernels (det.cu) ----
namespace det {
int spmv(const DevBsr &A, const double *x, double *y, cudaStream_t s);
// Y_j = A X_j for the t columns of n x t column-major blocks (set-up order)
int spmv_cols(const DevBsr &A, int t, const double *X, double *Y, cudaStream_t s);
struct FsaiOut {
  int *np;        // [n] pattern nodes per row
  int *pat;       // [n*maxg]
  double *val;    // [n*(maxg+1)*9]
};
int fsai(const DevBsr &A, const DevBsr *Gs, int ksteps, int rho, double eps, int maxg, int maxdeg,
         FsaiOut out, int *status, cudaStream_t s);
int lanczos(const DevBsr &A, const DevBsr &G, const DevBsr &GT, int m, uint64_t seed, int level,
            double safety, double *d_out /*[lmax, omega_loop, omega]*/, cudaStream_t s, bool sync = true);
int srqcg(const DevBsr &A, const DevBsr &G, const DevBsr &GT, int kmax, int k_ritz, int t,
          const double *V0, double *V, int *status, cudaStream_t s);
int mgs(int n, int t, double *V, cudaStream_t s);
int soc_filter(const DevBsr &A, int t, const double *V, int theta, unsigned char *strong,
               cudaStream_t s);
int dpls(const DevBsr &A, const unsigned char *strong, const int *cf, const int *cidx,
         const int *fnodes, int nf, const int *cand_ptr, const int *cand, int t, const double *V,
         int n_max, double kappa_p, int *out_cnt, int *out_col, double *out_val, int *status,
         cudaStream_t s);
int spgemm_numeric(const DevBsr &X, const DevBsr &Y, DevBsr &Z, cudaStream_t s);
int gather_rows(const int *src_idx, int nrows_out, int n_in, int t, const double *Vin, double *Vout,
                cudaStream_t s);
int uniform_fill(double *v, int n, int col0, int ncols, uint64_t seed, cudaStream_t s);
}  // namespace det

// ---- integer pattern work on the GPU (graph.cu) ----
// out[i] = sum_{j<i} (in[j] + add), out[n] = total (launch only)
int dev_scan(int n, const int *in, int add, int *out, cudaStream_t s);
int read_int(const int *d, int *h, cudaStream_t s);  // blocking
int dev_row_max(int n, const int *rp, int *out, cudaStream_t s);
int transpose_bsr(const DevBsr &A, DevBsr &T, cudaStream_t s);
// Z = pattern of X Y (values of b x b blocks allocated, unset; b = 0: none)
int symbolic_product(const DevBsr &X, const DevBsr &Y, DevBsr &Z, int b, cudaStream_t s);
// coarse nodes within d_p strong edges of each fine node, ascending:
// cptr[0..nf] (device) and cand (allocated here)
int dpls_candidates_gpu(const DevBsr &A, const unsigned char *strong, const int *cf, const int *fnodes, int nf,
                        int d_p, int *cptr, DBuf<int> &cand, cudaStream_t s);

}  // namespace amg
