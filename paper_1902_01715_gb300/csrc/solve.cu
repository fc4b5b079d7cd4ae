// Solve phase: PCG preconditioned by one V(1,1)-cycle per iteration
// (Algorithm 2 with nu1 = nu2 = 1; post-smoothing with M^{-T} = M^{-1} since
// M^{-1} = omega G^T G is symmetric, Sec. 2), with the FP64 CG recurrence of
// Sec. 4 (x0 = 0, stop at ||r||_2 <= rtol ||b||_2).
//
// Every level matrix is stored in the sliced layout of spmv.cu (32 block
// rows per slice, one lane per row, coalesced entry loads).  One sparse
// kernel computes y = A x with a fused epilogue (plain, scaled, residual,
// scaled-add, accumulate), which covers the two smoother products, the
// residual, restriction and prolongation.  The V-cycle runs in FP64, FP32, or FP32 with bf16-stored
// G, G^T, P, R; the CG recurrence, its reductions and the coarse solve are
// FP64 in every mode.  One PCG iteration is captured in a CUDA graph; each
// kernel returns at once when the device-side `done` flag is set, so the
// host replays the graph and polls the flag.
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

int prepare_solve(Handle *h) {
  PdlScope plain(false);  // the timed mappings read the layout just built
  cudaStream_t s = h->stream;
  const int prec = h->prm.vcycle_prec;
  const bool f64 = prec == AMG_FP64, f32 = prec != AMG_FP64, b16 = prec == AMG_FP32_BF16GP;
  const int kv = f64 ? 0 : 1, kg = f64 ? 0 : (b16 ? 2 : 1);
  std::vector<SolveJob> jobs;
  for (int k = 0; k < h->nlev; ++k) {
    Level &L = *h->lev[k];
    // level 0 A is always kept in FP64 for the outer CG operator
    jobs.push_back({&L.A, &L.sA, f64 || k == 0, f32, false});
    if (k < h->nlev - 1) {
      jobs.push_back({&L.G, &L.sG, f64, f32 && !b16, b16});
      jobs.push_back({&L.GT, &L.sGT, f64, f32 && !b16, b16});
      jobs.push_back({&L.P, &L.sP, f64, f32 && !b16, b16});
      jobs.push_back({&L.R, &L.sR, f64, f32 && !b16, b16});
    }
  }
  AMG_TRY(make_solvemats(jobs, s));
  for (int k = 0; k < h->nlev; ++k) {
    Level &L = *h->lev[k];
    AMG_TRY(tune_solvemat(L.sA, kv, s));
    if (k == 0 && !f64) AMG_TRY(tune_solvemat(L.sA, 0, s));  // FP64 copy of the CG operator
    if (k < h->nlev - 1) {
      AMG_TRY(tune_solvemat(L.sG, kg, s));
      AMG_TRY(tune_solvemat(L.sGT, kg, s));
      AMG_TRY(tune_solvemat(L.sP, kg, s));
      AMG_TRY(tune_solvemat(L.sR, kg, s));
    }
    const size_t n3 = (size_t)h->b * L.n;
    if (f64) {
      AMG_TRY(L.y64.alloc(n3)); AMG_TRY(L.z64.alloc(n3));
      AMG_TRY(L.s64.alloc(n3)); AMG_TRY(L.r64.alloc(n3)); AMG_TRY(L.t64.alloc(n3));
    } else {
      AMG_TRY(L.y32.alloc(n3)); AMG_TRY(L.z32.alloc(n3));
      AMG_TRY(L.s32.alloc(n3)); AMG_TRY(L.r32.alloc(n3)); AMG_TRY(L.t32.alloc(n3));
    }
  }
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    h->graph_k = -1;
  }
  h->kcap = 0;  // PCG work buffers are sized by the coarse level: reallocate
  h->x.release();
  free_batch(h);
  AMG_CU(cudaStreamSynchronize(s));
  AMG_TRY(vtail_prepare(h));
  return AMG_OK;
}

// ---------------------------------------------------------------- coarse solve
// z = Cinv y with the explicit inverse of the last level (symmetric, so row i
// is also column i); one warp per row, FP64.
template <typename TX>
__global__ void k_coarse_mv(int m, const double *__restrict__ Ci, const TX *__restrict__ y, TX *__restrict__ z,
                            const int *__restrict__ done) {
  const int row = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double s = 0.0;
  const double *Cr = Ci + (size_t)row * m;
  // the loads of 16 terms are issued before their FMAs (same order of terms);
  // the first 16 entries of the row (set-up data) before the wait for the
  // preceding kernel
  constexpr int CU = 16;
  double a[CU];
#pragma unroll
  for (int u = 0; u < CU; ++u) a[u] = lane + 32 * u < m ? Cr[lane + 32 * u] : 0.0;
  pdl_wait();
  if (done && *done) return;
  for (int k0 = lane; k0 < m; k0 += 32 * CU) {
    double b[CU];
#pragma unroll
    for (int u = 0; u < CU; ++u) {
      const int k = k0 + 32 * u;
      if (k0 != lane) a[u] = k < m ? Cr[k] : 0.0;
      b[u] = k < m ? (double)y[k] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < CU; ++u)
      if (k0 + 32 * u < m) s = fma(a[u], b[u], s);
  }
  pdl_trigger();
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) z[row] = (TX)s;
}

// ---------------------------------------------------------------- V-cycle
template <typename TX> struct Vec;
template <> struct Vec<double> {
  static double *y(Level &L) { return L.y64.p; }
  static double *z(Level &L) { return L.z64.p; }
  static double *s(Level &L) { return L.s64.p; }
  static double *r(Level &L) { return L.r64.p; }
  static double *t(Level &L) { return L.t64.p; }
};
template <> struct Vec<float> {
  static float *y(Level &L) { return L.y32.p; }
  static float *z(Level &L) { return L.z32.p; }
  static float *s(Level &L) { return L.s32.p; }
  static float *r(Level &L) { return L.r32.p; }
  static float *t(Level &L) { return L.t32.p; }
};

template <typename TX>
static const TX *vals(const SolveMat &M, bool lowp);
template <>
const double *vals<double>(const SolveMat &M, bool) { return M.v64.p; }
template <>
const float *vals<float>(const SolveMat &M, bool) { return M.v32.p; }

template <typename TX>
static void mv(int ep, const SolveMat &M, bool b16, const TX *x, TX *y, const TX *aux, TX w, const int *done,
               cudaStream_t s) {
  if (b16) bsrmv<__nv_bfloat16, TX>(ep, M, M.v16.p, x, y, aux, w, done, s);
  else bsrmv<TX, TX>(ep, M, vals<TX>(M, false), x, y, aux, w, done, s);
}

template <>
void mv<double>(int ep, const SolveMat &M, bool, const double *x, double *y, const double *aux, double w,
                const int *done, cudaStream_t s) {
  bsrmv<double, double>(ep, M, M.v64.p, x, y, aux, w, done, s);
}

// z = B(y) on level k; y and z are the level's vectors (or the caller's at k=0)
template <typename TX>
static void vcycle_level(Handle *h, int k, const TX *y, TX *z, const int *done) {
  cudaStream_t st = h->stream;
  if (k > 0 && k == h->vt_level) {  // levels k.. in one persistent kernel (vtail.cu)
    vtail_run(h, done, st);
    return;
  }
  Level &L = *h->lev[k];
  const bool b16 = h->prm.vcycle_prec == AMG_FP32_BF16GP;
  if (k == h->nlev - 1) {
    const int m = h->nL;
    if (m == 0) return;
    launch_k(k_coarse_mv<TX>, nblk(32L * m, 256), 256, 0, st, m, (const double *)h->Cinv.p, y, z, done);
    return;
  }
  Level &C = *h->lev[k + 1];
  TX *s = Vec<TX>::s(L), *r = Vec<TX>::r(L), *t = Vec<TX>::t(L);
  const TX w = (TX)L.omega;
  mv<TX>(EP_SET, L.sG, b16, y, t, (const TX *)nullptr, w, done, st);       // t = G y
  mv<TX>(EP_SCALE, L.sGT, b16, t, s, (const TX *)nullptr, w, done, st);    // s = w G^T t
  mv<TX>(EP_RESID, L.sA, false, s, r, y, w, done, st);                    // r = y - A s
  mv<TX>(EP_SET, L.sR, b16, r, Vec<TX>::y(C), (const TX *)nullptr, w, done, st);  // y_c = P^T r
  vcycle_level<TX>(h, k + 1, Vec<TX>::y(C), Vec<TX>::z(C), done);
  mv<TX>(EP_ACC, L.sP, b16, Vec<TX>::z(C), s, (const TX *)nullptr, w, done, st);  // s += P z_c
  mv<TX>(EP_RESID, L.sA, false, s, r, y, w, done, st);                    // r = y - A s
  mv<TX>(EP_SET, L.sG, b16, r, t, (const TX *)nullptr, w, done, st);       // t = G r
  mv<TX>(EP_SADD, L.sGT, b16, t, z, s, w, done, st);                       // z = s + w G^T t
}

// ---------------------------------------------------------------- PCG
// scalar slots (doubles) and flags (ints) on the device
enum { P_BN2 = 0, P_RZ, P_PQ, P_ALPHA, P_RR, P_RZN, P_RZO, P_BETA, P_TOL2, P_TRR, P_TRRP, P_NSC };
enum { F_DONE = 0, F_ITERS, F_STATUS, F_MAXIT, F_TICKET, F_NFL };

constexpr int RED_BLOCKS = 296;
// true-residual restarts of one solve (each one V-cycle and one FP64 product more)
constexpr int kMaxRestarts = 8;
constexpr int RED_THREADS = 256;
// elements per thread and pass of the PCG vector kernels, their loads issued
// first (the same elements in the same order as one at a time: same sums)
constexpr int VUNR = 4;

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  }
  return t;  // valid in thread 0
}

// Deterministic two-level reduction: block partials, then the last block to
// finish sums them in block order and runs `fin` on thread 0.
template <class Fin>
__device__ __forceinline__ void finish_reduce(double v, double *part, int *flags, double *sh, Fin fin) {
  const double bs = block_sum(v, sh);
  __shared__ int last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(&flags[F_TICKET], 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += ((volatile double *)part)[b];
  const double tot = block_sum(t, sh);
  if (threadIdx.x == 0) {
    flags[F_TICKET] = 0;
    fin(tot);
  }
}

// pq = p.q ; alpha = rz / pq
__global__ void __launch_bounds__(RED_THREADS) k_pcg_pq(long n, const double *__restrict__ p, const double *__restrict__ q,
                                                        double *sc, int *flags, double *part) {
  pdl_wait();
  if (flags[F_DONE]) return;
  __shared__ double sh[32];
  double v = 0.0;
  const long S = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VUNR * S) {
    double pv[VUNR], qv[VUNR];
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      pv[u] = i < n ? p[i] : 0.0;
      qv[u] = i < n ? q[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < VUNR; ++u)
      if (i0 + u * S < n) v += pv[u] * qv[u];
  }
  pdl_trigger();
  finish_reduce(v, part, flags, sh, [&](double tot) {
    sc[P_PQ] = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      flags[F_STATUS] = AMG_ERR_BREAKDOWN;
      flags[F_DONE] = 1;
    } else {
      sc[P_ALPHA] = sc[P_RZ] / tot;
    }
  });
}

// x += alpha p ; r -= alpha q ; rr = r.r ; convergence ; rlow = (TX) r
template <typename TX>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_xr(long n, double *__restrict__ x, double *__restrict__ r,
                                                        const double *__restrict__ p, const double *__restrict__ q,
                                                        TX *__restrict__ rlow, double *sc, int *flags, double *part) {
  pdl_wait();
  if (flags[F_DONE]) return;
  __shared__ double sh[32];
  const double a = sc[P_ALPHA];
  double v = 0.0;
  const long S = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VUNR * S) {
    double xv[VUNR], rv[VUNR], pv[VUNR], qv[VUNR];
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      const bool in = i < n;
      xv[u] = in ? x[i] : 0.0;
      rv[u] = in ? r[i] : 0.0;
      pv[u] = in ? p[i] : 0.0;
      qv[u] = in ? q[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      if (i >= n) break;
      x[i] = xv[u] + a * pv[u];
      const double ri = rv[u] - a * qv[u];
      r[i] = ri;
      if (rlow) rlow[i] = (TX)ri;
      v += ri * ri;
    }
  }
  pdl_trigger();
  finish_reduce(v, part, flags, sh, [&](double tot) {
    sc[P_RR] = tot;
    const int it = flags[F_ITERS] + 1;
    flags[F_ITERS] = it;
    if (!isfinite(tot)) {
      flags[F_STATUS] = AMG_ERR_BREAKDOWN;
      flags[F_DONE] = 1;
    } else if (tot <= sc[P_TOL2]) {
      flags[F_DONE] = 1;
    } else if (it >= flags[F_MAXIT]) {
      flags[F_STATUS] = AMG_ERR_NOT_CONVERGED;
      flags[F_DONE] = 1;
    }
  });
}

// z = (double) zlow (mixed modes); rz = r.z and, for flexible CG, r.z_old;
// beta = (rz - r.z_old) / rz_prev (flexible) or rz / rz_prev.
template <typename TX>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_rz(long n, const double *__restrict__ r, double *__restrict__ z,
                                                        const TX *__restrict__ zlow, const double *__restrict__ zold,
                                                        int flexible, double *sc, int *flags, double *part,
                                                        double *part2) {
  pdl_wait();
  if (flags[F_DONE]) return;
  __shared__ double sh[32];
  double v = 0.0, v2 = 0.0;
  const long S = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VUNR * S) {
    double zv[VUNR], rv[VUNR], ov[VUNR];
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      const bool in = i < n;
      zv[u] = in ? (zlow ? (double)zlow[i] : z[i]) : 0.0;
      rv[u] = in ? r[i] : 0.0;
      ov[u] = in && flexible ? zold[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      if (i >= n) break;
      if (zlow) z[i] = zv[u];
      v += rv[u] * zv[u];
      if (flexible) v2 += rv[u] * ov[u];
    }
  }
  const double b2 = flexible ? block_sum(v2, sh) : 0.0;
  if (flexible && threadIdx.x == 0) part2[blockIdx.x] = b2;
  __syncthreads();
  pdl_trigger();
  finish_reduce(v, part, flags, sh, [&](double tot) {
    double rzo = 0.0;
    if (flexible)
      for (int b = 0; b < (int)gridDim.x; ++b) rzo += ((volatile double *)part2)[b];
    const double prev = sc[P_RZ];
    sc[P_BETA] = flexible ? (tot - rzo) / prev : tot / prev;
    sc[P_RZ] = tot;
    if (!isfinite(sc[P_BETA])) {
      flags[F_STATUS] = AMG_ERR_BREAKDOWN;
      flags[F_DONE] = 1;
    }
  });
}

__global__ void k_pcg_p(long n, double *__restrict__ p, const double *__restrict__ z, double *__restrict__ zold,
                        int flexible, const double *sc, const int *flags) {
  pdl_wait();
  if (flags[F_DONE]) return;
  const double b = sc[P_BETA];
  const long S = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += VUNR * S) {
    double zv[VUNR], pv[VUNR];
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      zv[u] = i < n ? z[i] : 0.0;
      pv[u] = i < n ? p[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < VUNR; ++u) {
      const long i = i0 + u * S;
      if (i >= n) break;
      p[i] = zv[u] + b * pv[u];
      if (flexible) zold[i] = zv[u];
    }
  }
}

// start: x = 0, r = b, rlow = (TX) b, bn2 = b.b, tol2 = rtol^2 bn2
template <typename TX>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_start(long n, const double *__restrict__ b, double *__restrict__ x,
                                                           double *__restrict__ r, TX *__restrict__ rlow, double rtol,
                                                           double *sc, int *flags, double *part) {
  pdl_wait();
  __shared__ double sh[32];
  double v = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = 0.0;
    r[i] = b[i];
    if (rlow) rlow[i] = (TX)b[i];
    v += b[i] * b[i];
  }
  pdl_trigger();
  finish_reduce(v, part, flags, sh, [&](double tot) {
    sc[P_BN2] = tot;
    sc[P_TOL2] = (rtol * rtol) * tot;
    sc[P_RR] = tot;
    sc[P_RZ] = 1.0;
    if (!isfinite(tot)) {
      flags[F_STATUS] = AMG_ERR_BREAKDOWN;
      flags[F_DONE] = 1;
    } else if (tot == 0.0) {
      flags[F_DONE] = 1;
    }
  });
}

// first direction: p = z, z_old = z, rz = r.z
__global__ void k_pcg_first_p(long n, double *__restrict__ p, const double *__restrict__ z, double *__restrict__ zold,
                              const int *flags) {
  pdl_wait();
  if (flags[F_DONE]) return;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    p[i] = z[i];
    zold[i] = z[i];
  }
}

// True residual after the recurrence stopped: r already holds b - K x (FP64
// level-0 K); trr = r.r.  When the column stopped as converged but
// ||b - K x||^2 > rtol^2 ||b||^2, the recurrence restarts from the true
// residual (done is cleared, so the V-cycle and first-direction kernels that
// follow run; rlow receives (TX) r for the V-cycle; the iteration count
// carries on) -- unless this is restart number kMaxRestarts, the iteration
// limit is reached, or the previous restart did not halve the true residual
// (rtol is then below the accuracy FP64 attains on this system).  The status
// stays that of the recurrence rule (Sec. 4); the true residual is reported.
template <typename TX>
__global__ void __launch_bounds__(RED_THREADS) k_pcg_true(long n, const double *__restrict__ r, TX *__restrict__ rlow,
                                                          int phase, int max_phase, double *sc, int *flags,
                                                          double *part) {
  pdl_wait();
  __shared__ double sh[32];
  double v = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double ri = r[i];
    if (rlow) rlow[i] = (TX)ri;
    v += ri * ri;
  }
  pdl_trigger();
  finish_reduce(v, part, flags, sh, [&](double tot) {
    const double prev = sc[P_TRRP];
    sc[P_TRR] = tot;
    sc[P_TRRP] = tot;
    if (!isfinite(tot)) {
      if (flags[F_STATUS] == 0) flags[F_STATUS] = AMG_ERR_BREAKDOWN;
    } else if (flags[F_STATUS] == 0 && tot > sc[P_TOL2] && phase < max_phase && flags[F_ITERS] < flags[F_MAXIT] &&
               !(phase > 0 && tot > 0.25 * prev)) {
      sc[P_RR] = tot;
      flags[F_DONE] = 0;
    }
  });
}

__global__ void k_set_flags(int *flags, int maxit) {
  flags[F_DONE] = 0;
  flags[F_ITERS] = 0;
  flags[F_STATUS] = 0;
  flags[F_MAXIT] = maxit;
  flags[F_TICKET] = 0;
}

static int ensure_pcg(Handle *h) {
  if (h->kcap >= 1 && h->x.p) return AMG_OK;
  const size_t n3 = (size_t)h->b * h->n;
  AMG_TRY(h->x.alloc(n3));
  AMG_TRY(h->r.alloc(n3));
  AMG_TRY(h->z.alloc(n3));
  AMG_TRY(h->p.alloc(n3));
  AMG_TRY(h->q.alloc(n3));
  AMG_TRY(h->zold.alloc(n3));
  AMG_TRY(h->bvec.alloc(n3));
  AMG_TRY(h->scal.alloc(P_NSC + 8));
  AMG_TRY(h->flags.alloc(F_NFL + 4));
  AMG_TRY(h->red.alloc(4 * RED_BLOCKS + 16));
  if (!h->pinned) AMG_CU(cudaMallocHost((void **)&h->pinned, 4 * sizeof(int)));
  h->kcap = 1;
  return AMG_OK;
}

template <typename TX>
static TX *low_r(Handle *h) { return Vec<TX>::y(*h->lev[0]); }
template <typename TX>
static TX *low_z(Handle *h) { return Vec<TX>::z(*h->lev[0]); }

// one PCG iteration (graph body)
template <typename TX>
static void pcg_iteration(Handle *h, bool mixed) {
  cudaStream_t s = h->stream;
  Level &L0 = *h->lev[0];
  const long n = (long)h->b * h->n;
  double *part = h->red.p, *part2 = h->red.p + 2 * RED_BLOCKS;
  int *fl = h->flags.p;
  double *sc = h->scal.p;
  const int *done = fl + F_DONE;
  bsrmv<double, double>(EP_SET, L0.sA, L0.sA.v64.p, h->p.p, h->q.p, nullptr, 0.0, done, s);
  launch_k(k_pcg_pq, RED_BLOCKS, RED_THREADS, 0, s, n, h->p.p, h->q.p, sc, fl, part);
  if (mixed) {
    launch_k(k_pcg_xr<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, h->x.p, h->r.p, h->p.p, h->q.p, low_r<TX>(h), sc, fl, part);
    vcycle_level<TX>(h, 0, low_r<TX>(h), low_z<TX>(h), done);
    launch_k(k_pcg_rz<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, h->r.p, h->z.p, low_z<TX>(h), h->zold.p, 1, sc, fl, part,
                                                     part2);
    launch_k(k_pcg_p, RED_BLOCKS, RED_THREADS, 0, s, n, h->p.p, h->z.p, h->zold.p, 1, sc, fl);
  } else {
    launch_k(k_pcg_xr<double>, RED_BLOCKS, RED_THREADS, 0, s, n, h->x.p, h->r.p, h->p.p, h->q.p, (double *)nullptr, sc, fl,
                                                         part);
    vcycle_level<double>(h, 0, h->r.p, h->z.p, done);
    launch_k(k_pcg_rz<double>, RED_BLOCKS, RED_THREADS, 0, s, n, h->r.p, h->z.p, (const double *)nullptr, h->zold.p, 0, sc,
                                                         fl, part, part2);
    launch_k(k_pcg_p, RED_BLOCKS, RED_THREADS, 0, s, n, h->p.p, h->z.p, h->zold.p, 0, sc, fl);
  }
}

template <typename TX>
static int pcg_solve_one(Handle *h, const double *b, double *x, double rtol, int *iters, double *relres,
                         double *rec_relres, int *nrestart, bool mixed) {
  PdlScope pdl;
  cudaStream_t s = h->stream;
  const long n = (long)h->b * h->n;
  double *part = h->red.p;
  int *fl = h->flags.p;
  double *sc = h->scal.p;
  AMG_KCOUNT k_set_flags<<<1, 1, 0, s>>>(fl, h->prm.maxit);
  launch_k(k_pcg_start<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, b, h->x.p, h->r.p, mixed ? low_r<TX>(h) : (TX *)nullptr, rtol,
                                                      sc, fl, part);
  if (mixed) {
    vcycle_level<TX>(h, 0, low_r<TX>(h), low_z<TX>(h), fl + F_DONE);
  } else {
    vcycle_level<double>(h, 0, h->r.p, h->z.p, fl + F_DONE);
  }
  // rz = r.z (beta unused)
  launch_k(k_pcg_rz<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, h->r.p, h->z.p, mixed ? low_z<TX>(h) : (const TX *)nullptr,
                                                   h->zold.p, 0, sc, fl, part, part + 2 * RED_BLOCKS);
  launch_k(k_pcg_first_p, RED_BLOCKS, RED_THREADS, 0, s, n, h->p.p, h->z.p, h->zold.p, fl);
  AMG_LAUNCH_CHECK();
  const int key = mixed ? 1 : 0;
  if (!h->graph_exec || h->graph_k != 1 || h->graph_prec != key) {
    if (h->graph_exec) {
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    cudaGraph_t g;
    const long long before = launch_count();
    AMG_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    pcg_iteration<TX>(h, mixed);
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    // captured launches run only when the graph is replayed
    h->graph_nodes = launch_count() - before;
    count_launches(-h->graph_nodes);
    if (ce != cudaSuccess) {
      set_error("graph capture failed: %s", cudaGetErrorString(ce));
      return AMG_ERR_CUDA;
    }
    AMG_CU(cudaGraphInstantiate(&h->graph_exec, g, 0));
    cudaGraphDestroy(g);
    h->graph_k = 1;
    h->graph_prec = key;
  }
  int hflags[F_NFL];
  int *pinned = h->pinned;
  Level &L0 = *h->lev[0];
  int restarts = 0;
  // Phases: replay the iteration graph until the device flag says the
  // recurrence stopped (the host checks it every `chunk` launches), then form
  // the FP64 true residual b - K x; if it is above rtol ||b|| the recurrence
  // restarts from it (see k_pcg_true for the limits).
  const int chunk = 4;
  for (;;) {
    for (int it = 0; it < h->prm.maxit + chunk; it += chunk) {
      for (int c = 0; c < chunk; ++c) {
        cudaError_t e = cudaGraphLaunch(h->graph_exec, s);
        if (e != cudaSuccess) {
          set_error("cudaGraphLaunch: %s", cudaGetErrorString(e));
          return AMG_ERR_CUDA;
        }
        count_launches(h->graph_nodes);
      }
      AMG_CU(cudaMemcpyAsync(pinned, fl, sizeof(int), cudaMemcpyDeviceToHost, s));
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error("PCG: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
      }
      if (pinned[0]) break;
    }
    // r = b - K x with the FP64 level-0 K, its norm, and the restart decision
    bsrmv<double, double>(EP_RESID, L0.sA, L0.sA.v64.p, h->x.p, h->r.p, b, 0.0, nullptr, s);
    launch_k(k_pcg_true<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, h->r.p, mixed ? low_r<TX>(h) : (TX *)nullptr,
                                                                restarts, kMaxRestarts, sc, fl, part);
    // restart (all done-gated: nothing runs unless k_pcg_true cleared done)
    if (mixed) vcycle_level<TX>(h, 0, low_r<TX>(h), low_z<TX>(h), fl + F_DONE);
    else vcycle_level<double>(h, 0, h->r.p, h->z.p, fl + F_DONE);
    launch_k(k_pcg_rz<TX>, RED_BLOCKS, RED_THREADS, 0, s, n, h->r.p, h->z.p, mixed ? low_z<TX>(h) : (const TX *)nullptr,
                                                     h->zold.p, 0, sc, fl, part, part + 2 * RED_BLOCKS);
    launch_k(k_pcg_first_p, RED_BLOCKS, RED_THREADS, 0, s, n, h->p.p, h->z.p, h->zold.p, fl);
    AMG_LAUNCH_CHECK();
    AMG_CU(cudaMemcpyAsync(pinned, fl, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
    if (pinned[0]) break;
    ++restarts;
  }
  double hsc[P_NSC];
  AMG_CU(cudaMemcpy(hflags, fl, sizeof hflags, cudaMemcpyDeviceToHost));
  AMG_CU(cudaMemcpy(hsc, sc, sizeof hsc, cudaMemcpyDeviceToHost));
  AMG_CU(cudaMemcpyAsync(x, h->x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  AMG_CU(cudaStreamSynchronize(s));
  *iters = hflags[F_ITERS];
  *relres = hsc[P_BN2] > 0.0 ? std::sqrt(hsc[P_TRR] / hsc[P_BN2]) : 0.0;
  *rec_relres = hsc[P_BN2] > 0.0 ? std::sqrt(hsc[P_RR] / hsc[P_BN2]) : 0.0;
  *nrestart = restarts;
  if (mixed) AMG_TRY(bulk_copy_error());
  if (h->vt_level >= 0) AMG_TRY(vtail_error());
  return hflags[F_STATUS];
}

int solve(Handle *h, int k, const double *B, double *X, double rtol, int *iters, double *relres) {
  if (k > 1) return solve_batched(h, k, B, X, rtol, iters, relres);
  AMG_TRY(ensure_pcg(h));
  const long n = (long)h->b * h->n;
  const bool mixed = h->prm.vcycle_prec != AMG_FP64;
  int worst = AMG_OK, maxit = 0, nrs = 0;
  double rec_max = 0.0, true_max = 0.0;
  for (int j = 0; j < k; ++j) {
    int it = 0, rs = 0;
    double rr = 0.0, rec = 0.0;
    const int rc = mixed ? pcg_solve_one<float>(h, B + (size_t)j * n, X + (size_t)j * n, rtol, &it, &rr, &rec, &rs, true)
                         : pcg_solve_one<double>(h, B + (size_t)j * n, X + (size_t)j * n, rtol, &it, &rr, &rec, &rs, false);
    if (rc == AMG_ERR_CUDA) return rc;
    if (rc && !worst) worst = rc;
    iters[j] = it;
    relres[j] = rr;
    maxit = it > maxit ? it : maxit;
    rec_max = rec > rec_max ? rec : rec_max;
    true_max = rr > true_max ? rr : true_max;
    nrs += rs;
  }
  h->stats.n_it = maxit;
  h->stats.relres_rec = rec_max;
  h->stats.relres_true = true_max;
  h->stats.restarts = nrs;
  return worst;
}

__global__ void k_d2f(long n, const double *__restrict__ a, float *__restrict__ b) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_f2d(long n, const float *__restrict__ a, double *__restrict__ b) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

int vcycle_apply(Handle *h, const double *y, double *z) {
  AMG_TRY(ensure_pcg(h));
  PdlScope pdl;
  cudaStream_t s = h->stream;
  const long n = (long)h->b * h->n;
  AMG_KCOUNT k_set_flags<<<1, 1, 0, s>>>(h->flags.p, 1);
  if (h->prm.vcycle_prec == AMG_FP64) {
    vcycle_level<double>(h, 0, y, z, h->flags.p + F_DONE);
  } else {
    AMG_KCOUNT k_d2f<<<nblk(n, 256), 256, 0, s>>>(n, y, low_r<float>(h));
    vcycle_level<float>(h, 0, low_r<float>(h), low_z<float>(h), h->flags.p + F_DONE);
    AMG_KCOUNT k_f2d<<<nblk(n, 256), 256, 0, s>>>(n, low_z<float>(h), z);
  }
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  // a bulk-copy stage or a fused-kernel barrier that timed out left rows of z unwritten
  if (h->prm.vcycle_prec != AMG_FP64) AMG_TRY(bulk_copy_error());
  if (h->vt_level >= 0) AMG_TRY(vtail_error());
  return AMG_OK;
}

// ---------------------------------------------------------------- V-cycle without allocation
// Scratch of amg_vcycle_noalloc: a state flag block of 256 bytes.  It is a
// file-scope device array, so every GPU that loads the library holds it
// until the process exits, and every call shares it.
constexpr int VC_STATIC_FLAG_BYTES = 256;
static __device__ __align__(256) unsigned char g_vc_scratch[VC_STATIC_FLAG_BYTES];

// Device address of g_vc_scratch for each device, looked up once per device
// (with that device current) on the first call there.
static void *g_vc_scratch_addr[64] = {nullptr};
static std::mutex g_vc_scratch_mu;

static int vc_scratch_address(void **out) {
  int dev = 0;
  AMG_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("amg_vcycle_noalloc: device ordinal %d beyond the supported 64", dev);
    return AMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_vc_scratch_mu);
  if (!g_vc_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("amg_vcycle_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return AMG_ERR_CUDA;
    }
    g_vc_scratch_addr[dev] = p;
  }
  *out = g_vc_scratch_addr[dev];
  return AMG_OK;
}

int vcycle_apply_noalloc(Handle *h, const double *y, double *z) {
  // the scratch address is per device: it must be the device of the handle
  int cur = -1;
  AMG_CU(cudaGetDevice(&cur));
  if (cur != h->dev) {
    set_error("amg_vcycle_noalloc: current device %d is not the handle's device %d", cur, h->dev);
    return AMG_ERR_ARG;
  }
  void *base = nullptr;
  AMG_TRY(vc_scratch_address(&base));
  PdlScope pdl;
  int *flags = (int *)base;
  cudaStream_t s = h->stream;
  const long n = (long)h->b * h->n;
  // the flag block keeps the previous call's contents: reset it first
  AMG_KCOUNT k_set_flags<<<1, 1, 0, s>>>(flags, 1);
  if (h->prm.vcycle_prec == AMG_FP64) {
    vcycle_level<double>(h, 0, y, z, flags + F_DONE);
  } else {
    AMG_KCOUNT k_d2f<<<nblk(n, 256), 256, 0, s>>>(n, y, low_r<float>(h));
    vcycle_level<float>(h, 0, low_r<float>(h), low_z<float>(h), flags + F_DONE);
    AMG_KCOUNT k_f2d<<<nblk(n, 256), 256, 0, s>>>(n, low_z<float>(h), z);
  }
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  // a bulk-copy stage or a fused-kernel barrier that timed out left rows of z
  // unwritten (the error words are read and cleared with plain symbol copies:
  // no allocation)
  if (h->prm.vcycle_prec != AMG_FP64) AMG_TRY(bulk_copy_error());
  if (h->vt_level >= 0) AMG_TRY(vtail_error());
  return AMG_OK;
}

// Average time of one solve-phase sparse product of a level matrix, launched
// back to back on the handle's stream between CUDA events.
int bench_spmv(Handle *h, int lev, int which, int a64, int reps, double *ms, double *bytes) {
  if (lev < 0 || lev >= h->nlev || which < 0 || which > 6 || reps < 1) return AMG_ERR_ARG;
  Level &L = *h->lev[lev];
  if (which == 6) {  // the set-up's first aFSAI pass on A_lev
    if (lev == h->nlev - 1) return AMG_ERR_ARG;
    *bytes = 0.0;
    return bench_fsai(h, lev, reps, ms);
  }
  if (which == 5) {  // the set-up's FP64 product of A_k with the n_tv test-space columns
    const int t = h->prm.n_tv;
    const size_t n = (size_t)L.A.b * L.A.nr;
    if (L.A.nr == 0) return AMG_ERR_ARG;
    cudaStream_t s = h->stream;
    DBuf<double> X, Y;
    AMG_TRY(X.alloc(n * t));
    AMG_TRY(Y.alloc(n * t));
    AMG_TRY(X.zero(s));
    cudaEvent_t e0, e1;
    AMG_CU(cudaEventCreate(&e0));
    AMG_CU(cudaEventCreate(&e1));
    AMG_TRY(det::spmv_cols(L.A, t, X.p, Y.p, s));
    AMG_CU(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) AMG_TRY(det::spmv_cols(L.A, t, X.p, Y.p, s));
    AMG_CU(cudaEventRecord(e1, s));
    AMG_CU(cudaEventSynchronize(e1));
    float tm = 0.f;
    AMG_CU(cudaEventElapsedTime(&tm, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)tm / reps;
    *bytes = (double)L.A.nnzb * (L.A.b * L.A.b * 8.0 + 4.0) + 4.0 * (L.A.nr + 1) + 8.0 * t * (2.0 * n);
    return AMG_OK;
  }
  SolveMat *M = which == 0 ? &L.sA : which == 1 ? &L.sG : which == 2 ? &L.sGT : which == 3 ? &L.sP : &L.sR;
  if (M->nr == 0) return AMG_ERR_ARG;
  cudaStream_t s = h->stream;
  const int prec = h->prm.vcycle_prec;
  const bool dbl = (prec == AMG_FP64) || (which == 0 && a64 && M->v64.p);
  const bool b16 = !dbl && prec == AMG_FP32_BF16GP && which != 0;
  const size_t nx = (size_t)M->b * M->nc, ny = (size_t)M->b * M->nr;
  const size_t xs = dbl ? 8 : 4, vs = dbl ? 8 : (b16 ? 2 : 4);
  DBuf<double> x64, y64;
  DBuf<float> x32, y32;
  cudaEvent_t e0, e1;
  AMG_CU(cudaEventCreate(&e0));
  AMG_CU(cudaEventCreate(&e1));
  if (dbl) {
    AMG_TRY(x64.alloc(nx));
    AMG_TRY(y64.alloc(ny));
    AMG_TRY(x64.zero(s));
  } else {
    AMG_TRY(x32.alloc(nx));
    AMG_TRY(y32.alloc(ny));
    AMG_TRY(x32.zero(s));
  }
  auto launch = [&]() {
    if (dbl) bsrmv<double, double>(EP_SET, *M, M->v64.p, x64.p, y64.p, nullptr, 0.0, nullptr, s);
    else if (b16) bsrmv<__nv_bfloat16, float>(EP_SET, *M, M->v16.p, x32.p, y32.p, nullptr, 0.f, nullptr, s);
    else bsrmv<float, float>(EP_SET, *M, M->v32.p, x32.p, y32.p, nullptr, 0.f, nullptr, s);
  };
  launch();
  AMG_CU(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) launch();
  AMG_CU(cudaEventRecord(e1, s));
  AMG_CU(cudaEventSynchronize(e1));
  float t = 0.f;
  AMG_CU(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  AMG_LAUNCH_CHECK();
  *ms = (double)t / reps;
  *bytes = (double)M->nnzb * (M->b * M->b * vs + 4.0) + 4.0 * (M->nr + 1) + (double)xs * (nx + ny);
  return AMG_OK;
}

Handle::~Handle() {
  free_batch(this);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (pinned) cudaFreeHost(pinned);
  lev.clear();
  // buffers are returned on the stream they were taken on: before it goes
  for (DBuf<double> *b : {&Cinv, &x, &r, &z, &p, &q, &zold, &bvec, &scal, &red, &V0keep}) b->release();
  flags.release();
  vt_prog.release();
  vt_bar.release();
  vt_flag.release();
  if (aux) cudaStreamDestroy(aux);
  if (ev_main) cudaEventDestroy(ev_main);
  if (ev_aux) cudaEventDestroy(ev_aux);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

}  // namespace amg

// One V-cycle z = B(y) that allocates no memory: for callers that cannot
// allocate while they run it, e.g. an outer Krylov solver of another code
// whose process keeps all device memory in its own pool (where a device
// allocation inside the call would fail or fragment that pool), or one that must keep
// every allocation out of its iteration loop.  Its scratch is the file-scope
// array above; see include/aspamg.h for the limits.
extern "C" int amg_vcycle_noalloc(amg_handle hh, const double *y, double *z) {
  amg::Handle *h = (amg::Handle *)hh;
  if (!h || !y || !z) return AMG_ERR_ARG;
  return amg::vcycle_apply_noalloc(h, y, z);
}
