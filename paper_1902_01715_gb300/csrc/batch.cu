// Batched solve: k right-hand sides at once (block PCG with one V-cycle per
// iteration and per-column convergence masks).  Vectors are stored
// "interleaved" — entry (dof d, column c) at d*k + c — so one warp walks a
// block row once and applies each 3x3 block (read once, broadcast to the
// lanes) to all k columns with coalesced loads of the neighbour's 3 x k
// values.  Each column runs its own CG recurrence (alpha, beta, residual,
// convergence) in FP64; a converged column is frozen (its x, r, p no longer
// change) while the V-cycle keeps processing the whole block.  Reductions
// are deterministic (per-column partials per block, summed in block order by
// the last block).
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ double cvb(double v, double) { return v; }
__device__ __forceinline__ float cvb(float v, float) { return v; }
__device__ __forceinline__ float cvb(__nv_bfloat16 v, float) { return __bfloat162float(v); }

enum { BE_SET = 0, BE_SCALE = 1, BE_RESID = 2, BE_SADD = 3, BE_ACC = 4 };

// Y = epilogue(A X) on interleaved n x k blocks of the sliced layout.
// Mapping (L, NC): a warp holds 32 / L lane groups of L lanes, one block row
// per group; lane l of a group handles columns c0 + l + i L (i < NC) of each
// tile of L NC columns, reading the row's blocks once per tile (every lane of
// the group reads the same block: a broadcast) and its columns of the
// neighbours' B x k values with coalesced loads.  Every (row, column) sum
// adds the row's blocks in the same order whatever the mapping, so the
// mapping changes the time, not the result.
template <typename TM, typename TX, int B, int EP, int L, int NC>
__global__ void __launch_bounds__(256) k_bsrmm(int nr, int k, const int *__restrict__ prow, const int *__restrict__ rp,
                                               const int *__restrict__ slp,
                                               const int *__restrict__ scol, const TM *__restrict__ v,
                                               const TX *__restrict__ X, TX *__restrict__ Y,
                                               const TX *__restrict__ AUX, TX w, const int *__restrict__ done) {
  if (done && *done) return;
  constexpr int R = 32 / L, BB = B * B;
  const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, gl = lane % L;
  const long posl = gw * R + lane / L;  // position in the sliced layout
  if (posl >= nr) return;
  const int pos = (int)posl, rl = pos & 31;
  const int row = prow ? prow[pos] : pos;
  const int len = rp[row + 1] - rp[row];
  const long sbase = slp[pos >> 5];
  for (int c0 = 0; c0 < k; c0 += L * NC) {
    RowAcc<TX> acc[NC];
    for (int q = 0; q < len; ++q) {
      const long slot = sbase + 32L * q;
      const long j = scol[slot + rl];
      const TM *mp = v + BB * slot + rl;
      TX m[BB];
#pragma unroll
      for (int e = 0; e < BB; ++e) m[e] = cvb(mp[32 * e], TX(0));
      const TX *xj = X + (long)B * j * k;
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        const int c = c0 + gl + i * L;
        if (c < k) {
          if constexpr (B == 3) {
            const TX x0 = xj[c], x1 = xj[k + c], x2 = xj[2 * k + c];
            acc[i].add(0, m[0], m[1], m[2], x0, x1, x2);
            acc[i].add(1, m[3], m[4], m[5], x0, x1, x2);
            acc[i].add(2, m[6], m[7], m[8], x0, x1, x2);
          } else {
            acc[i].add1(0, m[0], xj[c]);
          }
        }
      }
    }
    const long o = (long)B * row * k;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int c = c0 + gl + i * L;
      if (c >= k) continue;
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const long at = o + (long)r * k + c;
        const TX a = acc[i].get(r);
        if (EP == BE_SET) Y[at] = a;
        if (EP == BE_SCALE) Y[at] = w * a;
        if (EP == BE_RESID) Y[at] = AUX[at] - a;
        if (EP == BE_SADD) Y[at] = AUX[at] + w * a;
        if (EP == BE_ACC) Y[at] += a;
      }
    }
  }
}

// candidate mappings (lanes per row, columns per lane and tile)
struct BMap {
  int L, NC;
};
static const BMap kBMaps[] = {{32, 1}, {32, 2}, {16, 2}, {16, 4}, {8, 4}};
constexpr int kNumBMaps = (int)(sizeof(kBMaps) / sizeof(kBMaps[0]));

template <typename TM, typename TX, int B, int L, int NC>
static void bmm_launch(int ep, const SolveMat &M, const TM *v, int k, const TX *X, TX *Y, const TX *AUX, TX w,
                       const int *done, cudaStream_t s) {
  constexpr int R = 32 / L;
  const long warps = (M.nr + R - 1) / R;
  const int nb = nblk(32L * warps, 256);
  if (!nb) return;
#define AMG_BMM_ARGS M.nr, k, M.prow.p, M.rowptr, M.slp.p, M.scol.p, v, X, Y, AUX, w, done
  switch (ep) {
    case BE_SET: AMG_KCOUNT k_bsrmm<TM, TX, B, BE_SET, L, NC><<<nb, 256, 0, s>>>(AMG_BMM_ARGS); break;
    case BE_SCALE: AMG_KCOUNT k_bsrmm<TM, TX, B, BE_SCALE, L, NC><<<nb, 256, 0, s>>>(AMG_BMM_ARGS); break;
    case BE_RESID: AMG_KCOUNT k_bsrmm<TM, TX, B, BE_RESID, L, NC><<<nb, 256, 0, s>>>(AMG_BMM_ARGS); break;
    case BE_SADD: AMG_KCOUNT k_bsrmm<TM, TX, B, BE_SADD, L, NC><<<nb, 256, 0, s>>>(AMG_BMM_ARGS); break;
    default: AMG_KCOUNT k_bsrmm<TM, TX, B, BE_ACC, L, NC><<<nb, 256, 0, s>>>(AMG_BMM_ARGS); break;
  }
#undef AMG_BMM_ARGS
}

template <typename TM, typename TX, int B>
static void bmm_b(int map, int ep, const SolveMat &M, const TM *v, int k, const TX *X, TX *Y, const TX *AUX, TX w,
                  const int *done, cudaStream_t s) {
  switch (map) {
    case 0: bmm_launch<TM, TX, B, 32, 1>(ep, M, v, k, X, Y, AUX, w, done, s); break;
    case 2: bmm_launch<TM, TX, B, 16, 2>(ep, M, v, k, X, Y, AUX, w, done, s); break;
    case 3: bmm_launch<TM, TX, B, 16, 4>(ep, M, v, k, X, Y, AUX, w, done, s); break;
    case 4: bmm_launch<TM, TX, B, 8, 4>(ep, M, v, k, X, Y, AUX, w, done, s); break;
    default: bmm_launch<TM, TX, B, 32, 2>(ep, M, v, k, X, Y, AUX, w, done, s); break;
  }
}

// the mapping the batched autotuner chose for this matrix, storage and k
// (32 x 2 until tuned)
template <typename TM>
static int bmap_of(const SolveMat &M, int k) {
  const int kind = std::is_same<TM, double>::value ? 0 : (std::is_same<TM, float>::value ? 1 : 2);
  return M.bmap_k[kind] == k ? M.bmap[kind] : 1;
}

template <typename TM, typename TX>
static void bmm(int ep, const SolveMat &M, const TM *v, int k, const TX *X, TX *Y, const TX *AUX, TX w, const int *done,
                cudaStream_t s) {
  const int map = bmap_of<TM>(M, k);
  if (M.b == 1) bmm_b<TM, TX, 1>(map, ep, M, v, k, X, Y, AUX, w, done, s);
  else bmm_b<TM, TX, 3>(map, ep, M, v, k, X, Y, AUX, w, done, s);
}

// ---------------------------------------------------------------- batched autotuner
// Each level matrix of a batched solve is timed with every mapping for the
// solve's k (CUDA events, one warm-up and two timed launches) on scratch
// blocks, in the storage the solve uses; the winner is kept on the matrix
// and cached per (storage, slice count, average row length, k), so later
// hierarchies of the same shape reuse it.  AMG_BMAP=<0..4> pins a mapping.
static std::mutex g_btune_mu;
static std::vector<std::pair<long long, int>> g_btune_cache;

template <typename TM, typename TX>
static int tune_bmm(SolveMat &M, const TM *v, int k, cudaStream_t s) {
  const int kind = std::is_same<TM, double>::value ? 0 : (std::is_same<TM, float>::value ? 1 : 2);
  if (M.nr == 0 || !v) return AMG_OK;
  if (const char *pin = getenv("AMG_BMAP")) {
    const int m = atoi(pin);
    if (m >= 0 && m < kNumBMaps) {
      M.bmap[kind] = m;
      M.bmap_k[kind] = k;
      return AMG_OK;
    }
  }
  const double avg = (double)M.nnzb / M.nr;
  const long long key = ((long long)kind << 60) | ((long long)M.b << 56) | ((long long)k << 40) |
                        ((long long)M.ns << 16) | (long long)(avg * 16.0 + 0.5);
  {
    std::lock_guard<std::mutex> lock(g_btune_mu);
    for (auto &e : g_btune_cache)
      if (e.first == key) {
        M.bmap[kind] = e.second;
        M.bmap_k[kind] = k;
        return AMG_OK;
      }
  }
  DBuf<TX> X, Y;
  AMG_TRY(X.alloc((size_t)M.b * M.nc * k));
  AMG_TRY(Y.alloc((size_t)M.b * M.nr * k));
  AMG_TRY(X.zero(s));
  cudaEvent_t e0, e1;
  AMG_CU(cudaEventCreate(&e0));
  AMG_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int bm = 1;
  for (int c = 0; c < kNumBMaps; ++c) {
    auto launch = [&]() {
      if (M.b == 1) bmm_b<TM, TX, 1>(c, BE_SET, M, v, k, X.p, Y.p, (const TX *)nullptr, TX(0), nullptr, s);
      else bmm_b<TM, TX, 3>(c, BE_SET, M, v, k, X.p, Y.p, (const TX *)nullptr, TX(0), nullptr, s);
    };
    launch();
    AMG_CU(cudaEventRecord(e0, s));
    launch();
    launch();
    AMG_CU(cudaEventRecord(e1, s));
    AMG_CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      bm = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  AMG_LAUNCH_CHECK();
  M.bmap[kind] = bm;
  M.bmap_k[kind] = k;
  if (getenv("AMG_TRACE"))
    fprintf(stderr, "[amg] batched mapping kind %d rows %d k %d -> L %d NC %d (%.4f ms)\n", kind, M.nr, k,
            kBMaps[bm].L, kBMaps[bm].NC, best / 2.0);
  std::lock_guard<std::mutex> lock(g_btune_mu);
  g_btune_cache.push_back({key, bm});
  return AMG_OK;
}

// every matrix the batched solve of k columns applies, in its storage
static int tune_batch(Handle *h, int k) {
  cudaStream_t s = h->stream;
  const int prec = h->prm.vcycle_prec;
  const bool b16 = prec == AMG_FP32_BF16GP;
  AMG_TRY((tune_bmm<double, double>(h->lev[0]->sA, h->lev[0]->sA.v64.p, k, s)));  // CG operator
  for (int l = 0; l < h->nlev - 1; ++l) {
    Level &L = *h->lev[l];
    if (prec == AMG_FP64) {
      for (SolveMat *M : {&L.sG, &L.sGT, &L.sP, &L.sR}) AMG_TRY((tune_bmm<double, double>(*M, M->v64.p, k, s)));
      if (l > 0) AMG_TRY((tune_bmm<double, double>(L.sA, L.sA.v64.p, k, s)));
    } else {
      AMG_TRY((tune_bmm<float, float>(L.sA, L.sA.v32.p, k, s)));
      for (SolveMat *M : {&L.sG, &L.sGT, &L.sP, &L.sR}) {
        if (b16) AMG_TRY((tune_bmm<__nv_bfloat16, float>(*M, M->v16.p, k, s)));
        else AMG_TRY((tune_bmm<float, float>(*M, M->v32.p, k, s)));
      }
    }
  }
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

template <typename TX>
static void bmv(int ep, const SolveMat &M, bool b16, int k, const TX *X, TX *Y, const TX *AUX, TX w, const int *done,
                cudaStream_t s);
template <>
void bmv<double>(int ep, const SolveMat &M, bool, int k, const double *X, double *Y, const double *AUX, double w,
                 const int *done, cudaStream_t s) {
  bmm<double, double>(ep, M, M.v64.p, k, X, Y, AUX, w, done, s);
}
template <>
void bmv<float>(int ep, const SolveMat &M, bool b16, int k, const float *X, float *Y, const float *AUX, float w,
                const int *done, cudaStream_t s) {
  if (b16) bmm<__nv_bfloat16, float>(ep, M, M.v16.p, k, X, Y, AUX, w, done, s);
  else bmm<float, float>(ep, M, M.v32.p, k, X, Y, AUX, w, done, s);
}

// coarse level: Z = Cinv Y with the explicit inverse (interleaved n x k, FP64
// arithmetic)
template <typename TX>
__global__ void k_bcoarse_mm(int m, int k, const double *__restrict__ Ci, const TX *__restrict__ Y,
                             TX *__restrict__ Z, const int *__restrict__ done) {
  if (done && *done) return;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)m * k) return;
  const int i = (int)(t / k), c = (int)(t % k);
  double s = 0.0;
  const double *Cr = Ci + (size_t)i * m;
  for (int q = 0; q < m; ++q) s = fma(Cr[q], (double)Y[(size_t)q * k + c], s);
  Z[t] = (TX)s;
}

// ---------------------------------------------------------------- block state
struct BatchLevel {
  DBuf<double> y64, z64, s64, r64, t64;
  DBuf<float> y32, z32, s32, r32, t32;
};

struct Batch {
  int k = 0, prec = -1;
  std::vector<BatchLevel> lev;
  DBuf<double> x, r, z, p, q, zold, sc, part;
  DBuf<int> flags;
  DBuf<float> rlow, zlow;
  cudaGraphExec_t graph = nullptr;
  long long graph_nodes = 0;
  int *pinned = nullptr;
  ~Batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (pinned) cudaFreeHost(pinned);
  }
};

// per-column scalar slots: sc[slot * k + c]
enum { BS_BN2 = 0, BS_RZ, BS_PQ, BS_ALPHA, BS_RR, BS_BETA, BS_TOL2, BS_TRR, BS_TRRP, BS_NUM };
// flags: [0] all done, [1] ticket, [2] status, [3] maxit, [4] iteration,
// [5] a column restarts from its true residual, then per column:
// [8 + c] state (0 active, 1 converged, 2 breakdown, 3 not converged),
// [8 + k + c] iterations of column c
enum { BF_DONE = 0, BF_TICKET = 1, BF_STATUS = 2, BF_MAXIT = 3, BF_ITER = 4, BF_RESTART = 5, BF_COL = 8 };
// true-residual restarts of one batched solve
constexpr int kMaxBatchRestarts = 8;

// Grid of the per-iteration vector kernels: two CTAs per SM (of 152), each
// thread streaming BUNR elements per pass with all their loads issued first
// (enough bytes in flight to keep HBM busy), and few block partials for the
// last block to add up.
constexpr int BRED_BLOCKS = 304;
constexpr int BUNR = 4;

// Per-column partial sums of one block into part[blockIdx][c]; the last
// block adds the partials in block order and runs fin(c, total) per column.
template <class Fin>
__device__ void bfinish(double v, int k, double *part, int *flags, Fin fin) {
  extern __shared__ double sh[];
  const int c = threadIdx.x % k;
  sh[threadIdx.x] = v;
  __syncthreads();
  const int per = blockDim.x / k;
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int q = 0; q < per; ++q) s += sh[c + q * k];
    part[(size_t)blockIdx.x * k + c] = s;
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&flags[BF_TICKET], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile double *)part)[(size_t)b * k + c];
    fin(c, s);
  }
  __syncthreads();
  if (threadIdx.x == 0) flags[BF_TICKET] = 0;
}

__device__ __forceinline__ bool col_active(const int *flags, int c) { return flags[BF_COL + c] == 0; }

// x = 0, r = b (from column-major B), rlow = (TX) r, bn2_c, tol2_c
template <typename TX>
__global__ void k_bstart(long n, int k, const double *__restrict__ B, double *__restrict__ x, double *__restrict__ r,
                         TX *__restrict__ rlow, double rtol, double *sc, int *flags, double *part) {
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += stride) {
    const long d = t / k;
    const int c = (int)(t - d * k);
    const double b = B[(size_t)c * n + d];
    x[t] = 0.0;
    r[t] = b;
    if (rlow) rlow[t] = (TX)b;
    v += b * b;
  }
  bfinish(v, k, part, flags, [&](int c, double tot) {
    sc[BS_BN2 * k + c] = tot;
    sc[BS_TOL2 * k + c] = (rtol * rtol) * tot;
    sc[BS_RZ * k + c] = 1.0;
    flags[BF_COL + c] = (tot == 0.0) ? 1 : 0;
    flags[BF_COL + k + c] = 0;
  });
}

__global__ void k_bflags(int k, int maxit, int *flags) {
  flags[BF_DONE] = 0;
  flags[BF_TICKET] = 0;
  flags[BF_STATUS] = 0;
  flags[BF_MAXIT] = maxit;
  flags[BF_ITER] = 0;
}

// pq_c = p.q ; alpha_c = rz_c / pq_c
__global__ void k_bpq(long n, int k, const double *__restrict__ p, const double *__restrict__ q, double *sc,
                      int *flags, double *part) {
  if (flags[BF_DONE]) return;
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x, N = n * k;
  for (long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x; t0 < N; t0 += BUNR * stride) {
    double pv[BUNR], qv[BUNR];
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      pv[u] = t < N ? p[t] : 0.0;
      qv[u] = t < N ? q[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BUNR; ++u) v += pv[u] * qv[u];
  }
  bfinish(v, k, part, flags, [&](int c, double tot) {
    sc[BS_PQ * k + c] = tot;
    if (col_active(flags, c)) {
      if (!(tot > 0.0) || !isfinite(tot)) {
        flags[BF_STATUS] = AMG_ERR_BREAKDOWN;
        flags[BF_COL + c] = 2;
      } else {
        sc[BS_ALPHA * k + c] = sc[BS_RZ * k + c] / tot;
      }
    }
  });
}

// active columns: x += alpha p, r -= alpha q ; rr_c ; convergence ; rlow
template <typename TX>
__global__ void k_bxr(long n, int k, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                      const double *__restrict__ q, TX *__restrict__ rlow, double *sc, int *flags, double *part) {
  if (flags[BF_DONE]) return;
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x, N = n * k;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  // the stride is a multiple of k: a thread keeps its column
  const int c = (int)(tid % k);
  const bool act = col_active(flags, c);
  const double a = act ? sc[BS_ALPHA * k + c] : 0.0;
  for (long t0 = tid; t0 < N; t0 += BUNR * stride) {
    double rv[BUNR], xv[BUNR], pv[BUNR], qv[BUNR];
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      const bool in = t < N;
      rv[u] = in ? r[t] : 0.0;
      xv[u] = in && act ? x[t] : 0.0;
      pv[u] = in && act ? p[t] : 0.0;
      qv[u] = in && act ? q[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      if (t >= N) break;
      double ri = rv[u];
      if (act) {
        x[t] = xv[u] + a * pv[u];
        ri = ri - a * qv[u];
        r[t] = ri;
      }
      if (rlow) rlow[t] = (TX)ri;
      v += ri * ri;
    }
  }
  bfinish(v, k, part, flags, [&](int c, double tot) {
    if (!col_active(flags, c)) return;
    sc[BS_RR * k + c] = tot;
    const int it = flags[BF_COL + k + c] + 1;
    flags[BF_COL + k + c] = it;
    if (!isfinite(tot)) {
      flags[BF_STATUS] = AMG_ERR_BREAKDOWN;
      flags[BF_COL + c] = 2;
    } else if (tot <= sc[BS_TOL2 * k + c]) {
      flags[BF_COL + c] = 1;
    } else if (it >= flags[BF_MAXIT]) {
      flags[BF_COL + c] = 3;
    }
  });
}

// z = (double) zlow ; rz_c (flexible: minus r.z_old) ; beta_c ; all-done test
template <typename TX>
__global__ void k_brz(long n, int k, const double *__restrict__ r, double *__restrict__ z, const TX *__restrict__ zlow,
                      const double *__restrict__ zold, int flexible, double *sc, int *flags, double *part) {
  if (flags[BF_DONE]) return;
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x, N = n * k;
  for (long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x; t0 < N; t0 += BUNR * stride) {
    double zv[BUNR], rv[BUNR], ov[BUNR];
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      const bool in = t < N;
      zv[u] = in ? (zlow ? (double)zlow[t] : z[t]) : 0.0;
      rv[u] = in ? r[t] : 0.0;
      ov[u] = in && flexible ? zold[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      if (t >= N) break;
      if (zlow) z[t] = zv[u];
      v += rv[u] * (flexible ? zv[u] - ov[u] : zv[u]);
    }
  }
  // for the flexible variant the sum above is r.(z - z_old); r.z itself is
  // needed as the next rz: accumulate it in a second pass over the block
  bfinish(v, k, part, flags, [&](int c, double tot) { sc[BS_BETA * k + c] = tot; });
}

// second reduction of the flexible variant: rz_c = r.z, then beta_c =
// (r.(z - z_old)) / rz_prev (flexible) or rz_c / rz_prev
__global__ void k_brz2(long n, int k, const double *__restrict__ r, const double *__restrict__ z, int flexible,
                       double *sc, int *flags, double *part) {
  if (flags[BF_DONE]) return;
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x, N = n * k;
  for (long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x; t0 < N; t0 += BUNR * stride) {
    double rv[BUNR], zv[BUNR];
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      rv[u] = t < N ? r[t] : 0.0;
      zv[u] = t < N ? z[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BUNR; ++u) v += rv[u] * zv[u];
  }
  bfinish(v, k, part, flags, [&](int c, double tot) {
    const double prev = sc[BS_RZ * k + c];
    const double num = flexible ? sc[BS_BETA * k + c] : tot;
    if (col_active(flags, c)) {
      sc[BS_BETA * k + c] = num / prev;
      sc[BS_RZ * k + c] = tot;
    }
  });
}

// active columns: p = z + beta p (z_old = z); the last thread checks whether
// every column has stopped
__global__ void k_bp(long n, int k, double *__restrict__ p, const double *__restrict__ z, double *__restrict__ zold,
                     int flexible, const double *sc, int *flags) {
  if (flags[BF_DONE]) return;
  const long stride = (long)gridDim.x * blockDim.x, N = n * k;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = (int)(tid % k);  // the stride is a multiple of k: a thread keeps its column
  if (!col_active(flags, c)) return;
  const double b = sc[BS_BETA * k + c];
  for (long t0 = tid; t0 < N; t0 += BUNR * stride) {
    double zv[BUNR], pv[BUNR];
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      zv[u] = t < N ? z[t] : 0.0;
      pv[u] = t < N ? p[t] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BUNR; ++u) {
      const long t = t0 + u * stride;
      if (t >= N) break;
      p[t] = zv[u] + b * pv[u];
      if (flexible) zold[t] = zv[u];
    }
  }
}

__global__ void k_bcheck(int k, int *flags) {
  int all = 1;
  for (int c = 0; c < k; ++c)
    if (flags[BF_COL + c] == 0) all = 0;
  if (all) flags[BF_DONE] = 1;
}

// first direction: p = z, z_old = z
__global__ void k_bfirst(long n, double *__restrict__ p, const double *__restrict__ z, double *__restrict__ zold,
                         const int *flags) {
  if (flags[BF_DONE]) return;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    p[t] = z[t];
    zold[t] = z[t];
  }
}

// True residuals after every column stopped: q holds K x (FP64 level-0 K);
// r = b - q (b read from the column-major right-hand sides), rlow = (TX) r,
// trr_c = ||r_c||^2.  A column that stopped as converged but whose true
// residual is above rtol ||b_c|| becomes active again (restart from its true
// residual, iteration count kept), within the limits of the single
// right-hand-side solve: at most max_phase restarts, below the iteration
// limit, and only while the previous restart halved its true residual.
template <typename TX>
__global__ void k_btrue(long n, int k, const double *__restrict__ B, const double *__restrict__ q,
                        double *__restrict__ r, TX *__restrict__ rlow, int phase, int max_phase, double *sc,
                        int *flags, double *part) {
  double v = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += stride) {
    const long d = t / k;
    const int c = (int)(t - d * k);
    const double ri = B[(size_t)c * n + d] - q[t];
    r[t] = ri;
    if (rlow) rlow[t] = (TX)ri;
    v += ri * ri;
  }
  bfinish(v, k, part, flags, [&](int c, double tot) {
    const double prev = sc[BS_TRRP * k + c];
    sc[BS_TRR * k + c] = tot;
    sc[BS_TRRP * k + c] = tot;
    if (flags[BF_COL + c] != 1) return;
    if (!isfinite(tot)) {
      flags[BF_STATUS] = AMG_ERR_BREAKDOWN;
      flags[BF_COL + c] = 2;
    } else if (tot > sc[BS_TOL2 * k + c] && phase < max_phase && flags[BF_COL + k + c] < flags[BF_MAXIT] &&
               !(phase > 0 && tot > 0.25 * prev)) {
      sc[BS_RR * k + c] = tot;
      flags[BF_COL + c] = 0;
      flags[BF_RESTART] = 1;
    }
  });
}

// done again unless a column restarts
__global__ void k_brestart_done(int *flags) {
  flags[BF_DONE] = flags[BF_RESTART] ? 0 : 1;
  flags[BF_RESTART] = 0;
}

// interleaved -> column-major
__global__ void k_bout(long n, int k, const double *__restrict__ x, double *__restrict__ X) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const long d = t / k;
  const int c = (int)(t - d * k);
  X[(size_t)c * n + d] = x[t];
}

template <typename TX> struct BVec;
template <> struct BVec<double> {
  static double *y(BatchLevel &L) { return L.y64.p; }
  static double *z(BatchLevel &L) { return L.z64.p; }
  static double *s(BatchLevel &L) { return L.s64.p; }
  static double *r(BatchLevel &L) { return L.r64.p; }
  static double *t(BatchLevel &L) { return L.t64.p; }
};
template <> struct BVec<float> {
  static float *y(BatchLevel &L) { return L.y32.p; }
  static float *z(BatchLevel &L) { return L.z32.p; }
  static float *s(BatchLevel &L) { return L.s32.p; }
  static float *r(BatchLevel &L) { return L.r32.p; }
  static float *t(BatchLevel &L) { return L.t32.p; }
};

template <typename TX>
static void bvcycle(Handle *h, Batch &B, int lv, const TX *y, TX *z, const int *done) {
  cudaStream_t st = h->stream;
  const int k = B.k;
  const bool b16 = h->prm.vcycle_prec == AMG_FP32_BF16GP;
  if (lv == h->nlev - 1) {
    const int m = h->nL;
    if (!m) return;
    AMG_KCOUNT k_bcoarse_mm<TX><<<nblk((long)m * k, 256), 256, 0, st>>>(m, k, h->Cinv.p, y, z, done);
    return;
  }
  Level &L = *h->lev[lv];
  BatchLevel &BL = B.lev[lv], &BC = B.lev[lv + 1];
  TX *s = BVec<TX>::s(BL), *r = BVec<TX>::r(BL), *t = BVec<TX>::t(BL);
  const TX w = (TX)L.omega;
  bmv<TX>(BE_SET, L.sG, b16, k, y, t, (const TX *)nullptr, w, done, st);
  bmv<TX>(BE_SCALE, L.sGT, b16, k, t, s, (const TX *)nullptr, w, done, st);
  bmv<TX>(BE_RESID, L.sA, false, k, s, r, y, w, done, st);
  bmv<TX>(BE_SET, L.sR, b16, k, r, BVec<TX>::y(BC), (const TX *)nullptr, w, done, st);
  bvcycle<TX>(h, B, lv + 1, BVec<TX>::y(BC), BVec<TX>::z(BC), done);
  bmv<TX>(BE_ACC, L.sP, b16, k, BVec<TX>::z(BC), s, (const TX *)nullptr, w, done, st);
  bmv<TX>(BE_RESID, L.sA, false, k, s, r, y, w, done, st);
  bmv<TX>(BE_SET, L.sG, b16, k, r, t, (const TX *)nullptr, w, done, st);
  bmv<TX>(BE_SADD, L.sGT, b16, k, t, z, s, w, done, st);
}

static int block_threads(int k) { return (256 / k) * k; }

template <typename TX>
static void biteration(Handle *h, Batch &B, bool mixed) {
  cudaStream_t s = h->stream;
  const int k = B.k;
  const long n = (long)h->b * h->n;
  Level &L0 = *h->lev[0];
  const int bt = block_threads(k);
  const size_t shm = bt * sizeof(double);
  int *fl = B.flags.p;
  const int *done = fl + BF_DONE;
  bmm<double, double>(BE_SET, L0.sA, L0.sA.v64.p, k, B.p.p, B.q.p, nullptr, 0.0, done, s);
  AMG_KCOUNT k_bpq<<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.p.p, B.q.p, B.sc.p, fl, B.part.p);
  if (mixed) {
    AMG_KCOUNT k_bxr<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.x.p, B.r.p, B.p.p, B.q.p, B.rlow.p, B.sc.p, fl, B.part.p);
    bvcycle<float>(h, B, 0, B.rlow.p, B.zlow.p, done);
    AMG_KCOUNT k_brz<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.r.p, B.z.p, B.zlow.p, B.zold.p, 1, B.sc.p, fl, B.part.p);
    AMG_KCOUNT k_brz2<<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.r.p, B.z.p, 1, B.sc.p, fl, B.part.p);
    AMG_KCOUNT k_bp<<<BRED_BLOCKS, bt, 0, s>>>(n, k, B.p.p, B.z.p, B.zold.p, 1, B.sc.p, fl);
  } else {
    AMG_KCOUNT k_bxr<double><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.x.p, B.r.p, B.p.p, B.q.p, (double *)nullptr, B.sc.p, fl,
                                                          B.part.p);
    bvcycle<double>(h, B, 0, B.r.p, B.z.p, done);
    AMG_KCOUNT k_brz2<<<BRED_BLOCKS, bt, shm, s>>>(n, k, B.r.p, B.z.p, 0, B.sc.p, fl, B.part.p);
    AMG_KCOUNT k_bp<<<BRED_BLOCKS, bt, 0, s>>>(n, k, B.p.p, B.z.p, B.zold.p, 0, B.sc.p, fl);
  }
  AMG_KCOUNT k_bcheck<<<1, 1, 0, s>>>(k, fl);
}

static int ensure_batch(Handle *h, Batch &B, int k) {
  const int prec = h->prm.vcycle_prec;
  if (B.k == k && B.prec == prec && B.x.p) return AMG_OK;
  if (B.graph) {
    cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
  }
  AMG_TRY(tune_batch(h, k));
  B.k = k;
  B.prec = prec;
  const size_t nk = (size_t)h->b * h->n * k;
  AMG_TRY(B.x.alloc(nk));
  AMG_TRY(B.r.alloc(nk));
  AMG_TRY(B.z.alloc(nk));
  AMG_TRY(B.p.alloc(nk));
  AMG_TRY(B.q.alloc(nk));
  AMG_TRY(B.zold.alloc(nk));
  AMG_TRY(B.sc.alloc((size_t)BS_NUM * k));
  AMG_TRY(B.part.alloc((size_t)BRED_BLOCKS * k + 16));
  AMG_TRY(B.flags.alloc(BF_COL + 2 * k + 8));
  if (!B.pinned) AMG_CU(cudaMallocHost((void **)&B.pinned, 4 * sizeof(int)));
  B.lev.clear();
  B.lev.resize(h->nlev);
  const bool mixed = prec != AMG_FP64;
  if (mixed) {
    AMG_TRY(B.rlow.alloc(nk));
    AMG_TRY(B.zlow.alloc(nk));
  }
  for (int l = 0; l < h->nlev; ++l) {
    const size_t m = (size_t)h->b * h->lev[l]->n * k;
    BatchLevel &BL = B.lev[l];
    if (mixed) {
      if (l > 0) {
        AMG_TRY(BL.y32.alloc(m));
        AMG_TRY(BL.z32.alloc(m));
      }
      AMG_TRY(BL.s32.alloc(m));
      AMG_TRY(BL.r32.alloc(m));
      AMG_TRY(BL.t32.alloc(m));
    } else {
      if (l > 0) {
        AMG_TRY(BL.y64.alloc(m));
        AMG_TRY(BL.z64.alloc(m));
      }
      AMG_TRY(BL.s64.alloc(m));
      AMG_TRY(BL.r64.alloc(m));
      AMG_TRY(BL.t64.alloc(m));
    }
  }
  return AMG_OK;
}

int solve_batched(Handle *h, int k, const double *B, double *X, double rtol, int *iters, double *relres) {
  if (k > 256) {
    // independent groups of at most 256 columns
    int worst = AMG_OK, nit = 0, nrs = 0;
    double rec = 0.0, tru = 0.0;
    const size_t n = (size_t)h->b * h->n;
    for (int c0 = 0; c0 < k; c0 += 256) {
      const int kk = k - c0 < 256 ? k - c0 : 256;
      const int rc = solve_batched(h, kk, B + c0 * n, X + c0 * n, rtol, iters + c0, relres + c0);
      if (rc == AMG_ERR_CUDA) return rc;
      if (rc && !worst) worst = rc;
      nit = std::max(nit, h->stats.n_it);
      rec = std::max(rec, h->stats.relres_rec);
      tru = std::max(tru, h->stats.relres_true);
      nrs += h->stats.restarts;
    }
    h->stats.n_it = nit;
    h->stats.relres_rec = rec;
    h->stats.relres_true = tru;
    h->stats.restarts = nrs;
    return worst;
  }
  if (!h->batch) h->batch = new Batch();
  Batch &Bt = *h->batch;
  AMG_TRY(ensure_batch(h, Bt, k));
  cudaStream_t s = h->stream;
  const long n = (long)h->b * h->n;
  const bool mixed = h->prm.vcycle_prec != AMG_FP64;
  const int bt = block_threads(k);
  const size_t shm = bt * sizeof(double);
  int *fl = Bt.flags.p;
  AMG_KCOUNT k_bflags<<<1, 1, 0, s>>>(k, h->prm.maxit, fl);
  if (mixed) {
    AMG_KCOUNT k_bstart<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B, Bt.x.p, Bt.r.p, Bt.rlow.p, rtol, Bt.sc.p, fl,
                                                            Bt.part.p);
    AMG_KCOUNT k_bcheck<<<1, 1, 0, s>>>(k, fl);
    bvcycle<float>(h, Bt, 0, Bt.rlow.p, Bt.zlow.p, fl + BF_DONE);
    AMG_KCOUNT k_brz<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, Bt.r.p, Bt.z.p, Bt.zlow.p, Bt.zold.p, 0, Bt.sc.p, fl,
                                                         Bt.part.p);
  } else {
    AMG_KCOUNT k_bstart<double><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B, Bt.x.p, Bt.r.p, (double *)nullptr, rtol, Bt.sc.p,
                                                             fl, Bt.part.p);
    AMG_KCOUNT k_bcheck<<<1, 1, 0, s>>>(k, fl);
    bvcycle<double>(h, Bt, 0, Bt.r.p, Bt.z.p, fl + BF_DONE);
  }
  AMG_KCOUNT k_brz2<<<BRED_BLOCKS, bt, shm, s>>>(n, k, Bt.r.p, Bt.z.p, 0, Bt.sc.p, fl, Bt.part.p);
  AMG_KCOUNT k_bfirst<<<BRED_BLOCKS, 256, 0, s>>>(n * k, Bt.p.p, Bt.z.p, Bt.zold.p, fl);
  AMG_LAUNCH_CHECK();
  if (!Bt.graph) {
    cudaGraph_t g;
    const long long before = launch_count();
    AMG_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    if (mixed) biteration<float>(h, Bt, true);
    else biteration<double>(h, Bt, false);
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    Bt.graph_nodes = launch_count() - before;
    count_launches(-Bt.graph_nodes);
    if (ce != cudaSuccess) {
      set_error("batched solve: graph capture failed: %s", cudaGetErrorString(ce));
      return AMG_ERR_CUDA;
    }
    AMG_CU(cudaGraphInstantiate(&Bt.graph, g, 0));
    cudaGraphDestroy(g);
  }
  const int chunk = 4;
  int rc = AMG_OK;
  Level &L0 = *h->lev[0];
  int restarts = 0;
  // Phases: replay until every column stopped, then the FP64 true residuals;
  // columns above rtol restart from theirs (one V-cycle of the block).
  for (;;) {
    for (int it = 0; it < h->prm.maxit + chunk; it += chunk) {
      for (int c = 0; c < chunk; ++c) {
        if (cudaGraphLaunch(Bt.graph, s) != cudaSuccess) {
          set_error("batched solve: graph launch failed");
          return AMG_ERR_CUDA;
        }
        count_launches(Bt.graph_nodes);
      }
      AMG_CU(cudaMemcpyAsync(Bt.pinned, fl, sizeof(int), cudaMemcpyDeviceToHost, s));
      const cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error("batched solve: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
      }
      if (Bt.pinned[0]) break;
    }
    bmm<double, double>(BE_SET, L0.sA, L0.sA.v64.p, k, Bt.x.p, Bt.q.p, nullptr, 0.0, nullptr, s);
    if (mixed)
      AMG_KCOUNT k_btrue<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B, Bt.q.p, Bt.r.p, Bt.rlow.p, restarts,
                                                             kMaxBatchRestarts, Bt.sc.p, fl, Bt.part.p);
    else
      AMG_KCOUNT k_btrue<double><<<BRED_BLOCKS, bt, shm, s>>>(n, k, B, Bt.q.p, Bt.r.p, (double *)nullptr, restarts,
                                                              kMaxBatchRestarts, Bt.sc.p, fl, Bt.part.p);
    AMG_KCOUNT k_brestart_done<<<1, 1, 0, s>>>(fl);
    // restart of the reopened columns (done-gated, as the start sequence)
    if (mixed) {
      bvcycle<float>(h, Bt, 0, Bt.rlow.p, Bt.zlow.p, fl + BF_DONE);
      AMG_KCOUNT k_brz<float><<<BRED_BLOCKS, bt, shm, s>>>(n, k, Bt.r.p, Bt.z.p, Bt.zlow.p, Bt.zold.p, 0, Bt.sc.p, fl,
                                                           Bt.part.p);
    } else {
      bvcycle<double>(h, Bt, 0, Bt.r.p, Bt.z.p, fl + BF_DONE);
    }
    AMG_KCOUNT k_brz2<<<BRED_BLOCKS, bt, shm, s>>>(n, k, Bt.r.p, Bt.z.p, 0, Bt.sc.p, fl, Bt.part.p);
    AMG_KCOUNT k_bfirst<<<BRED_BLOCKS, 256, 0, s>>>(n * k, Bt.p.p, Bt.z.p, Bt.zold.p, fl);
    AMG_LAUNCH_CHECK();
    AMG_CU(cudaMemcpyAsync(Bt.pinned, fl, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
    if (Bt.pinned[0]) break;
    ++restarts;
  }
  AMG_KCOUNT k_bout<<<nblk(n * k, 256), 256, 0, s>>>(n, k, Bt.x.p, X);
  AMG_LAUNCH_CHECK();
  std::vector<int> hf(BF_COL + 2 * k);
  std::vector<double> hs((size_t)BS_NUM * k);
  AMG_CU(cudaMemcpyAsync(hf.data(), fl, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaMemcpyAsync(hs.data(), Bt.sc.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  int maxit = 0;
  double rec_max = 0.0, true_max = 0.0;
  for (int c = 0; c < k; ++c) {
    iters[c] = hf[BF_COL + k + c];
    const double bn2 = hs[BS_BN2 * k + c];
    relres[c] = bn2 > 0.0 ? std::sqrt(hs[BS_TRR * k + c] / bn2) : 0.0;
    const double rec = bn2 > 0.0 ? std::sqrt(hs[BS_RR * k + c] / bn2) : 0.0;
    rec_max = rec > rec_max ? rec : rec_max;
    true_max = relres[c] > true_max ? relres[c] : true_max;
    const int st = hf[BF_COL + c];
    if (st == 2) rc = AMG_ERR_BREAKDOWN;
    else if ((st == 3 || st == 0) && rc == AMG_OK) rc = AMG_ERR_NOT_CONVERGED;
    if (iters[c] > maxit) maxit = iters[c];
  }
  h->stats.n_it = maxit;
  h->stats.relres_rec = rec_max;
  h->stats.relres_true = true_max;
  h->stats.restarts = restarts;
  return rc;
}

void free_batch(Handle *h) {
  delete h->batch;
  h->batch = nullptr;
}

}  // namespace amg
