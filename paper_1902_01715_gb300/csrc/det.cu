// Set-up kernels whose floating-point results decide the hierarchy's
// structure: FSAI rows, the Lanczos estimate of lambda_1(G A G^T), SRQCG,
// affinity SoC and its filter, DPLS least-squares fits and the Galerkin
// product.  This file is compiled with -fmad=false: every sum is taken in the
// fixed order stated at each kernel, so that the hierarchy (C/F split,
// patterns of G, P and A_c) is reproducible bit for bit by any implementation
// that follows the same order.  The accumulations of dot products, sparse
// row sums, Cholesky updates, triangular-solve updates, the aFSAI functional
// and gradients and the Galerkin block product are explicit fused
// multiply-adds, s <- fma(a, b, s) (one IEEE rounding per term; FP64 issue
// slots are the scarce resource of this GPU); everything else rounds each
// multiply and each add separately (the compiler fuses nothing).
// Fixed orders used throughout:
//  * sparse row sums: blocks in ascending column order, then the block's
//    columns, starting from 0;
//  * global dot products: chunks of 1024 entries; inside a chunk, lane l of a
//    warp sums entries l, l+32, ... ascending, the 32 lane sums are combined
//    by xor-exchange steps 16, 8, 4, 2, 1; one level up, lane l sums chunk
//    sums l, l+32, ... ascending and the same exchange steps give the total.
#include <cfloat>
#include <cstdlib>

#include "amg_internal.h"

namespace amg {
namespace det {

constexpr int CHUNK = 1024;
constexpr int MAXTICKETS = 512;  // per-pair tickets of one dot launch, plus one
constexpr int TMAXD = 16;  // largest test space handled by the DPLS kernel

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  // SplitMix64 (Steele, Lea, Flood 2014): state seed + (counter+1)*gamma,
  // then the published 30/27/31 xor-shift-multiply finaliser.
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t counter) {
  const uint64_t m = splitmix64(seed, counter) >> 11;
  return ((double)m * 0x1.0p-53) * 2.0 - 1.0;
}

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- SpMV
// sum_k sum_c A_k[r][c] x[BS J_k + c] over the blocks kb..ke-1 of one block
// row (BS x BS blocks), one fused multiply-add per term in block and column
// order.  The indices and operands of U blocks are loaded ahead of their
// chain, so a long row waits on memory once per U blocks rather than once per
// block.
template <int BS, int U>
__device__ __forceinline__ double row_chain(int kb, int ke, int r, const int *__restrict__ col,
                                            const double *__restrict__ val, const double *__restrict__ x, double s) {
  for (int k0 = kb; k0 < ke; k0 += U) {
    long J[U];
    double a[U][BS], xv[U][BS];
#pragma unroll
    for (int u = 0; u < U; ++u) J[u] = k0 + u < ke ? col[k0 + u] : 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        a[u][c] = k0 + u < ke ? val[(size_t)(k0 + u) * BS * BS + r * BS + c] : 0.0;
        xv[u][c] = k0 + u < ke ? x[J[u] * BS + c] : 0.0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < ke)
#pragma unroll
        for (int c = 0; c < BS; ++c) s = fma(a[u][c], xv[u][c], s);
  }
  return s;
}

template <int BS, int U>
__global__ void k_spmv(int nr, const int *__restrict__ rowptr, const int *__restrict__ col,
                       const double *__restrict__ val, const double *__restrict__ x,
                       double *__restrict__ y) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)BS * nr) return;
  const int I = (int)(t / BS), r = (int)(t - (long)BS * I);
  y[t] = row_chain<BS, U>(rowptr[I], rowptr[I + 1], r, col, val, x, 0.0);
}

// Below this many block rows a product has too few warps to hide memory
// latency and the loads are batched (more registers per thread); above it the
// plain loop keeps more warps resident.
constexpr int SMALL_ROWS = 16384;

template <int BS>
static void spmv_b(const DevBsr &A, const double *x, double *y, cudaStream_t s) {
  const long n = (long)BS * A.nr;
  if (A.nr < SMALL_ROWS)
    launch_k(k_spmv<BS, 8>, nblk(n, 256), 256, 0, s, A.nr, A.rowptr.p, A.col.p, A.val.p, x, y);
  else
    launch_k(k_spmv<BS, 1>, nblk(n, 256), 256, 0, s, A.nr, A.rowptr.p, A.col.p, A.val.p, x, y);
}

int spmv(const DevBsr &A, const double *x, double *y, cudaStream_t s) {
  if (A.nr == 0) return AMG_OK;
  if (A.b == 1) spmv_b<1>(A, x, y, s);
  else spmv_b<3>(A, x, y, s);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// ---------------------------------------------------------------- dots
// One launch per group of dot products, one-warp blocks.  Warp w computes
// chunk c of pair d (lane sums of stride 32, then the exchange steps); the
// warp that completes the last chunk of a pair (per-pair ticket) combines
// that pair's chunk sums in the fixed order; the warp that completes the
// last pair (one more ticket) runs the scalar step that consumes the sums
// (Fin), so no separate scalar kernel is needed.  Warps are spread over the
// SMs because each SM's FP64 pipe is narrow.
constexpr int MAXD = 8;
struct DotArgs {
  const double *x[MAXD];
  const double *y[MAXD];
};

enum { FIN_NONE = 0, FIN_SRQ_ALPHA = 1, FIN_SRQ_Q = 2, FIN_SRQ_BETA = 3, FIN_LZ_BETA = 4 };
struct Fin {
  int op = FIN_NONE;
  double *sc = nullptr;
  int *skip = nullptr;
  int i = 0, j = 0, m = 0;
};

__device__ double line_min(double a, double b, double c, double d, double e, double f);
__device__ int gen_eig_cta(int t, const double *H, const double *M, double *U, double *lam, double *w, int tid);

__device__ __forceinline__ double exchange32(double s) {
  for (int off = 16; off >= 1; off >>= 1) s = s + __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Chunk [base, end) of x . y: lane l accumulates entries base+l, base+l+32,
// ... (at most 32 of them, loads issued 16 at a time ahead of the chain),
// then the exchange steps.
__device__ __forceinline__ double chunk_sum(const double *__restrict__ x, const double *__restrict__ y,
                                            int base, int end, int lane) {
  double s = 0.0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    double xv[16], yv[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = base + lane + 32 * (16 * h + u);
      xv[u] = i < end ? x[i] : 0.0;
      yv[u] = i < end ? y[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (base + lane + 32 * (16 * h + u) < end) s = fma(xv[u], yv[u], s);
  }
  return exchange32(s);
}

// Chunk sums p[0..nchunks) of one pair: lane l adds sums l, l+32, ... in
// increasing order (loads 8 at a time ahead), then the exchange steps.
__device__ __forceinline__ double sum_chunks(const double *p, int nchunks, int lane) {
  double t = 0.0;
  for (int c0 = lane; c0 < nchunks; c0 += 32 * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (c0 + 32 * u < nchunks) ? __ldcg(p + c0 + 32 * u) : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c0 + 32 * u < nchunks) t = t + v[u];
  }
  return exchange32(t);
}

// Ticket: returns true in every lane of the warp that finished last.
__device__ __forceinline__ bool last_warp(unsigned *ticket, unsigned total, int lane) {
  unsigned t = 0;
  if (lane == 0) {
    __threadfence();
    t = atomicAdd(ticket, 1u);
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  return t == total - 1;
}

// Second half of a dot launch for warp w (nchunks > 0): store this warp's
// chunk sum sc, and in the warp completing pair d add the pair's chunk sums
// in order and put the total; returns true in the warp completing the last
// pair.
template <class Put>
__device__ __forceinline__ bool dot_finish(long w, int nd, int nchunks, double *part, unsigned *ticket, int lane,
                                           double sc, Put put) {
  const int d = (int)(w / nchunks), c = (int)(w - (long)d * nchunks);
  if (lane == 0) part[(size_t)d * nchunks + c] = sc;
  if (!last_warp(ticket + d, (unsigned)nchunks, lane)) return false;
  const double tot = sum_chunks(part + (size_t)d * nchunks, nchunks, lane);
  if (lane == 0) {
    put(d, tot);
    ticket[d] = 0u;
  }
  if (!last_warp(ticket + nd, (unsigned)nd, lane)) return false;
  if (lane == 0) ticket[nd] = 0u;
  return true;
}

// The work of warp w in a dot launch over nd pairs (x_d, y_d given by xy);
// the finished sum of pair d goes to put(d, value) from lane 0.  Returns true
// in the one warp that completed the last pair (every put is then visible
// through __ldcg).  With empty vectors a single warp puts zeros.
template <class XY, class Put>
__device__ __forceinline__ bool dot_warp(long w, int n, int nd, int nchunks, double *part, unsigned *ticket, int lane,
                                         XY xy, Put put) {
  if (nchunks == 0) {
    if (lane == 0)
      for (int d = 0; d < nd; ++d) put(d, 0.0);
    __threadfence();
    return true;
  }
  const int d = (int)(w / nchunks), c = (int)(w - (long)d * nchunks);
  const double *x, *y;
  xy(d, x, y);
  const int base = c * CHUNK, end = min(base + CHUNK, n);
  return dot_finish(w, nd, nchunks, part, ticket, lane, chunk_sum(x, y, base, end, lane), put);
}

// scalar steps of Algorithm 4 and of the Lanczos recurrence
__device__ void run_fin(const Fin &f, const double *v) {
  double *sc = f.sc;
  if (f.op == FIN_SRQ_ALPHA) {  // v = a, b, c, d, e (stored at sc[S_A..])
    const double b = v[1];
    if (!(b > 0.0)) {
      *f.skip = 1;
      return;
    }
    *f.skip = 0;
    sc[5] = line_min(v[0], b, v[2], v[3], v[4], sc[16 + f.i]);
  } else if (f.op == FIN_SRQ_Q) {  // v = f_new, z.Sz
    sc[8] = v[1] / v[0];
  } else if (f.op == FIN_SRQ_BETA) {  // v = g.Sp
    sc[10] = -(v[0] / sc[1]);
  } else if (f.op == FIN_LZ_BETA) {  // v = w.w ; beta_j and the breakdown test
    const double b = sqrt(v[0]);
    sc[64 + f.j] = b;
    sc[256 + f.j] = 1.0 / b;
    if (sc[128] < 0.0 && f.j < f.m - 1 && !(b > 1e-12 * fabs(sc[f.j]))) sc[128] = (double)(f.j + 1);
  }
}

__global__ void __launch_bounds__(32) k_dots(int n, int nd, DotArgs a, double *__restrict__ part, unsigned *ticket,
                                             int nchunks, double *__restrict__ out, Fin fin) {
  pdl_wait();
  const long w = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const long total = nchunks > 0 ? (long)nchunks * nd : 1;
  if (w >= total) return;
  const bool last = dot_warp(
      w, n, nd, nchunks, part, ticket, lane,
      [&](int d, const double *&x, const double *&y) {
        x = a.x[d];
        y = a.y[d];
      },
      [&](int d, double v) { out[d] = v; });
  if (!last || lane != 0) return;
  double v[MAXD];
  for (int d = 0; d < MAXD; ++d) v[d] = d < nd ? __ldcg(out + d) : 0.0;
  run_fin(fin, v);
}

struct DotCtx {
  double *part;
  unsigned *ticket;
};

static int dots(int n, int nd, const DotArgs &a, double *out, DotCtx ctx, cudaStream_t s, Fin fin = Fin()) {
  const int nchunks = (n + CHUNK - 1) / CHUNK;
  const long warps = nchunks > 0 ? (long)nchunks * nd : 1;
  launch_k(k_dots, (int)warps, 32, 0, s, n, nd, a, ctx.part, ctx.ticket, nchunks, out, fin);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int dot1(int n, const double *x, const double *y, double *out, DotCtx ctx, cudaStream_t s,
                Fin fin = Fin()) {
  DotArgs a{};
  a.x[0] = x;
  a.y[0] = y;
  return dots(n, 1, a, out, ctx, s, fin);
}

// Gram sums of the Ritz step, H[i][j] = Z_i . SZ_j and M[i][j] = Z_i . Z_j for
// i <= j (each in the fixed dot order, mirrored to j < i); k_ritz_eig then
// solves the pencil (H, M) for U.
__device__ __forceinline__ void pair_of(int d, int t, int &which, int &i, int &j) {
  const int npair = t * (t + 1) / 2;
  which = d / npair;
  int pr = d - which * npair;
  i = 0;
  while (pr >= t - i) { pr -= t - i; ++i; }
  j = i + pr;
}

__global__ void __launch_bounds__(32) k_gram(int n, int t, const double *__restrict__ Z, const double *__restrict__ SZ,
                                             double *__restrict__ part, unsigned *ticket, int nchunks,
                                             double *__restrict__ H, double *__restrict__ M) {
  pdl_wait();
  const int nd = t * (t + 1);
  const long w = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const long total = nchunks > 0 ? (long)nchunks * nd : 1;
  if (w >= total) return;
  dot_warp(
      w, n, nd, nchunks, part, ticket, lane,
      [&](int d, const double *&x, const double *&y) {
        int which, i, j;
        pair_of(d, t, which, i, j);
        x = Z + (size_t)i * n;
        y = which == 0 ? SZ + (size_t)j * n : Z + (size_t)j * n;
      },
      [&](int d, double v) {
        int which, i, j;
        pair_of(d, t, which, i, j);
        double *O = which == 0 ? H : M;
        O[i * t + j] = v;
        O[j * t + i] = v;
      });
}

// The pencil (H, M) of the Gram kernel solved for U (and lam); the quotient
// scalars f_i reset to 1.  One CTA of 4 warps.
__global__ void __launch_bounds__(128) k_ritz_eig(int t, const double *__restrict__ H, const double *__restrict__ M,
                                                 double *__restrict__ U, double *__restrict__ lam,
                                                 double *__restrict__ f, int *__restrict__ status) {
  pdl_wait();
  extern __shared__ double wk[];  // 6 t^2 + t doubles
  const int tid = threadIdx.x;
  // the pencil was written by other CTAs: read it through L2 into shared memory
  double *Hs = wk + 4 * t * t + t, *Ms = Hs + t * t;
  for (int q = tid; q < t * t; q += 128) {
    Hs[q] = __ldcg(H + q);
    Ms[q] = __ldcg(M + q);
  }
  __syncthreads();
  const int bad = gen_eig_cta(t, Hs, Ms, U, lam, wk, tid);
  if (tid == 0) {
    if (bad) atomicMin(status, AMG_ERR_NOT_SPD);
    for (int i = 0; i < t; ++i) f[i] = 1.0;
  }
}

// ---------------------------------------------------------------- vector ops

// v = v (1 / sqrt(*nn)) when *nn > 0 (normalisation by a squared norm)
__global__ void k_div_sqrt(long n, double *__restrict__ v, const double *__restrict__ nn) {
  pdl_wait();
  const double nr = sqrt(*nn);
  if (!(nr > 0.0)) return;
  const double rn = 1.0 / nr;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] * rn;
}

// out = in * (*rd), rd a reciprocal formed once
__global__ void k_mul_by(long n, double *__restrict__ out, const double *__restrict__ in,
                         const double *__restrict__ rd) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] * (*rd);
}

__global__ void k_uniform(long n, int col0, int ncols, uint64_t seed, double *__restrict__ V, int ld) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ncols) return;
  const int j = col0 + (int)(t / n);
  const long i = t - (long)(j - col0) * n;
  V[(size_t)j * ld + i] = uniform_pm1(seed, ((uint64_t)j << 40) | (uint64_t)i);
}

int uniform_fill(double *v, int n, int col0, int ncols, uint64_t seed, cudaStream_t s) {
  if (ncols <= 0 || n <= 0) return AMG_OK;
  launch_k(k_uniform, nblk((long)n * ncols, 256), 256, 0, s, n, col0, ncols, seed, v, n);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

__global__ void k_gather_rows(const int *__restrict__ src, int nout, int nin, int t, const double *__restrict__ Vin,
                              double *__restrict__ Vout) {
  pdl_wait();
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)nout * t) return;
  const int j = (int)(q / nout);
  const long i = q - (long)j * nout;
  Vout[(size_t)j * nout + i] = Vin[(size_t)j * nin + src[i]];
}

int gather_rows(const int *src_idx, int nout, int nin, int t, const double *Vin, double *Vout, cudaStream_t s) {
  if (nout <= 0) return AMG_OK;
  launch_k(k_gather_rows, nblk((long)nout * t, 256), 256, 0, s, src_idx, nout, nin, t, Vin, Vout);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// Modified Gram-Schmidt on the columns of V (n x t), column order; each column
// divided by its norm when that is positive.
// Step (j, i) of modified Gram-Schmidt, fused with the vector work the
// previous step left pending, chunk by chunk (warp c owns chunk c, lane l its
// entries base+l, base+l+32, ..., the dot order): for i = 0 and j > 0 column
// j-1 is divided by sqrt(sc[t]) (its norm square); for i > 0,
// v_j -= sc[i-1] v_{i-1}; then the chunk's part of v_i . v_j (i < j, into
// sc[i]) or v_j . v_j (i = j, into sc[t]), from the values this lane has
// just formed, in the two-level dot order.  Each entry receives the same
// rounded operations, in the same order, as the column-by-column definition.
// Chunk c of step (j, i): the fused vector work and this chunk's part of the
// step's dot product (exchanged over the warp); sc holds the totals of the
// earlier steps (sc[i'] for i' < j, sc[t] the norm square of column j - 1).
__device__ __forceinline__ double mgs_chunk(int n, int t, double *__restrict__ V, int j, int i, int c,
                                           const double *sc, int lane) {
  double *vj = V + (size_t)j * n;
  const int base = c * CHUNK, end = min(base + CHUNK, n);
  const bool norm_prev = i == 0 && j > 0;
  double *vp = V + (size_t)(j > 0 ? j - 1 : 0) * n;
  const double nr = norm_prev ? sqrt(sc[t]) : 1.0, rn = 1.0 / nr;
  const double r = i > 0 ? sc[i - 1] : 0.0;
  const double *vu = V + (size_t)(i > 0 ? i - 1 : 0) * n;  // v_{i-1}
  const double *vi = V + (size_t)i * n;
  // the lane's entries in groups of MB: every load of a group is issued
  // before any of its entries is formed (a lane reads and writes only its own
  // entries, and the columns read are other than the ones written, except
  // v_i = v_j and v_i = v_{j-1}, which take the values just formed)
  const bool load_i = i != j && !(norm_prev && i == j - 1);
  constexpr int MB = 8;
  double s = 0.0;
  for (int k0 = base + lane; k0 < end; k0 += 32 * MB) {
    double pv[MB], jv[MB], uv[MB], iv[MB];
#pragma unroll
    for (int u = 0; u < MB; ++u) {
      const int k = k0 + 32 * u;
      const bool in = k < end;
      pv[u] = (in && norm_prev) ? vp[k] : 0.0;
      jv[u] = in ? vj[k] : 0.0;
      uv[u] = (in && i > 0) ? vu[k] : 0.0;
      iv[u] = (in && load_i) ? vi[k] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < MB; ++u) {
      const int k = k0 + 32 * u;
      if (k < end) {
        double xp = 0.0;
        if (norm_prev) {
          xp = pv[u];
          if (nr > 0.0) {
            xp = xp * rn;
            vp[k] = xp;
          }
        }
        double y = jv[u];
        if (i > 0) {
          y = fma(-r, uv[u], y);
          vj[k] = y;
        }
        const double x = i == j ? y : (norm_prev && i == j - 1) ? xp : iv[u];
        s = fma(x, y, s);
      }
    }
  }
  return exchange32(s);
}

__global__ void __launch_bounds__(32) k_mgs_step(int n, int t, int nchunks, double *__restrict__ V, int j, int i,
                                                 double *__restrict__ sc, double *__restrict__ part,
                                                 unsigned *ticket) {
  pdl_wait();
  const long w = blockIdx.x;
  const int lane = threadIdx.x & 31;
  if (nchunks == 0) {
    if (lane == 0) sc[i < j ? i : t] = 0.0;
    return;
  }
  const double s = mgs_chunk(n, t, V, j, i, (int)w, sc, lane);
  dot_finish(w, 1, nchunks, part, ticket, lane, s, [&](int, double v) { sc[i < j ? i : t] = v; });
}

// The whole Gram-Schmidt pass in one cooperative launch: warps own chunks
// (chunk c belongs to warp c mod warps for every step), each step ends with a
// grid barrier after which every CTA adds the chunks' parts in order -- the
// additions of the last-warp sum above, so every CTA holds the same total,
// which is the value the launch-per-step form computes.  Barrier waits are
// bounded: one that runs out sets g_mgs_err and every CTA leaves.
__device__ int g_mgs_err;

__device__ __forceinline__ bool mgs_grid_sync(unsigned *bar, unsigned &gen, int *fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], gen + 1u);
    } else {
      const long long t0 = clock64();
      while (((volatile unsigned *)bar)[1] == gen) {
        if (*(volatile int *)&g_mgs_err || clock64() - t0 > (1LL << 32)) {
          atomicExch(&g_mgs_err, 1);
          *fail = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  ++gen;
  return *(volatile int *)fail == 0;
}

constexpr int MGS_WARPS = 2;  // small CTAs: the chunks spread over all SMs

__global__ void __launch_bounds__(32 * MGS_WARPS) k_mgs_coop(int n, int t, int nchunks, double *__restrict__ V,
                                                             double *__restrict__ part, unsigned *bar) {
  __shared__ double ssc[TMAXD + 1];
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) fail = 0;
  for (int q = threadIdx.x; q <= TMAXD; q += blockDim.x) ssc[q] = 0.0;
  __syncthreads();
  const int wg = blockIdx.x * MGS_WARPS + warp, nw = gridDim.x * MGS_WARPS;
  unsigned gen = 0;
  for (int j = 0; j < t; ++j)
    for (int i = 0; i <= j; ++i) {
      // the steps alternate between two halves of part: a CTA writes step
      // s + 1's parts only after the barrier of step s, and the next write
      // to the same half waits for the barrier of step s + 1, which every CTA
      // reaches only after reading step s's total
      double *ps = part + (size_t)(gen & 1u) * nchunks;
      for (int c = wg; c < nchunks; c += nw) {
        const double s = mgs_chunk(n, t, V, j, i, c, ssc, lane);
        if (lane == 0) ps[c] = s;
      }
      if (!mgs_grid_sync(bar, gen, &fail)) return;
      if (warp == 0) {
        const double tot = sum_chunks(ps, nchunks, lane);
        if (lane == 0) ssc[i < j ? i : t] = tot;
      }
      __syncthreads();
    }
  // the last column divided by its norm (as k_div_sqrt), each warp on the
  // chunks it owns (it alone wrote them)
  if (t > 0) {
    const double nr = sqrt(ssc[t]);
    if (nr > 0.0) {
      const double rn = 1.0 / nr;
      double *v = V + (size_t)(t - 1) * n;
      for (int c = wg; c < nchunks; c += nw)
        for (int k = c * CHUNK + lane; k < min(c * CHUNK + CHUNK, n); k += 32) v[k] = v[k] * rn;
    }
  }
}

int mgs(int n, int t, double *V, cudaStream_t s) {
  const int nchunks = (n + CHUNK - 1) / CHUNK;
  if (t > 0 && nchunks > 0 && !getenv("AMG_MGS_STEPS")) {
    // one cooperative launch for the whole pass (at most one CTA per two
    // chunks, every CTA resident at once)
    int dev = 0, nsm = 0, per = 0, coop = 0;
    AMG_CU(cudaGetDevice(&dev));
    AMG_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    AMG_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    AMG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mgs_coop, 32 * MGS_WARPS, 0));
    if (coop && per > 0) {
      int grid = (nchunks + MGS_WARPS - 1) / MGS_WARPS;
      if (grid > nsm * per) grid = nsm * per;
      DBuf<double> part;
      DBuf<unsigned> bar;
      AMG_TRY(part.alloc(2 * (size_t)nchunks));
      AMG_TRY(bar.alloc(2));
      AMG_TRY(bar.zero(s));
      void *args[] = {&n, &t, (void *)&nchunks, &V, &part.p, &bar.p};
      count_launches(1);
      AMG_CU(cudaLaunchCooperativeKernel((const void *)k_mgs_coop, dim3(grid), dim3(32 * MGS_WARPS), args, 0, s));
      AMG_CU(cudaStreamSynchronize(s));
      int err = 0;
      AMG_CU(cudaMemcpyFromSymbol(&err, g_mgs_err, sizeof(int)));
      if (err) {
        const int z = 0;
        cudaMemcpyToSymbol(g_mgs_err, &z, sizeof(int));
        set_error("Gram-Schmidt: a grid barrier wait ran out");
        return AMG_ERR_CUDA;
      }
      return AMG_OK;
    }
  }
  DBuf<double> sc, part;
  DBuf<unsigned> tk;
  AMG_TRY(sc.alloc(t + 1));
  AMG_TRY(part.alloc((size_t)nchunks + 1));
  AMG_TRY(tk.alloc(MAXTICKETS));
  AMG_TRY(tk.zero(s));
  for (int j = 0; j < t; ++j)
    for (int i = 0; i <= j; ++i)
      launch_k(k_mgs_step, nchunks > 0 ? nchunks : 1, 32, 0, s, n, t, nchunks, V, j, i, sc.p, part.p, tk.p);
  if (t > 0 && n > 0) launch_k(k_div_sqrt, nblk(n, 256), 256, 0, s, n, V + (size_t)(t - 1) * n, sc.p + t);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- FSAI
// Warp-cooperative aFSAI rows (NG node rows per warp, below).  The
// arithmetic of each scalar follows the plain sequential definition:
//  * Cholesky of A[Q,Q] entry (i,j): A_ij - sum_{k<j} L_ik L_jk (k ascending),
//    then sqrt / division (the right-looking update subtracts the same
//    products in the same order);
//  * forward substitution sums k ascending, backward substitution k
//    descending (the column-oriented forms subtract in the same orders);
//  * psi = a_ii + sum_a A[i,Q_a] gh_a, a ascending;
//  * candidate gradient (A gt)_j over the row pattern in ascending dof order;
//    node score = sum over rows c, dofs d of gradient^2, c outer.
struct FsaiK {
  int n;
  const int *Arp, *Acol;
  const double *Aval;
  const int *Atr;  // per stored block (i, j): the index of block (j, i)
  int compact;     // compact a row's candidate entries before taking them
  const int *Gsrp, *Gscol;
  int ksteps, rho, maxg;
  double eps;
  int *out_np, *out_pat;
  double *out_val;
  int *status;
  double *dscr;
  int *iscr;
  unsigned long long *htab;
  long dper, iper;
  int candcap, mmax, hcap;
};

template <int B>
__device__ __forceinline__ const double *find_blk(const int *rp, const int *col, const double *val, int i, int j) {
  int lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1, c = col[mid];
    if (c == j) return val + (size_t)mid * B * B;
    if (c < j) lo = mid + 1; else hi = mid - 1;
  }
  return nullptr;
}

// Lockstep slots.  Each warp works on NG node rows at once, 32 / NG lanes
// per row ("slot"); every loop that contains a warp-wide step runs to the
// warp's largest bound with the per-slot work predicated, so the FP64
// instructions of the sequential parts (square roots and divisions of the
// Cholesky factor and of the substitutions) serve NG rows each.  FP64 issue
// slots are the scarce resource of this GPU: a warp instruction costs the
// same with one lane active as with 32.  Large levels take NG = 4; small
// ones fewer rows per warp (more lanes per row), so that their few rows
// still reach every SM's FP64 pipes.  Every scalar gets the same operations
// in the same order whatever NG: lanes only share out independent entries.

__device__ __forceinline__ int warp_max(int v) {
  for (int off = 16; off >= 1; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// (rr, kk) with kk <= rr from the row-major index of a lower triangle
__device__ __forceinline__ void tri_decode(int idx, int &rr, int &kk) {
  int r = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= idx) ++r;
  while (r * (r + 1) / 2 > idx) --r;
  rr = r;
  kk = idx - r * (r + 1) / 2;
}

// Solve the B dof rows of node I on pattern pat[0..np-1] (slots with act;
// B = 3 for nodal blocks, B = 1 for the scalar method); returns 0 or an
// error, the same in every lane of a slot.  The system of dof row c is
// A[Q_c, Q_c] with Q_c = (pattern dofs, BI, ..., BI+c-1), so the systems of
// rows 0 .. B-2 are leading principal blocks of the system of row B-1: one
// Cholesky factor of the largest serves all B (entry (r,k) of a Cholesky
// factor depends only on the leading (r+1)x(r+1) block, so each row's factor
// is exactly what factoring it alone gives).  A is read one BxB block per
// node pair: the lower triangle of the largest system, rhs_c = -A[Q_c, BI+c]
// and ent_c = A[BI+c, Q_c].  Column j of the factor is scaled by
// rho_j = 1 / L_jj, which the diagonal then holds for the substitutions (a
// product per unknown instead of a division).
template <int B, int NG>
__device__ int fsai_solve_rows(const FsaiK &K, bool act, int I, const int *pat, int np, int r0, double *M, double *gh,
                               double *rhs, double *ent, double *psi, int g, int gl) {
  constexpr int GL = 32 / NG;
  // Rows [0, r0) of the factor in M (stride mmax) are kept from the previous
  // solve of this row: the pattern only grew at its end, and entry (r, k) of
  // a Cholesky factor depends only on the leading (r+1) x (r+1) block.  Only
  // rows r0.. (the new pattern dofs and the row's own dofs, which follow
  // them) are formed and factored.
  const int m2 = act ? B * np + (B - 1) : 0, mm = K.mmax, nn = np + 1;
  const int p0 = r0 / B;  // first node whose rows are new
  const int npairs = act ? nn * (nn + 1) / 2 : 0;
  for (int idx = p0 * (p0 + 1) / 2 + gl; idx < npairs; idx += GL) {
    int p, q;
    tri_decode(idx, p, q);
    const double *b = find_blk<B>(K.Arp, K.Acol, K.Aval, p < np ? pat[p] : I, q < np ? pat[q] : I);
    for (int a = 0; a < B; ++a) {
      const int r = B * p + a;
      if (r >= m2) break;
      for (int e = 0; e < B; ++e) {
        const int cc = B * q + e;
        if (cc <= r) M[r * mm + cc] = b ? b[a * B + e] : 0.0;
      }
    }
  }
  // right-hand sides and entries of the new nodes and of I (those of the
  // kept nodes are unchanged, and rhs holds their forward-substitution
  // values y from the previous solve)
  for (int idx = p0 + gl; idx < (act ? nn : 0); idx += GL) {
    const int Np = idx < np ? pat[idx] : I;
    const double *bc = find_blk<B>(K.Arp, K.Acol, K.Aval, Np, I);
    const double *br = find_blk<B>(K.Arp, K.Acol, K.Aval, I, Np);
    for (int a = 0; a < B; ++a) {
      const int qa = B * idx + a;
      for (int c = 0; c < B; ++c)
        if (qa < B * np + c) {
          rhs[c * mm + qa] = -(bc ? bc[a * B + c] : 0.0);
          ent[c * mm + qa] = br ? br[c * B + a] : 0.0;
        }
    }
  }
  __syncwarp();
  // right-looking Cholesky of the lower triangle in panels of FS_PB columns
  // (each entry receives its updates k = 0, 1, ... in ascending order, then
  // the scaling by its column's reciprocal pivot, exactly as column by
  // column): inside a panel column by column; the trailing entries then
  // receive the panel's FS_PB updates in one pass, reading each of their two
  // panel rows once.  Columns below r0 already hold their reciprocal pivots:
  // only the new rows take their scalings and updates.
  constexpr int FS_PB = 8;
  const int mx = warp_max(m2);
  int bad = 0;
  for (int j0 = 0; j0 < mx; j0 += FS_PB) {
    const int j1 = min(j0 + FS_PB, m2);  // this slot's panel end
    for (int j = j0; j < j0 + FS_PB && j < mx; ++j) {
      const bool on = j < m2 && !bad;
      const bool kept = j < r0;  // pivot of a kept row
      double rho = 1.0;
      if (on) {
        const double sjj = M[j * mm + j];
        if (kept) rho = sjj;
        else if (!(sjj > 0.0)) bad = 1;
        else rho = 1.0 / sqrt(sjj);
      }
      __syncwarp();
      const int rb = max(j + 1, r0);  // first row this column updates
      if (on && !bad) {
        for (int r = rb + gl; r < m2; r += GL) M[r * mm + j] = M[r * mm + j] * rho;
        if (gl == 0 && !kept) M[j * mm + j] = rho;  // the diagonal holds 1 / L_jj
      }
      __syncwarp();
      if (on && !bad) {  // the panel's later columns, rows max(k, r0)..m2-1
        const int pk = j1 - j - 1;
        for (int idx = gl; idx < pk * (m2 - rb); idx += GL) {
          const int k = j + 1 + idx % pk, r = rb + idx / pk;
          if (r >= k) M[r * mm + k] = fma(-M[r * mm + j], M[k * mm + j], M[r * mm + k]);
        }
      }
      __syncwarp();
    }
    if (!bad && j1 < m2 && j0 < m2) {  // trailing rows max(j1, r0).. from column j1
      const int w = m2 - j1, nt = w * (w + 1) / 2;
      const int rb = max(r0, j1) - j1, t0 = rb * (rb + 1) / 2;
      for (int idx = t0 + gl; idx < nt; idx += GL) {
        int rr, kk;
        tri_decode(idx, rr, kk);
        const int r = j1 + rr, k = j1 + kk;
        double a = M[r * mm + k];
        for (int j = j0; j < j1; ++j) a = fma(-M[r * mm + j], M[k * mm + j], a);
        M[r * mm + k] = a;
      }
    }
    __syncwarp();
  }
  const bool ok = act && !bad;
  // forward substitution for the B right-hand sides together (row c
  // uses the leading B np + c rows): y_k = rhs_k (1 / L_kk), then rhs_r -= L_rk y_k
  // (k ascending for every r), in blocks of FS_PB columns: inside a block
  // column by column, then the rows below it take the block's updates in
  // one pass.  Rows below r0 already hold their y (a leading block of a
  // triangular solve does not depend on the rows after it); the new rows
  // take every update, from the kept columns too, in the same order.
  for (int k0 = 0; k0 < mx; k0 += FS_PB) {
    const int k1 = min(k0 + FS_PB, mx);
    for (int k = k0; k < k1; ++k) {
      if (ok && gl < B && k >= r0 && k < B * np + gl) rhs[gl * mm + k] = rhs[gl * mm + k] * M[k * mm + k];
      __syncwarp();
      const int rs = max(k + 1, r0), nr = k1 - rs;
      if (ok && nr > 0)
        for (int idx = gl; idx < B * nr; idx += GL) {
          const int c = idx / nr, r = rs + idx % nr;
          if (r < B * np + c) rhs[c * mm + r] = fma(-M[r * mm + k], rhs[c * mm + k], rhs[c * mm + r]);
        }
      __syncwarp();
    }
    const int rs2 = max(k1, r0), nr2 = m2 - rs2;
    if (ok && nr2 > 0)
      for (int idx = gl; idx < B * nr2; idx += GL) {
        const int c = idx / nr2, r = rs2 + idx % nr2;
        if (r < B * np + c) {
          double a = rhs[c * mm + r];
          for (int k = k0; k < k1; ++k) a = fma(-M[r * mm + k], rhs[c * mm + k], a);
          rhs[c * mm + r] = a;
        }
      }
    __syncwarp();
  }
  // backward substitution on a copy of y (rhs keeps y for the next solve of
  // this row): x_k = w_k (1 / L_kk) for k descending, then w_r -= L_kr x_k
  // for r < k (k descending for every r), in blocks of FS_PB columns from
  // the top; w and then x live in gh
  if (ok)
    for (int idx = gl; idx < B * m2; idx += GL) {
      const int c = idx / m2, k = idx % m2;
      if (k < B * np + c) gh[c * mm + k] = rhs[c * mm + k];
    }
  __syncwarp();
  for (int k1 = mx; k1 > 0; k1 -= FS_PB) {
    const int k0 = max(k1 - FS_PB, 0);
    for (int k = k1 - 1; k >= k0; --k) {
      if (ok && gl < B && k < B * np + gl) gh[gl * mm + k] = gh[gl * mm + k] * M[k * mm + k];
      __syncwarp();
      if (ok && k < m2)
        for (int idx = gl; idx < B * (k - k0); idx += GL) {
          const int c = idx / (k - k0), r = k0 + idx % (k - k0);
          if (k < B * np + c) gh[c * mm + r] = fma(-M[k * mm + r], gh[c * mm + k], gh[c * mm + r]);
        }
      __syncwarp();
    }
    if (ok)
      for (int idx = gl; idx < B * k0; idx += GL) {
        const int c = idx / k0, r = idx % k0;
        double a = gh[c * mm + r];
        for (int k = min(k1, B * np + c) - 1; k >= k0; --k) a = fma(-M[k * mm + r], gh[c * mm + k], a);
        gh[c * mm + r] = a;
      }
    __syncwarp();
  }
  // psi_c = a_ii + sum_a A[i, Q_a] gh_a (a ascending), i = B I + c
  double sv = 0.0;
  if (ok && gl < B) {
    const int c = gl;
    const double *bii = find_blk<B>(K.Arp, K.Acol, K.Aval, I, I);
    sv = bii ? bii[c * B + c] : 0.0;
    for (int a = 0; a < B * np + c; ++a) sv = fma(ent[c * mm + a], gh[c * mm + a], sv);
  }
  double ps[B];
  for (int c = 0; c < B; ++c) ps[c] = __shfl_sync(0xffffffffu, sv, g * GL + c);
  __syncwarp();
  if (!act) return AMG_OK;
  if (bad) return AMG_ERR_NOT_SPD;
  for (int c = 0; c < B; ++c) {
    if (!(ps[c] > 0.0)) return AMG_ERR_NOT_SPD;
    psi[c] = ps[c];
  }
  return AMG_OK;
}

__device__ __forceinline__ int in_sorted(const int *a, int n, int v) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] == v) return 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid - 1;
  }
  return 0;
}

// Find or insert J in a slot's open-addressing set for one (node, step);
// entries of earlier uses (another stamp) count as free.  Returns J's table
// position (and whether it was new), -1 if the table had no room (it holds
// at least twice as many entries as the step can insert).
__device__ __forceinline__ int set_find_insert(unsigned long long *tab, int cap, unsigned stamp, int J, bool &isnew) {
  const unsigned long long key = ((unsigned long long)stamp << 32) | (unsigned)J;
  unsigned h = ((unsigned)J * 2654435761u) & (unsigned)(cap - 1);
  isnew = false;
  for (int probe = 0; probe < cap; ++probe) {
    unsigned long long cur = ((volatile unsigned long long *)tab)[h];
    for (int tries = 0; (unsigned)(cur >> 32) != stamp && tries < 64; ++tries) {
      const unsigned long long prev = atomicCAS(&tab[h], cur, key);
      if (prev == cur) {
        isnew = true;
        return (int)h;
      }
      cur = prev;
    }
    if ((unsigned)(cur >> 32) == stamp && (unsigned)cur == (unsigned)J) return (int)h;
    h = (h + 1) & (unsigned)(cap - 1);
  }
  return -1;
}

// Index of the transposed block of every stored block (one warp per row):
// tr[k] = position of block (j, i) for block k = (i, j); a block without a
// transposed partner sets *asym.
__global__ void k_block_transpose_index(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                        int *__restrict__ tr, int *__restrict__ asym) {
  pdl_wait();
  const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int k = rp[i] + lane; k < rp[i + 1]; k += 32) {
    const int j = col[k];
    int lo = rp[j], hi = rp[j + 1] - 1, at = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1, c = col[mid];
      if (c == i) {
        at = mid;
        break;
      }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    tr[k] = at;
    if (at < 0) atomicExch(asym, 1);
  }
}

template <int B, int NG>
__global__ void __launch_bounds__(128) k_fsai(FsaiK K) {
  constexpr int GL = 32 / NG;
  static_assert(GL >= B, "a slot needs a lane per dof row of a node");
  constexpr unsigned lowmask = GL == 32 ? 0xffffffffu : ((1u << (GL & 31)) - 1u);
  const unsigned smask = lowmask << ((threadIdx.x & 31) / GL * GL);
  const int lane = threadIdx.x & 31, g = lane / GL, gl = lane % GL;
  const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  const long slot = gw * NG + g, nslots = nw * NG;
  const int mm = K.mmax;
  double *M = K.dscr + slot * K.dper;
  double *gh = M + (size_t)mm * mm;
  double *rhs = gh + B * mm;
  double *ent = rhs + B * mm;
  double *score = ent + B * mm;
  double *acc = score + K.candcap;  // per candidate: its B x B gradient sums
  int *pat = K.iscr + slot * K.iper;  // pattern in the order the nodes were added
  int *cand = pat + K.maxg + 1;
  int *ccount = cand + K.candcap;
  int *spat = ccount + 1;  // the same nodes in ascending order (membership tests)
  int *bidx = spat + K.maxg + 1;  // per candidate: its block (J, I), or -1
  int *hidx = bidx + K.candcap;   // per table position: the candidate index
  unsigned long long *tab = K.htab + slot * K.hcap;
  const long nrounds = (K.n + nslots - 1) / nslots;
  for (long rd = 0; rd < nrounds; ++rd) {
    // every lane has finished the previous row (its output reads the slot's
    // pattern arrays) before the first lane writes the next row's pattern
    __syncwarp();
    const long Il = rd * nslots + slot;
    const bool have = Il < K.n;
    const int I = have ? (int)Il : 0;
    int np = 0;
    if (have && gl == 0 && K.Gsrp) {
      for (int k = K.Gsrp[I]; k < K.Gsrp[I + 1]; ++k)
        if (K.Gscol[k] != I && np < K.maxg) {
          pat[np] = K.Gscol[k];  // a row of G_s: ascending
          spat[np] = K.Gscol[k];
          ++np;
        }
    }
    np = __shfl_sync(0xffffffffu, np, g * GL);
    __syncwarp();
    double psi[3] = {0.0, 0.0, 0.0}, psi_old[3];
    int rc = fsai_solve_rows<B, NG>(K, have, I, pat, np, 0, M, gh, rhs, ent, psi, g, gl);
    bool active = have && rc == 0;
    for (int step = 0; step < K.ksteps; ++step) {
      if (active && np >= K.maxg) active = false;
      if (!__any_sync(0xffffffffu, active)) break;
      // candidates: A-neighbours J < I of the pattern nodes and of I, outside
      // the pattern, each once (set of this node and step)
      const unsigned stamp = (unsigned)(rd * (K.ksteps + 1) + step + 1);
      if (gl == 0) *ccount = 0;
      __syncwarp();
      // gradient entries g[c][d] = (A gt_c)_{BJ+d}: the pattern dofs in the
      // pattern's order, then the dofs BI+e < BI+c, then the unit entry; node
      // score = sum over c, d of g^2.  The rows of the pattern nodes are
      // walked in the pattern's order (lanes over a row's entries, which name
      // distinct nodes), so every candidate's sums take their terms in that
      // order; the row of I then records each candidate's block (J, I).  The
      // block (J, K) of entry (K, J) comes from the transposed-block index.
      if (active)
        for (int run = 0; run <= np; ++run) {
          const int Kn = run < np ? pat[run] : I;
          const int b0 = K.Arp[Kn], len = K.Arp[Kn + 1] - b0;
          // one candidate entry e of the row (J = its column): its slot and
          // its gradient term
          auto take = [&](int e, int J) {
              bool isnew;
              const int h = set_find_insert(tab, K.hcap, stamp, J, isnew);
              if (h < 0) return;
              int idx;
              if (isnew) {
                idx = atomicAdd(ccount, 1);
                cand[idx] = J;
                hidx[h] = idx;
                bidx[idx] = -1;
                for (int q = 0; q < B * B; ++q) acc[(size_t)idx * B * B + q] = 0.0;
              } else {
                idx = hidx[h];
              }
              const int kt = K.Atr[b0 + e];
              if (run == np) {
                bidx[idx] = kt;
              } else if (kt >= 0) {
                const double *blk = K.Aval + (size_t)kt * B * B;
                double *a = acc + (size_t)idx * B * B;
                for (int c = 0; c < B; ++c)
                  for (int d = 0; d < B; ++d) {
                    double gs = a[c * B + d];
                    for (int q = 0; q < B; ++q) gs = fma(blk[d * B + q], gh[c * mm + B * run + q], gs);
                    a[c * B + d] = gs;
                  }
              }
          };
          if (K.compact) {
            // the row's entries that name candidates (J < I, outside the
            // pattern), compacted in the (still unused) score array so that
            // the lanes then take one candidate entry each
            int *elist = reinterpret_cast<int *>(score);
            int nq = 0;
            for (int e0 = 0; e0 < len; e0 += GL) {
              const int e = e0 + gl;
              bool c = false;
              if (e < len) {
                const int J = K.Acol[b0 + e];
                c = J < I && !in_sorted(spat, np, J);
              }
              const unsigned m = (__ballot_sync(smask, c) >> (g * GL)) & lowmask;
              if (c) elist[nq + __popc(m & ((1u << gl) - 1u))] = e;
              nq += __popc(m);
            }
            __syncwarp(smask);
            for (int u = gl; u < nq; u += GL) {
              const int e = elist[u];
              const int J = K.Acol[b0 + e];
              take(e, J);
            }
          } else {
            for (int e = gl; e < len; e += GL) {
              const int J = K.Acol[b0 + e];
              if (J >= I || in_sorted(spat, np, J)) continue;
              take(e, J);
            }
          }
          __syncwarp(smask);  // a later row may name the same candidates
        }
      __syncwarp();
      const int nc = active ? *(volatile int *)ccount : 0;
      for (int t = gl; t < nc; t += GL) {
        const double *a = acc + (size_t)t * B * B;
        const double *bI = bidx[t] >= 0 ? K.Aval + (size_t)bidx[t] * B * B : nullptr;
        double sc = 0.0;
        for (int c = 0; c < B; ++c)
          for (int d = 0; d < B; ++d) {
            double gv = a[c * B + d];
            if (bI) {
              for (int q = 0; q < c; ++q) gv = fma(bI[d * B + q], gh[c * mm + B * np + q], gv);
              gv = gv + bI[d * B + c] * 1.0;
            }
            sc = fma(gv, gv, sc);
          }
        score[t] = sc;
      }
      __syncwarp();
      // the rho best (score > 0, ties to the smaller node), by slot.  Scores
      // are sums of squares (>= +0), whose IEEE bit patterns order like
      // 64-bit integers, so the selection compares integers (the same
      // decisions; a double compare would take an FP64 issue slot); a taken
      // candidate gets the pattern of -1.0 (negative as an integer).
      const int want = active ? (K.rho < K.maxg - np ? K.rho : K.maxg - np) : 0;
      const int wmax = warp_max(want);
      int got = 0;
      bool more = true;
      for (int p = 0; p < wmax; ++p) {
        long long bs = -1;
        int bj = 0x7fffffff, bt = -1;
        if (more && p < want)
          for (int t = gl; t < nc; t += GL) {
            const long long sc = __double_as_longlong(score[t]);
            if (sc > 0 && (sc > bs || (sc == bs && cand[t] < bj))) { bs = sc; bj = cand[t]; bt = t; }
          }
        for (int off = GL / 2; off >= 1; off >>= 1) {
          const long long os = __shfl_xor_sync(0xffffffffu, bs, off);
          const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
          const int ot = __shfl_xor_sync(0xffffffffu, bt, off);
          if (os > bs || (os == bs && oj < bj)) { bs = os; bj = oj; bt = ot; }
        }
        if (more && p < want) {
          if (bt < 0) {
            more = false;
          } else {
            if (gl == 0) {
              pat[np + got] = bj;
              score[bt] = -1.0;
            }
            ++got;
          }
        }
        __syncwarp();
      }
      if (active && got == 0) active = false;
      if (active && gl == 0) {  // the new nodes stay at the end of pat; spat takes them in order
        for (int u = np; u < np + got; ++u) {
          const int v = pat[u];
          int w = u - 1;
          while (w >= 0 && spat[w] > v) { spat[w + 1] = spat[w]; --w; }
          spat[w + 1] = v;
        }
      }
      const int np_old = np;
      if (active) np += got;
      __syncwarp();
      for (int c = 0; c < B; ++c) psi_old[c] = psi[c];
      const int rc2 = fsai_solve_rows<B, NG>(K, active, I, pat, np, B * np_old, M, gh, rhs, ent, psi, g, gl);
      if (active) {
        if (rc2) {
          rc = rc2;
          active = false;
        } else {
          int stalled = 1;
          for (int c = 0; c < B; ++c)
            if (psi_old[c] - psi[c] > K.eps * psi_old[c]) stalled = 0;
          if (stalled) active = false;
        }
      }
    }
    if (!have) continue;
    if (rc) {
      if (gl == 0) atomicMin(K.status, rc);
      continue;
    }
    // G row in ascending node order: ord[j] = position in pat of spat[j]
    int *ord = cand;  // free once the steps are done
    for (int j = gl; j < np; j += GL) {
      const int v = spat[j];
      for (int q = 0; q < np; ++q)
        if (pat[q] == v) ord[j] = q;
    }
    __syncwarp(smask);  // only this slot's lanes are here
    if (gl == 0) K.out_np[I] = np;
    for (int j = gl; j < np; j += GL) K.out_pat[(size_t)I * K.maxg + j] = spat[j];
    double rs[B];  // 1 / sqrt(psi_c): one division per row, products per entry
    for (int c = 0; c < B; ++c) rs[c] = 1.0 / sqrt(psi[c]);
    double *ov = K.out_val + (size_t)I * (K.maxg + 1) * B * B;
    for (int idx = gl; idx < (np + 1) * B * B; idx += GL) {
      const int j = idx / (B * B), c = (idx % (B * B)) / B, d = idx % B;
      double gv;
      if (j < np) gv = gh[c * mm + B * ord[j] + d];
      else gv = (d < c) ? gh[c * mm + B * np + d] : (d == c ? 1.0 : 0.0);
      ov[idx] = (j < np || d <= c) ? gv * rs[c] : 0.0;
    }
  }
}

int fsai(const DevBsr &A, const DevBsr *Gs, int ksteps, int rho, double eps, int maxg, int maxdeg,
         FsaiOut out, int *status, cudaStream_t s) {
  FsaiK K{};
  K.n = A.nr;
  K.Arp = A.rowptr.p;
  K.Acol = A.col.p;
  K.Aval = A.val.p;
  K.Gsrp = Gs ? Gs->rowptr.p : nullptr;
  K.Gscol = Gs ? Gs->col.p : nullptr;
  K.ksteps = ksteps;
  K.rho = rho;
  K.maxg = maxg;
  K.eps = eps;
  K.out_np = out.np;
  K.out_pat = out.pat;
  K.out_val = out.val;
  K.status = status;
  // the largest pattern a row can reach: its starting pattern (a row of Gs
  // without the diagonal) plus rho nodes per step, at most maxg; the row
  // systems, candidate lists and hash sets are sized by it (the hash sets
  // are probed at random positions, so smaller ones stay in L2)
  long npcap = (long)ksteps * rho;
  if (Gs) {  // a row of G_s holds its pattern nodes and the diagonal
    int len = 0;
    AMG_TRY(Gs->row_max(s, &len));
    npcap += len > 0 ? len - 1 : 0;
  }
  if (npcap > maxg) npcap = maxg;
  K.mmax = A.b * (int)npcap + A.b;
  K.candcap = ((int)npcap + 1) * maxdeg;
  K.hcap = 64;
  while (K.hcap < 2 * K.candcap) K.hcap *= 2;
  K.dper = (long)K.mmax * K.mmax + 3L * A.b * K.mmax + K.candcap + (long)K.candcap * A.b * A.b;
  K.iper = (maxg + 1) + K.candcap + 1 + (maxg + 1) + K.candcap + K.hcap;
  // transposed-block index of A (the level matrices have symmetric patterns;
  // a pattern that is not is refused)
  DBuf<int> atr, asym;
  AMG_TRY(atr.alloc(A.nnzb));
  AMG_TRY(asym.alloc(1));
  AMG_TRY(asym.zero(s));
  if (A.nr) launch_k(k_block_transpose_index, (int)((32L * A.nr + 255) / 256), 256, 0, s, A.nr, A.rowptr.p,
                                                                                          A.col.p, atr.p, asym.p);
  AMG_LAUNCH_CHECK();
  {
    int ha = 0;
    AMG_CU(cudaMemcpyAsync(&ha, asym.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
    if (ha) {
      set_error("aFSAI: the matrix pattern is not symmetric");
      return AMG_ERR_ARG;
    }
  }
  K.Atr = atr.p;
  // long rows (coarse levels): most entries of a row are skipped by some
  // lane, so the candidate entries are compacted first (measured: faster on
  // the beam's levels 1-3, slower on its level 0 with rows of 27 blocks)
  K.compact = maxdeg >= 40;
  int dev = 0, nsm = 0;
  AMG_CU(cudaGetDevice(&dev));
  AMG_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // rows per warp: 4 while that still gives 32 warps per SM, else 2, else 1;
  // and 1 on levels with rows of 40 blocks or more, whose walks fill a whole
  // warp (measured first aFSAI pass on the beam's levels: 139k rows of at
  // most 27 blocks 15.1 ms with 4, 15.6 with 8, 16.6 with 2, 23.1 with 1;
  // 30k rows of 47 blocks on average 4.2 ms with 1, 4.9 with 2, 5.1 with 4, 5.5
  // with 8; 6.2k rows 1.2 with 1, 2.4 with 4; 1.3k rows 0.6 with 1, 2.4
  // with 4)
  int ng = 4;
  while (ng > 1 && (long)A.nr / ng < 32L * nsm) ng /= 2;
  if (K.compact) ng = 1;
  if (const char *e = getenv("AMG_FSAI_NG")) {
    const int v = atoi(e);
    if (v == 1 || v == 2 || v == 4 || v == 8) ng = v;
  }
  const void *fn = nullptr;
  if (A.b == 1)
    fn = ng == 8 ? (const void *)k_fsai<1, 8> : ng == 4 ? (const void *)k_fsai<1, 4>
       : ng == 2 ? (const void *)k_fsai<1, 2> : (const void *)k_fsai<1, 1>;
  else
    fn = ng == 8 ? (const void *)k_fsai<3, 8> : ng == 4 ? (const void *)k_fsai<3, 4>
       : ng == 2 ? (const void *)k_fsai<3, 2> : (const void *)k_fsai<3, 1>;
  const int threads = 128;
  int per_sm = 0;
  AMG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0));
  long nblocks = (long)nsm * (per_sm > 0 ? per_sm : 1);
  const long need = ((long)A.nr + 4 * ng - 1) / (4 * ng);
  if (nblocks > need) nblocks = need > 0 ? need : 1;
  const long nslots = nblocks * (threads / 32) * ng;
  DBuf<double> ds;
  DBuf<int> is;
  DBuf<unsigned long long> hs;
  AMG_TRY(ds.alloc((size_t)nslots * K.dper));
  AMG_TRY(is.alloc((size_t)nslots * K.iper));
  AMG_TRY(hs.alloc((size_t)nslots * K.hcap));
  AMG_TRY(hs.zero(s));
  K.dscr = ds.p;
  K.iscr = is.p;
  K.htab = hs.p;
  void *args[] = {&K};
  count_launches(1);
  AMG_CU(cudaLaunchKernel(fn, dim3((unsigned)nblocks), dim3(threads), args, 0, s));
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- Lanczos
// largest eigenvalue of the tridiagonal (alpha, beta) by bisection on Sturm
// counts; out = [lambda, 2/lambda, min(1, safety * 2/lambda)].
//
// One warp.  The bisection is a walk down a binary tree whose nodes are the
// intervals it can visit; each round the 31 lanes take the 31 nodes of the
// next five levels below the current interval (heap order: node q has
// children 2q+1, holding the lower half, and 2q+2), replay the midpoints on
// the path to their node, and form the Sturm count at its midpoint; the walk
// then takes five steps using those counts.  Every midpoint and count is the
// one the step-by-step bisection forms, so the result is the same number.
//
// The Sturm count is the number of sign changes among the leading principal
// minors of T - x I, q_0 = 1, q_1 = a_0 - x,
// q_{i+1} = (a_i - x) q_i - b_{i-1}^2 q_{i-1}: no division (a division costs
// about ten FP64 issue slots).  A zero minor becomes q_{i-1} 2^-200 (it keeps
// the previous sign and the next minor records the change); a minor whose
// binary exponent leaves [-512, 511] is multiplied, with its predecessor, by
// 2^-512 or 2^512 (exact, signs unchanged).
__device__ __forceinline__ int sturm_count(int mm, const double *al, const double *bb, double x) {
  int cnt = 0;
  double qp = 1.0, q = 1.0;
  for (int i = 0; i < mm; ++i) {
    double qn = (i == 0) ? (al[0] - x) : (al[i] - x) * q - bb[i - 1] * qp;
    if (qn == 0.0) qn = q * 0x1p-200;
    if ((qn < 0.0) != (q < 0.0)) ++cnt;
    qp = q;
    q = qn;
    const int e = (int)((__double_as_longlong(q) >> 52) & 0x7ff) - 1023;
    if (e > 511) {
      q = q * 0x1p-512;
      qp = qp * 0x1p-512;
    } else if (e < -512) {
      q = q * 0x1p512;
      qp = qp * 0x1p512;
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(32) k_lanczos_bisect(int m, const double *__restrict__ sc, double safety,
                                                       double *__restrict__ out) {
  pdl_wait();
  __shared__ double al[64], be[64], bb[64];
  const int lane = threadIdx.x;
  for (int i = lane; i < 64; i += 32) {
    al[i] = sc[i];
    be[i] = sc[64 + i];
    bb[i] = be[i] * be[i];
  }
  __syncwarp();
  const int mm = sc[128] < 0.0 ? m : (int)sc[128];
  double lo = al[0], hi = al[0];
  for (int i = 0; i < mm; ++i) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < mm - 1 ? fabs(be[i]) : 0.0);
    if (al[i] - r < lo) lo = al[i] - r;
    if (al[i] + r > hi) hi = al[i] + r;
  }
  int it = 0;
  bool done = false;
  while (!done && it < 200) {
    int qok = 0, qcnt = 0;
    double qmid = 0.0;
    if (lane < 31) {
      const int h = lane + 1, lev = 31 - __clz(h);
      double ql = lo, qh = hi;
      qok = 1;
      for (int b = lev - 1; b >= 0; --b) {
        const double md = 0.5 * (ql + qh);
        if (!(md > ql && md < qh)) {
          qok = 0;
          break;
        }
        if ((h >> b) & 1)
          ql = md;
        else
          qh = md;
      }
      if (qok) {
        qmid = 0.5 * (ql + qh);
        qok = qmid > ql && qmid < qh;
        if (qok) qcnt = sturm_count(mm, al, bb, qmid);
      }
    }
    int node = 0;
    for (int l = 0; l < 5 && it < 200; ++l) {
      const int ok = __shfl_sync(0xffffffffu, qok, node);
      const double md = __shfl_sync(0xffffffffu, qmid, node);
      const int cnt = __shfl_sync(0xffffffffu, qcnt, node);
      if (!ok) {
        done = true;
        break;
      }
      if (cnt >= mm) {
        hi = md;
        node = 2 * node + 1;
      } else {
        lo = md;
        node = 2 * node + 2;
      }
      ++it;
    }
  }
  if (lane == 0) {
    const double w = 2.0 / hi;
    double om = safety * w;
    if (om > 1.0) om = 1.0;
    out[0] = hi;
    out[1] = w;
    out[2] = om;
  }
}

__global__ void k_set_neg(double *p) {
  pdl_wait(); *p = -1.0; }

__global__ void k_lanczos_start(long n, uint64_t seed, uint64_t base, double *__restrict__ v) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = uniform_pm1(seed, base | (uint64_t)i);
}

// ---------------------------------------------------------------- SRQCG
// Scalar slots of the SRQCG state (device doubles).
enum { S_A = 0, S_B, S_C, S_D, S_E, S_ALPHA, S_FN, S_ZSZ, S_Q, S_GSP, S_BETA, S_TMP, S_F0 = 16 };

// Step length along p (Algorithm 4): root of
// (bc - ad) alpha^2 + (bf - de) alpha + (af - ce) = 0 giving the smaller
// Rayleigh quotient; same expression order as the reference definition.
__device__ double line_min(double a, double b, double c, double d, double e, double f) {
  const double p1 = d * e - b * f;
  const double q1 = b * c - a * d;
  const double r1 = a * f - c * e;
  const double delta = p1 * p1 - (4.0 * q1) * r1;
  if (q1 != 0.0 && delta >= 0.0) {
    const double sq = sqrt(delta);
    const double a1 = (p1 + sq) / (2.0 * q1), a2 = (p1 - sq) / (2.0 * q1);
    const double n1 = (e + (2.0 * a1) * a) + (a1 * a1) * b, d1 = (f + (2.0 * a1) * c) + (a1 * a1) * d;
    const double n2 = (e + (2.0 * a2) * a) + (a2 * a2) * b, d2 = (f + (2.0 * a2) * c) + (a2 * a2) * d;
    return (n1 / d1 <= n2 / d2) ? a1 : a2;
  }
  if (q1 == 0.0 && p1 != 0.0) return r1 / p1;
  return 0.0;
}

// Batched column kernels: the n_tv columns of Algorithm 4 are updated
// independently of one another, so column j of every n x t block is handled by
// the same per-entry arithmetic as one column at a time.  Per-column scalars
// live in cs[] (layout below) and the skip flags in skip[].
enum { C_ALPHA = 0, C_Q = 1, C_FN = 2, C_BETA = 3, C_B = 4, C_F = 5, C_RF = 6, C_NUM = 7 };

__global__ void k_b_z0(long nt, double *__restrict__ z, const double *__restrict__ v, const double *__restrict__ sv) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nt) z[i] = v[i] - sv[i];
}

// p = 2 (S z - q z) with q = out[j] (the first quotients, f = 1)
__global__ void k_b_p0(long n, int t, double *__restrict__ p, const double *__restrict__ z,
                       const double *__restrict__ sz, const double *__restrict__ q) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  const int j = (int)(i / n);
  p[i] = 2.0 * fma(-q[j], z[i], sz[i]);
}

// z += alpha p and, by linearity, S z += alpha S p
__global__ void k_b_zupd(long n, int t, double *__restrict__ z, const double *__restrict__ p,
                         double *__restrict__ sz, const double *__restrict__ sp, const double *__restrict__ cs,
                         const int *__restrict__ skip) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  const int j = (int)(i / n);
  if (skip[j]) return;
  const double al = cs[C_ALPHA * t + j];
  z[i] = fma(al, p[i], z[i]);
  sz[i] = fma(al, sp[i], sz[i]);
}

__global__ void k_b_grad(long n, int t, double *__restrict__ g, const double *__restrict__ sz,
                         const double *__restrict__ z, const double *__restrict__ cs, const int *__restrict__ skip) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  const int j = (int)(i / n);
  if (skip[j]) return;
  g[i] = (2.0 * fma(-cs[C_Q * t + j], z[i], sz[i])) * cs[C_RF * t + j];
}

// p = g + beta p and, by linearity, S p = S g + beta S p
__global__ void k_b_pupd(long n, int t, double *__restrict__ p, const double *__restrict__ g,
                         double *__restrict__ sp, const double *__restrict__ sg, double *__restrict__ cs,
                         const int *__restrict__ skip) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  const int j = (int)(i / n);
  if (skip[j]) return;
  const double be = cs[C_BETA * t + j];
  p[i] = fma(be, p[i], g[i]);
  sp[i] = fma(be, sp[i], sg[i]);
  if (i - (long)j * n == 0) cs[C_F * t + j] = cs[C_FN * t + j];
}

__global__ void k_fill(double *__restrict__ p, int n, double v) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Column dot products of n x t blocks: pair (kind, column j) is
// x_kind[:, j] . y_kind[:, j] in the fixed order; the last warp finishes the
// sums and the per-column scalar step of Algorithm 4 (fin).
enum { CF_NONE = 0, CF_ALPHA = 1, CF_Q = 2, CF_BETA = 3 };
struct CDot {
  const double *x[5];
  const double *y[5];
  long xs[5], ys[5];  // column strides of x and y (n, or 0 for one shared vector)
};

__global__ void __launch_bounds__(32) k_cdots(int n, int t, int nk, CDot a, double *__restrict__ part, unsigned *ticket,
                                              int nchunks, double *__restrict__ out, int fin, double *__restrict__ cs,
                                              int *__restrict__ skip) {
  pdl_wait();
  const int nd = nk * t;
  const long w = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const long total = nchunks > 0 ? (long)nchunks * nd : 1;
  if (w >= total) return;
  const bool last = dot_warp(
      w, n, nd, nchunks, part, ticket, lane,
      [&](int d, const double *&x, const double *&y) {
        const int kind = d / t, j = d - kind * t;
        x = a.x[kind] + j * a.xs[kind];
        y = a.y[kind] + j * a.ys[kind];
      },
      [&](int d, double v) { out[d] = v; });
  if (!last) return;
  // the sums were written by other warps: read them through L2
  auto o = [&](int k) { return __ldcg(out + k); };
  for (int j = lane; j < t; j += 32) {
    if (fin == CF_ALPHA) {  // out = a, b, c, d, e blocks of t
      const double bb = o(t + j);
      cs[C_B * t + j] = bb;
      if (!(bb > 0.0)) {
        skip[j] = 1;
      } else {
        skip[j] = 0;
        cs[C_ALPHA * t + j] = line_min(o(j), bb, o(2 * t + j), o(3 * t + j), o(4 * t + j), cs[C_F * t + j]);
      }
    } else if (fin == CF_Q) {  // out = f_new, z.Sz
      cs[C_FN * t + j] = o(j);
      cs[C_Q * t + j] = o(t + j) / o(j);
      cs[C_RF * t + j] = 1.0 / o(j);
    } else if (fin == CF_BETA) {  // out = g.Sp
      cs[C_BETA * t + j] = -(o(j) / cs[C_B * t + j]);
    }
  }
}

// y_j = A x_j for the t columns of n x t blocks, row sums in the fixed
// order.  rw block rows per warp (rw = 1 unless BS t <= 16): lane (g, j, r)
// computes dof row r of column j of the warp's block row g, so the lanes of
// a row walk the same blocks (the row's values are read once per lane group)
// and few lanes idle: with t = 10 columns a scalar row (BS = 1) fills 10
// lanes, three rows 30.  Every output is the same chain of fused
// multiply-adds whatever rw is.
template <int BS, int U>
__global__ void k_spmv_cols(int nr, int t, int rw, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ X, double *__restrict__ Y) {
  pdl_wait();
  const long n = (long)BS * nr;
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (rw > 1) {
    const int per = BS * t, g = lane / per, pr = lane - g * per;
    const long I = w * rw + g;
    if (g >= rw || I >= nr) return;
    const int j = pr / BS, r = pr - BS * j;
    Y[(size_t)j * n + BS * I + r] = row_chain<BS, U>(rowptr[I], rowptr[I + 1], r, col, val, X + (size_t)j * n, 0.0);
    return;
  }
  if (w >= nr) return;
  const int I = (int)w;
  const int kb = rowptr[I], ke = rowptr[I + 1];
  for (int pr = lane; pr < BS * t; pr += 32) {
    const int j = pr / BS, r = pr - BS * j;
    Y[(size_t)j * n + (long)BS * I + r] = row_chain<BS, U>(kb, ke, r, col, val, X + (size_t)j * n, 0.0);
  }
}

// X = X U for X = Z (blockIdx.y 0) and X = S Z (blockIdx.y 1)
__global__ void k_rotate(long n, int t, double *__restrict__ Z0, double *__restrict__ Z1,
                         const double *__restrict__ U) {
  pdl_wait();
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double *__restrict__ Z = blockIdx.y ? Z1 : Z0;
  double row[TMAXD];
  for (int j = 0; j < t; ++j) {
    double s = 0.0;
    for (int i = 0; i < t; ++i) s = fma(Z[(size_t)i * n + k], U[i * t + j], s);
    row[j] = s;
  }
  for (int j = 0; j < t; ++j) Z[(size_t)j * n + k] = row[j];
}

// Generalised eigenproblem H U = M U diag(lam) of the Ritz step, by one CTA of
// four warps (the factorisation and the back-transform on warp 0):
// M = L L^T (sub-diagonal entries scaled by 1 / L_jj, the triangular solves
// multiply by the reciprocals Ri); C = L^{-1} (L^{-1} H)^T symmetrised as (C + C^T) * 0.5; Jacobi
// sweeps in round-robin order (per round T/2 disjoint pairs from the circle
// method, rotations computed from the current C, then all column, all row
// and all W rotations applied) until the off-diagonal mass is negligible;
// eigenvalues sorted ascending (ties keep index order);
// U = L^{-T} W with each column signed so that its entry of largest magnitude
// (first on ties) is positive.  Lanes only split work between independent
// entries (rows of a rotation, columns of a triangular solve); every entry is
// computed by the same sequence of rounded operations as the sequential
// definition.  Scratch w holds 4 t*t + t doubles; returns 1 if M is not SPD.
__device__ int gen_eig_cta(int t, const double *H, const double *M, double *U, double *lam, double *w, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  __shared__ int sp[TMAXD / 2], sq[TMAXD / 2], sact[TMAXD / 2];
  __shared__ double scs[TMAXD / 2], ssn[TMAXD / 2];
  __shared__ int sbad;
  double *L = w, *W1 = w + t * t, *C = w + 2 * t * t, *Wv = w + 3 * t * t, *Ri = w + 4 * t * t;
  if (tid == 0) sbad = 0;
  __syncthreads();
  if (warp == 0) {
  for (int i = lane; i < t * t; i += 32) L[i] = 0.0;
  __syncwarp();
  for (int j = 0; j < t; ++j) {
    double sj = M[j * t + j];
    for (int k = 0; k < j; ++k) sj = fma(-L[j * t + k], L[j * t + k], sj);
    if (!(sj > 0.0)) {
      if (lane == 0) sbad = 1;
      break;
    }
    const double d = sqrt(sj), rho = 1.0 / d;
    for (int i = j + 1 + lane; i < t; i += 32) {
      double u = M[i * t + j];
      for (int k = 0; k < j; ++k) u = fma(-L[i * t + k], L[j * t + k], u);
      L[i * t + j] = u * rho;
    }
    if (lane == 0) {
      L[j * t + j] = d;
      Ri[j] = rho;
    }
    __syncwarp();
  }
  __syncwarp();
  if (!sbad) {
  for (int j = lane; j < t; j += 32)
    for (int i = 0; i < t; ++i) {
      double sv = H[i * t + j];
      for (int k = 0; k < i; ++k) sv = fma(-L[i * t + k], W1[k * t + j], sv);
      W1[i * t + j] = sv * Ri[i];
    }
  __syncwarp();
  for (int j = lane; j < t; j += 32)
    for (int i = 0; i < t; ++i) {
      double sv = W1[j * t + i];
      for (int k = 0; k < i; ++k) sv = fma(-L[i * t + k], C[k * t + j], sv);
      C[i * t + j] = sv * Ri[i];
    }
  __syncwarp();
  for (int q = lane; q < t * t; q += 32) {
    const int i = q / t, j = q % t;
    if (j < i) {
      const double v = (C[i * t + j] + C[j * t + i]) * 0.5;
      C[i * t + j] = v;
      C[j * t + i] = v;
    }
  }
  for (int q = lane; q < t * t; q += 32) Wv[q] = (q / t == q % t) ? 1.0 : 0.0;
  }  // not bad
  }  // warp 0
  __syncthreads();
  if (sbad) return 1;
  // Sweeps in round-robin order (T/2 disjoint pairs per round from the circle
  // method).  Per round: threads i < T/2 of warp 0 compute the rotation of
  // pair i from the current C (at the start of a sweep warp 2 forms the
  // off-diagonal and diagonal masses of the same C meanwhile, and the sweep
  // ends there if the off-diagonal mass is negligible); then warps 0-1
  // update C by 2 x 2 blocks (rows of pair I, columns of pair J), one lane
  // per block column: its two entries take the column rotation of pair J and
  // then the row rotation of pair I -- the operations of rotating all
  // columns and then all rows -- and the pivot entries of an active pair
  // become zero; warps 2-3 rotate the columns of W.
  const int T = t + (t & 1), hp = T / 2;
  __shared__ double s_off, s_dg;
  for (int sweep = 0; sweep < 100; ++sweep) {
    bool done_sw = false;
    for (int r = 0; r < T - 1; ++r) {
      if (tid < hp) {
        int p = 0, q = 0, act = 0;
        double c = 1.0, sn = 0.0;
        const int a = (tid == 0) ? 0 : 1 + (tid - 1 + r) % (T - 1);
        const int j2 = T - 1 - tid;
        const int b2 = (j2 == 0) ? 0 : 1 + (j2 - 1 + r) % (T - 1);
        p = a < b2 ? a : b2;
        q = a < b2 ? b2 : a;
        if (q < t) {
          const double apq = C[p * t + q];
          if (apq != 0.0) {
            // tangent sgn(d) a2 / (|d| + R): c = u / w, s = sgn(d) a2 / w
            const double d = C[q * t + q] - C[p * t + p], a2 = 2.0 * apq;
            const double R = sqrt(fma(a2, a2, d * d));
            const double u = fabs(d) + R;
            const double iw = 1.0 / sqrt(fma(a2, a2, u * u));
            c = u * iw;
            sn = (d >= 0.0 ? a2 : -a2) * iw;
            act = 1;
          }
        }
        sp[tid] = p;
        sq[tid] = q;
        sact[tid] = act;
        scs[tid] = c;
        ssn[tid] = sn;
      }
      if (r == 0 && tid == 64) {
        double off = 0.0, dg = 0.0;
        for (int p = 0; p < t; ++p) {
          dg = fma(C[p * t + p], C[p * t + p], dg);
          for (int q = p + 1; q < t; ++q) off = fma(C[p * t + q], C[p * t + q], off);
        }
        s_off = off;
        s_dg = dg;
      }
      __syncthreads();
      if (r == 0 && !(s_off > 1e-32 * s_dg)) {
        done_sw = true;
        break;
      }
      if (warp < 2) {
        // every lane of warps 0-1 takes the same number of passes (the
        // __syncwarp below is reached by all 32 lanes)
        for (int e0 = 0; e0 < 2 * hp * hp; e0 += 64) {
          const int e = e0 + tid;
          const bool task = e < 2 * hp * hp;
          const int b = task ? e >> 1 : 0, h = e & 1;
          const int I = b / hp, J = b % hp;
          const int pI = sp[I], qI = sq[I], pJ = sp[J], qJ = sq[J];
          const bool rI = sact[I] != 0, cJ = sact[J] != 0;
          const int col = h ? qJ : pJ;
          const bool hq = qI < t;  // row qI exists (q >= t only for an inactive pair, t odd)
          const bool live = task && col < t && (rI || cJ);
          double x_pp = 0.0, x_pq = 0.0, x_qp = 0.0, x_qq = 0.0;
          if (live) {
            x_pp = C[pI * t + pJ];
            x_qp = hq ? C[qI * t + pJ] : 0.0;
            if (qJ < t) {
              x_pq = C[pI * t + qJ];
              x_qq = hq ? C[qI * t + qJ] : 0.0;
            }
          }
          __syncwarp();  // the other lane of the block has read its inputs
          if (!live) continue;
          // column rotation of pair J, this lane's column, rows pI and qI
          double yp = h ? x_pq : x_pp, yq = h ? x_qq : x_qp;
          if (cJ) {
            const double c = scs[J], sn = ssn[J];
            if (h == 0) {
              yp = fma(c, x_pp, -(sn * x_pq));
              yq = fma(c, x_qp, -(sn * x_qq));
            } else {
              yp = fma(sn, x_pp, c * x_pq);
              yq = fma(sn, x_qp, c * x_qq);
            }
          }
          // row rotation of pair I
          double zp = yp, zq = yq;
          if (rI) {
            const double c = scs[I], sn = ssn[I];
            zp = fma(c, yp, -(sn * yq));
            zq = fma(sn, yp, c * yq);
          }
          if (I == J && rI) {  // pivot entries (pI, qI) and (qI, pI)
            if (h == 1) zp = 0.0;
            else zq = 0.0;
          }
          C[pI * t + col] = zp;
          if (hq) C[qI * t + col] = zq;
        }
      } else {
        for (int idx = tid - 64; idx < hp * t; idx += 64) {  // W: columns p_i, q_i, row k
          const int i = idx / t, k = idx - i * t;
          if (!sact[i]) continue;
          const double c = scs[i], sn = ssn[i];
          const int ip = k * t + sp[i], iq = k * t + sq[i];
          const double xp = Wv[ip], xq = Wv[iq];
          Wv[ip] = fma(c, xp, -(sn * xq));
          Wv[iq] = fma(sn, xp, c * xq);
        }
      }
      __syncthreads();
    }
    if (done_sw) break;
  }
  if (warp != 0) return 0;
  int order[TMAXD];
  for (int i = 0; i < t; ++i) order[i] = i;
  for (int i = 0; i < t; ++i) {
    int best = i;
    for (int j = i + 1; j < t; ++j)
      if (C[order[j] * t + order[j]] < C[order[best] * t + order[best]]) best = j;
    const int ti = order[best];
    for (int j = best; j > i; --j) order[j] = order[j - 1];
    order[i] = ti;
  }
  for (int jj = lane; jj < t; jj += 32) {
    const int j = order[jj];
    double col[TMAXD];
    lam[jj] = C[j * t + j];
    for (int i = t - 1; i >= 0; --i) {
      double sv = Wv[i * t + j];
      for (int k = t - 1; k > i; --k) sv = fma(-L[k * t + i], col[k], sv);
      col[i] = sv * Ri[i];
    }
    int im = 0;
    for (int i = 1; i < t; ++i)
      if (fabs(col[i]) > fabs(col[im])) im = i;
    const double sg = col[im] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < t; ++i) U[i * t + jj] = sg * col[i];
  }
  __syncwarp();
  return 0;
}

template <int BS>
static void spmv_cols_b(const DevBsr &A, int t, const double *X, double *Y, cudaStream_t s) {
  const int rw = BS * t <= 16 ? 32 / (BS * t) : 1;  // block rows per warp
  const long warps = ((long)A.nr + rw - 1) / rw;
  if (A.nr < SMALL_ROWS)
    launch_k(k_spmv_cols<BS, 4>, nblk(32L * warps, 256), 256, 0, s, A.nr, t, rw, A.rowptr.p, A.col.p, A.val.p, X, Y);
  else
    launch_k(k_spmv_cols<BS, 1>, nblk(32L * warps, 256), 256, 0, s, A.nr, t, rw, A.rowptr.p, A.col.p, A.val.p, X, Y);
}

int spmv_cols(const DevBsr &A, int t, const double *X, double *Y, cudaStream_t s) {
  if (A.nr == 0) return AMG_OK;
  if (A.b == 1) spmv_cols_b<1>(A, t, X, Y, s);
  else spmv_cols_b<3>(A, t, X, Y, s);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// S X = G A G^T X on t columns
static int apply_s_cols(const DevBsr &A, const DevBsr &G, const DevBsr &GT, int t, const double *X, double *Y,
                        double *T1, double *T2, cudaStream_t s) {
  AMG_TRY(spmv_cols(GT, t, X, T1, s));
  AMG_TRY(spmv_cols(A, t, T1, T2, s));
  AMG_TRY(spmv_cols(G, t, T2, Y, s));
  return AMG_OK;
}

static int cdots(int n, int t, int nk, const CDot &a, double *out, int fin, double *cs, int *skip, DotCtx ctx,
                 cudaStream_t s) {
  const int nchunks = (n + CHUNK - 1) / CHUNK;
  const long warps = nchunks > 0 ? (long)nchunks * nk * t : 1;
  launch_k(k_cdots, (int)warps, 32, 0, s, n, t, nk, a, ctx.part, ctx.ticket, nchunks, out, fin, cs,
                                                           skip);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int srqcg(const DevBsr &A, const DevBsr &G, const DevBsr &GT, int kmax, int k_ritz, int t, const double *V0, double *V,
          int *status, cudaStream_t s) {
  const int n = A.b * A.nr;
  if (t > TMAXD) {
    set_error("n_tv = %d exceeds the supported maximum %d", t, TMAXD);
    return AMG_ERR_ARG;
  }
  const size_t nt = (size_t)n * t;
  // S Z and S P are formed once and then carried by the recurrences of Z
  // and P (z += alpha p, p = g + beta p, Z = Z U are linear), so an
  // iteration applies S once, to the gradients
  DBuf<double> Zb, Pb, SZb, SPb, Gv, SG, T1, T2, cs, out, part, H, Mg, U, lam;
  DBuf<int> skip;
  DBuf<unsigned> tk;
  AMG_TRY(Zb.alloc(nt));
  AMG_TRY(Pb.alloc(nt));
  AMG_TRY(SZb.alloc(nt));
  AMG_TRY(SPb.alloc(nt));
  AMG_TRY(Gv.alloc(nt));
  AMG_TRY(SG.alloc(nt));
  AMG_TRY(T1.alloc(nt));
  AMG_TRY(T2.alloc(nt));
  struct Half {
    double *p;
  } Z{Zb.p}, P{Pb.p}, SZ{SZb.p}, SP{SPb.p};
  AMG_TRY(cs.alloc(C_NUM * t));
  AMG_TRY(out.alloc(5 * t));
  const int nchunks = (n + CHUNK - 1) / CHUNK;
  AMG_TRY(part.alloc((size_t)(nchunks + 1) * (t * (t + 1) + 5 * t + 8)));
  AMG_TRY(H.alloc(t * t));
  AMG_TRY(Mg.alloc(t * t));
  AMG_TRY(U.alloc(t * t));
  AMG_TRY(lam.alloc(t));
  AMG_TRY(skip.alloc(t));
  AMG_TRY(tk.alloc(MAXTICKETS));
  AMG_TRY(cs.zero(s));
  AMG_TRY(skip.zero(s));
  AMG_TRY(tk.zero(s));
  const DotCtx ctx{part.p, tk.p};
  const int nb = nblk((long)nt, 256);
  // Z0 = (I - S) V0, orthonormalised
  AMG_TRY(apply_s_cols(A, G, GT, t, V0, SZ.p, T1.p, T2.p, s));
  launch_k(k_b_z0, nb, 256, 0, s, (long)nt, Z.p, V0, SZ.p);
  AMG_LAUNCH_CHECK();
  AMG_TRY(mgs(n, t, Z.p, s));
  // first quotients (unit columns), directions P = 2 (S Z - q Z), then S P
  AMG_TRY(apply_s_cols(A, G, GT, t, Z.p, SZ.p, T1.p, T2.p, s));
  {
    CDot a{};
    a.x[0] = Z.p;
    a.y[0] = SZ.p;
    a.xs[0] = a.ys[0] = n;
    AMG_TRY(cdots(n, t, 1, a, out.p, CF_NONE, cs.p, skip.p, ctx, s));
    launch_k(k_b_p0, nb, 256, 0, s, n, t, P.p, Z.p, SZ.p, out.p);
    launch_k(k_fill, 1, 64, 0, s, cs.p + C_F * t, t, 1.0);
    AMG_LAUNCH_CHECK();
  }
  AMG_TRY(apply_s_cols(A, G, GT, t, P.p, SP.p, T1.p, T2.p, s));
  // one iteration of the outer loop (optionally with the Ritz step)
  auto iteration = [&](bool ritz) -> int {
    if (ritz) {
      const long warps = nchunks > 0 ? (long)nchunks * t * (t + 1) : 1;
      launch_k(k_gram, (int)warps, 32, 0, s, n, t, Z.p, SZ.p, part.p, tk.p, nchunks, H.p, Mg.p);
      launch_k(k_ritz_eig, 1, 128, (6 * t * t + t) * sizeof(double), s, t, H.p, Mg.p, U.p, lam.p, cs.p + C_F * t,
                                                                           status);
      launch_k(k_rotate, dim3(nblk(n, 256), 2), 256, 0, s, n, t, Z.p, SZ.p, U.p);  // Z U, (S Z) U
      AMG_LAUNCH_CHECK();
    }
    CDot a5{};
    a5.x[0] = P.p; a5.y[0] = SZ.p;
    a5.x[1] = P.p; a5.y[1] = SP.p;
    a5.x[2] = P.p; a5.y[2] = Z.p;
    a5.x[3] = P.p; a5.y[3] = P.p;
    a5.x[4] = Z.p; a5.y[4] = SZ.p;
    for (int q = 0; q < 5; ++q) a5.xs[q] = a5.ys[q] = n;
    AMG_TRY(cdots(n, t, 5, a5, out.p, CF_ALPHA, cs.p, skip.p, ctx, s));
    launch_k(k_b_zupd, nb, 256, 0, s, n, t, Z.p, P.p, SZ.p, SP.p, cs.p, skip.p);
    AMG_LAUNCH_CHECK();
    CDot a2{};
    a2.x[0] = Z.p; a2.y[0] = Z.p;
    a2.x[1] = Z.p; a2.y[1] = SZ.p;
    a2.xs[0] = a2.ys[0] = a2.xs[1] = a2.ys[1] = n;
    AMG_TRY(cdots(n, t, 2, a2, out.p, CF_Q, cs.p, skip.p, ctx, s));
    launch_k(k_b_grad, nb, 256, 0, s, n, t, Gv.p, SZ.p, Z.p, cs.p, skip.p);
    AMG_LAUNCH_CHECK();
    AMG_TRY(apply_s_cols(A, G, GT, t, Gv.p, SG.p, T1.p, T2.p, s));  // the one product with S
    CDot a1{};
    a1.x[0] = Gv.p;
    a1.y[0] = SP.p;
    a1.xs[0] = a1.ys[0] = n;
    AMG_TRY(cdots(n, t, 1, a1, out.p, CF_BETA, cs.p, skip.p, ctx, s));
    launch_k(k_b_pupd, nb, 256, 0, s, n, t, P.p, Gv.p, SP.p, SG.p, cs.p, skip.p);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  // every iteration issues the same kernels: record each kind once as a CUDA
  // graph and replay it
  cudaGraphExec_t ge[2] = {nullptr, nullptr};
  long long nodes[2] = {0, 0};
  int rc = AMG_OK;
  for (int it = 1; it <= kmax && rc == AMG_OK; ++it) {
    const int ritz = (k_ritz > 0 && it % k_ritz == 0) ? 1 : 0;
    if (!ge[ritz]) {
      cudaGraph_t g = nullptr;
      const long long before = launch_count();
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = AMG_ERR_CUDA;
        break;
      }
      const int rc_body = iteration(ritz != 0);
      const cudaError_t ce = cudaStreamEndCapture(s, &g);
      nodes[ritz] = launch_count() - before;
      count_launches(-nodes[ritz]);
      if (rc_body || ce != cudaSuccess || cudaGraphInstantiate(&ge[ritz], g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error("SRQCG: recording the iteration graph failed");
        rc = rc_body ? rc_body : AMG_ERR_CUDA;
        break;
      }
      cudaGraphDestroy(g);
    }
    if (cudaGraphLaunch(ge[ritz], s) != cudaSuccess) {
      set_error("SRQCG: graph launch failed");
      rc = AMG_ERR_CUDA;
      break;
    }
    count_launches(nodes[ritz]);
  }
  for (int k = 0; k < 2; ++k)
    if (ge[k]) cudaGraphExecDestroy(ge[k]);
  if (rc) return rc;
  AMG_TRY(spmv_cols(GT, t, Z.p, V, s));
  AMG_TRY(mgs(n, t, V, s));
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- Lanczos
// w = (w - alpha_j v_j) - beta_{j-1} v_{j-1}
__global__ void k_lz_ab(long n, double *__restrict__ w, const double *__restrict__ v, const double *__restrict__ vp,
                        const double *__restrict__ sc, int j) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = fma(-sc[j], v[i], w[i]);
  if (vp) x = fma(-sc[64 + j - 1], vp[i], x);
  w[i] = x;
}

// w_i - sum_{k <= j} h_k v_k,i, k ascending (one classical Gram-Schmidt pass)
__global__ void k_lz_reorth(long n, int j, double *__restrict__ w, const double *__restrict__ Vs,
                            const double *__restrict__ h) {
  pdl_wait();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = w[i];
  for (int k = 0; k <= j; ++k) x = fma(-h[k], Vs[(size_t)k * n + i], x);
  w[i] = x;
}

// Largest eigenvalue of G A G^T by m Lanczos steps with full
// re-orthogonalisation (one classical Gram-Schmidt pass per step), from the
// counter-generator start vector of this level; bisection on Sturm counts.
// sc layout: [0..63] alpha, [64..127] beta, [128] breakdown step, [129] norm
// square, [160..223] re-orthogonalisation coefficients, [256..319] 1 / beta.
int lanczos(const DevBsr &A, const DevBsr &G, const DevBsr &GT, int m, uint64_t seed, int level,
            double safety, double *d_out, cudaStream_t s, bool sync) {
  const int n = A.b * A.nr;
  if (m > n) m = n;
  if (m > 64) m = 64;
  DBuf<double> Vs, w, t1, t2, sc, part;
  DBuf<unsigned> tk;
  AMG_TRY(tk.alloc(MAXTICKETS));
  AMG_TRY(tk.zero(s));
  AMG_TRY(Vs.alloc((size_t)m * n));
  AMG_TRY(w.alloc(n));
  AMG_TRY(t1.alloc(n));
  AMG_TRY(t2.alloc(n));
  AMG_TRY(sc.alloc(320));
  AMG_TRY(part.alloc((size_t)((n + CHUNK - 1) / CHUNK + 1) * 66));
  AMG_TRY(sc.zero(s));
  launch_k(k_set_neg, 1, 1, 0, s, sc.p + 128);
  launch_k(k_lanczos_start, nblk(n, 256), 256, 0, s, n, seed, (1ull << 62) | ((uint64_t)level << 40), Vs.p);
  AMG_LAUNCH_CHECK();
  const DotCtx ctx{part.p, tk.p};
  AMG_TRY(dot1(n, Vs.p, Vs.p, sc.p + 129, ctx, s));
  launch_k(k_div_sqrt, nblk(n, 256), 256, 0, s, n, Vs.p, sc.p + 129);
  for (int j = 0; j < m; ++j) {
    double *v = Vs.p + (size_t)j * n;
    AMG_TRY(spmv(GT, v, t1.p, s));
    AMG_TRY(spmv(A, t1.p, t2.p, s));
    AMG_TRY(spmv(G, t2.p, w.p, s));
    AMG_TRY(dot1(n, w.p, v, sc.p + j, ctx, s));
    launch_k(k_lz_ab, nblk(n, 256), 256, 0, s, n, w.p, v, j > 0 ? v - n : nullptr, sc.p, j);
    CDot a{};
    a.x[0] = w.p;
    a.xs[0] = 0;
    a.y[0] = Vs.p;
    a.ys[0] = n;
    AMG_TRY(cdots(n, j + 1, 1, a, sc.p + 160, CF_NONE, nullptr, nullptr, ctx, s));
    launch_k(k_lz_reorth, nblk(n, 256), 256, 0, s, n, j, w.p, Vs.p, sc.p + 160);
    Fin fb;
    fb.op = FIN_LZ_BETA;
    fb.sc = sc.p;
    fb.j = j;
    fb.m = m;
    AMG_TRY(dot1(n, w.p, w.p, sc.p + 129, ctx, s, fb));
    if (j < m - 1) launch_k(k_mul_by, nblk(n, 256), 256, 0, s, n, v + n, w.p, sc.p + 256 + j);
    AMG_LAUNCH_CHECK();
  }
  launch_k(k_lanczos_bisect, 1, 32, 0, s, m, sc.p, safety, d_out);
  AMG_LAUNCH_CHECK();
  // the temporaries above are returned to the pool in the order of s
  if (sync) AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- SoC + filter
// Node gram of the test space: M[r][c] = sum_k V[k][BI+r] V[k][BJ+c], k ascending.
template <int B>
__device__ __forceinline__ void node_gram(long n, int t, const double *__restrict__ V, int I, int J, double *M) {
  for (int r = 0; r < B; ++r)
    for (int c = 0; c < B; ++c) {
      double s = 0.0;
      for (int k = 0; k < t; ++k) s = fma(V[(size_t)k * n + (long)B * I + r], V[(size_t)k * n + (long)B * J + c], s);
      M[r * B + c] = s;
    }
}

template <int B>
__device__ __forceinline__ double fro2(const double *M) {
  double s = 0.0;
  for (int i = 0; i < B * B; ++i) s = fma(M[i], M[i], s);
  return s;
}

template <int B>
__global__ void k_soc_nrm(int nn, int t, const double *__restrict__ V, double *__restrict__ nrm) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  double M[B * B];
  node_gram<B>((long)B * nn, t, V, I, I, M);
  nrm[I] = sqrt(fro2<B>(M));
}

__device__ __forceinline__ int find_in_row(const int *rp, const int *col, int row, int v) {
  int lo = rp[row], hi = rp[row + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] == v) return mid;
    if (col[mid] < v) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// SoC of the block pair {(I,J), (J,I)} with I < J, computed once from the
// smaller node first and written to both positions (one thread per stored
// block of the upper triangle); diagonal blocks get 0.
template <int B>
__device__ __forceinline__ void soc_entry(int nn, int t, int I, int k, const int *__restrict__ rp,
                                          const int *__restrict__ col, const double *__restrict__ V,
                                          const double *__restrict__ nrm, double *__restrict__ soc) {
  const int J = col[k];
  if (J == I) {
    soc[k] = 0.0;
    return;
  }
  const int kt = find_in_row(rp, col, J, I);
  if (J < I && kt >= 0) return;  // the mirror's thread writes both
  const int a = I < J ? I : J, b = I < J ? J : I;
  double M[B * B];
  node_gram<B>((long)B * nn, t, V, a, b, M);
  const double num = fro2<B>(M), den = nrm[a] * nrm[b];
  const double v = den > 0.0 ? num / den : 0.0;
  soc[k] = v;
  if (kt >= 0) soc[kt] = v;
}

// one thread per block (large levels: full lanes)
template <int B>
__global__ void k_soc_pairs(int nn, int nnzb, int t, const int *__restrict__ rp, const int *__restrict__ col,
                            const double *__restrict__ V, const double *__restrict__ nrm, double *__restrict__ soc) {
  pdl_wait();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  int lo = 0, hi = nn - 1;
  while (lo < hi) {  // row of block k: last row with rp[row] <= k
    const int mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= k) lo = mid; else hi = mid - 1;
  }
  soc_entry<B>(nn, t, lo, k, rp, col, V, nrm, soc);
}

// one warp per block row, lanes over its blocks (small levels: no row search)
template <int B>
__global__ void k_soc_pairs_rows(int nn, int t, const int *__restrict__ rp, const int *__restrict__ col,
                                 const double *__restrict__ V, const double *__restrict__ nrm,
                                 double *__restrict__ soc) {
  pdl_wait();
  const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (I >= nn) return;
  for (int k = rp[I] + lane; k < rp[I + 1]; k += 32) soc_entry<B>(nn, t, I, k, rp, col, V, nrm, soc);
}

// The theta largest positive SoC of row I are kept (ties to the smaller
// column).  One warp per row: each pick is a warp arg-max over the row's
// entries not yet kept (larger SoC first, then the smaller position, which
// is the smaller column).
__global__ void k_soc_select(int nn, const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ soc, int theta, unsigned char *__restrict__ kept) {
  pdl_wait();
  const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (I >= nn) return;
  const int k0 = rp[I], k1 = rp[I + 1];
  for (int k = k0 + lane; k < k1; k += 32) kept[k] = 0;
  __syncwarp();
  for (int p = 0; p < theta; ++p) {
    double bv = 0.0;
    int bk = -1;
    for (int k = k0 + lane; k < k1; k += 32)
      if (!kept[k] && col[k] != I && soc[k] > 0.0 && (bk < 0 || soc[k] > bv)) {
        bv = soc[k];
        bk = k;
      }
    for (int off = 16; off >= 1; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
      if (ok >= 0 && (bk < 0 || ov > bv || (ov == bv && ok < bk))) {
        bv = ov;
        bk = ok;
      }
    }
    if (bk < 0) break;
    if (lane == 0) kept[bk] = 1;
    __syncwarp();
  }
}

__global__ void k_strong(int nn, const int *__restrict__ rp, const int *__restrict__ col,
                         const unsigned char *__restrict__ kept, unsigned char *__restrict__ strong) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    int lo = rp[J], hi = rp[J + 1] - 1, kt = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      if (col[mid] == I) { kt = mid; break; }
      if (col[mid] < I) lo = mid + 1; else hi = mid - 1;
    }
    strong[k] = (unsigned char)(kept[k] || (kt >= 0 && kept[kt]));
  }
}

int soc_filter(const DevBsr &A, int t, const double *V, int theta, unsigned char *strong, cudaStream_t s) {
  DBuf<double> nrm, soc;
  DBuf<unsigned char> kept;
  AMG_TRY(nrm.alloc(A.nr));
  AMG_TRY(soc.alloc(A.nnzb));
  AMG_TRY(kept.alloc(A.nnzb));
  const int nb = nblk(A.nr, 128);
  AMG_TRY(soc.zero(s));
  const bool rows = A.nr < 32768;
  const int nbr = nblk(32L * A.nr, 128), nbe = nblk(A.nnzb, 128);
  if (A.b == 1) {
    launch_k(k_soc_nrm<1>, nb, 128, 0, s, A.nr, t, V, nrm.p);
    if (rows) launch_k(k_soc_pairs_rows<1>, nbr, 128, 0, s, A.nr, t, A.rowptr.p, A.col.p, V, nrm.p, soc.p);
    else launch_k(k_soc_pairs<1>, nbe, 128, 0, s, A.nr, A.nnzb, t, A.rowptr.p, A.col.p, V, nrm.p, soc.p);
  } else {
    launch_k(k_soc_nrm<3>, nb, 128, 0, s, A.nr, t, V, nrm.p);
    if (rows) launch_k(k_soc_pairs_rows<3>, nbr, 128, 0, s, A.nr, t, A.rowptr.p, A.col.p, V, nrm.p, soc.p);
    else launch_k(k_soc_pairs<3>, nbe, 128, 0, s, A.nr, A.nnzb, t, A.rowptr.p, A.col.p, V, nrm.p, soc.p);
  }
  launch_k(k_soc_select, nblk(32L * A.nr, 128), 128, 0, s, A.nr, A.rowptr.p, A.col.p, soc.p, theta, kept.p);
  launch_k(k_strong, nb, 128, 0, s, A.nr, A.rowptr.p, A.col.p, kept.p, strong);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- DPLS
// One thread per fine node (Algorithm 5 in nodal-block form).  Householder
// step on column x (rows p..t-1): sigma = sqrt(sum x^2), alpha = -sigma if
// x_p >= 0 else sigma, v = x with v_p = x_p - alpha, vv = sum v^2; a column y
// becomes y - ((2 v.y)(1/vv)) v, the reciprocal rvv = 1/vv formed once per v.  Affinity of residual X and candidate Y over
// the trailing rows: ||X^T Y||_F^2 / (||X^T X||_F ||Y^T Y||_F).
__device__ __forceinline__ void reflect(int t, int p, const double *v, double rvv, double *y, int stride) {
  double s = 0.0;
  for (int k = p; k < t; ++k) s = fma(v[k], y[k * stride], s);
  const double f = (2.0 * s) * rvv;
  for (int k = p; k < t; ++k) y[k * stride] = fma(-f, v[k], y[k * stride]);
}

// ||X^T X||_F^2 over rows p..t-1.  Entry (a, c) and entry (c, a) are the
// same chain of fused multiply-adds with the factors swapped, hence equal
// bit for bit: the six distinct entries are formed once and the nine squares
// are added in row-major order.
template <int B>
__device__ __forceinline__ double gram_fro2(int t, int p, const double *X) {
  double g[B][B];
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int c = a; c < B; ++c) {
      double s = 0.0;
      for (int k = p; k < t; ++k) s = fma(X[k * B + a], X[k * B + c], s);
      g[a][c] = s;
      g[c][a] = s;
    }
  double f = 0.0;
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int c = 0; c < B; ++c) f = fma(g[a][c], g[a][c], f);
  return f;
}

// affinity of residual X and candidate Y; xx = gram_fro2(X), the same for
// every candidate of one step
template <int B>
__device__ __forceinline__ double affinity(int t, int p, const double *X, double xx, const double *Y) {
  double xy = 0.0;
#pragma unroll
  for (int a = 0; a < B; ++a)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      double s = 0.0;
      for (int k = p; k < t; ++k) s = fma(X[k * B + a], Y[k * B + c], s);
      xy = fma(s, s, xy);
    }
  const double yy = gram_fro2<B>(t, p, Y);
  const double den = sqrt(xx) * sqrt(yy);
  return den > 0.0 ? xy / den : -1.0;
}

template <int B>
__global__ void k_dpls(int nf, const int *__restrict__ fnodes, long n, int t, const double *__restrict__ V,
                       const int *__restrict__ cptr, const int *__restrict__ cand, const int *__restrict__ cidx,
                       double *__restrict__ Vt, unsigned char *__restrict__ taken, int n_max, double kappa_p,
                       int nsel_cap, int *__restrict__ out_cnt, int *__restrict__ out_col,
                       double *__restrict__ out_val) {
  pdl_wait();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int I = fnodes[f];
  const int c0 = cptr[f], ncand = cptr[f + 1] - c0;
  double *vt = Vt + (size_t)c0 * t * B;
  unsigned char *tk = taken + c0;
  double r[TMAXD * B], R[TMAXD * TMAXD], Y[TMAXD * B], hv[B][TMAXD], hvv[B], w[TMAXD * B];
  int sel[TMAXD];
  for (int i = 0; i < TMAXD * TMAXD; ++i) R[i] = 0.0;
  for (int k = 0; k < t; ++k)
    for (int c = 0; c < B; ++c) r[k * B + c] = V[(size_t)k * n + (long)B * I + c];
  for (int j = 0; j < ncand; ++j) {
    tk[j] = 0;
    for (int k = 0; k < t; ++k)
      for (int c = 0; c < B; ++c) vt[((size_t)j * t + k) * B + c] = V[(size_t)k * n + (long)B * cand[c0 + j] + c];
  }
  int nsel = 0, p = 0;
  double rdmax = 0.0, rdmin = 0.0;
  for (;;) {
    if (nsel >= n_max || p + B > t) break;
    double rr = 0.0;
    for (int k = p; k < t; ++k)
      for (int c = 0; c < B; ++c) rr = fma(r[k * B + c], r[k * B + c], rr);
    if (rr == 0.0) break;
    const double xx = gram_fro2<B>(t, p, r);
    int best = -1;
    double baff = 0.0;
    for (int j = 0; j < ncand; ++j) {
      if (tk[j]) continue;
      const double a = affinity<B>(t, p, r, xx, vt + (size_t)j * t * B);
      if (a < 0.0) continue;
      if (best < 0 || a > baff) {
        best = j;
        baff = a;
      }
    }
    if (best < 0) break;
    for (int i = 0; i < t * B; ++i) Y[i] = vt[(size_t)best * t * B + i];
    int ok = 1;
    double dmax = rdmax, dmin = rdmin;
    for (int c = 0; c < B && ok; ++c) {
      const int pc = p + c;
      double sg = 0.0;
      for (int k = pc; k < t; ++k) sg = fma(Y[k * B + c], Y[k * B + c], sg);
      sg = sqrt(sg);
      if (!(sg > 0.0)) {
        ok = 0;
        break;
      }
      const double alpha = Y[pc * B + c] >= 0.0 ? -sg : sg;
      for (int k = 0; k < t; ++k) hv[c][k] = (k >= pc) ? Y[k * B + c] : 0.0;
      hv[c][pc] = Y[pc * B + c] - alpha;
      double vv = 0.0;
      for (int k = pc; k < t; ++k) vv = fma(hv[c][k], hv[c][k], vv);
      hvv[c] = 1.0 / vv;  // reciprocal
      for (int c2 = c + 1; c2 < B; ++c2) reflect(t, pc, hv[c], hvv[c], Y + c2, B);
      Y[pc * B + c] = alpha;
      for (int k = pc + 1; k < t; ++k) Y[k * B + c] = 0.0;
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
    for (int c = 0; c < B; ++c)
      for (int k = 0; k <= p + c; ++k) R[k * TMAXD + p + c] = Y[k * B + c];
    for (int c = 0; c < B; ++c) {
      for (int c2 = 0; c2 < B; ++c2) reflect(t, p + c, hv[c], hvv[c], r + c2, B);
      for (int j = 0; j < ncand; ++j) {
        if (tk[j] || j == best) continue;
        for (int c2 = 0; c2 < B; ++c2) reflect(t, p + c, hv[c], hvv[c], vt + (size_t)j * t * B + c2, B);
      }
    }
    tk[best] = 1;
    sel[nsel++] = cand[c0 + best];
    p += B;
    rdmax = dmax;
    rdmin = dmin;
  }
  for (int c = 0; c < B; ++c)
    for (int i = p - 1; i >= 0; --i) {
      double s = r[i * B + c];
      for (int k = p - 1; k > i; --k) s = fma(-R[i * TMAXD + k], w[k * B + c], s);
      w[i * B + c] = s / R[i * TMAXD + i];
    }
  // entries sorted by coarse index
  int ord[TMAXD];
  for (int m = 0; m < nsel; ++m) ord[m] = m;
  for (int u = 1; u < nsel; ++u) {
    const int v = ord[u];
    int q = u - 1;
    while (q >= 0 && cidx[sel[ord[q]]] > cidx[sel[v]]) { ord[q + 1] = ord[q]; --q; }
    ord[q + 1] = v;
  }
  out_cnt[f] = nsel;
  for (int u = 0; u < nsel; ++u) {
    const int m = ord[u];
    out_col[(size_t)f * nsel_cap + u] = cidx[sel[m]];
    double *o = out_val + ((size_t)f * nsel_cap + u) * B * B;
    for (int c = 0; c < B; ++c)
      for (int d = 0; d < B; ++d) o[c * B + d] = w[(B * m + d) * B + c];
  }
}

int dpls(const DevBsr &A, const unsigned char *strong, const int *cf, const int *cidx, const int *fnodes, int nf,
         const int *cand_ptr, const int *cand, int t, const double *V, int n_max, double kappa_p, int *out_cnt,
         int *out_col, double *out_val, int *status, cudaStream_t s) {
  (void)strong; (void)cf; (void)status;
  if (t > TMAXD) {
    set_error("n_tv = %d exceeds the supported maximum %d", t, TMAXD);
    return AMG_ERR_ARG;
  }
  if (nf == 0) return AMG_OK;
  int total = 0;
  AMG_CU(cudaMemcpyAsync(&total, cand_ptr + nf, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  DBuf<double> Vt;
  DBuf<unsigned char> taken;
  const int B = A.b;
  AMG_TRY(Vt.alloc((size_t)total * t * B));
  AMG_TRY(taken.alloc(total));
  const int cap = n_max < t / B ? n_max : t / B;
  if (B == 1)
    launch_k(k_dpls<1>, nblk(nf, 64), 64, 0, s, nf, fnodes, (long)A.nr, t, V, cand_ptr, cand, cidx, Vt.p, taken.p,
                                                    n_max, kappa_p, cap > 0 ? cap : 1, out_cnt, out_col, out_val);
  else
    launch_k(k_dpls<3>, nblk(nf, 64), 64, 0, s, nf, fnodes, 3L * A.nr, t, V, cand_ptr, cand, cidx, Vt.p, taken.p,
                                                    n_max, kappa_p, cap > 0 ? cap : 1, out_cnt, out_col, out_val);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- SpGEMM
// Z = X Y on Z's given pattern; each output block adds the block products
// X_ik Y_kc over k ascending (entry (r,q) of a product: sum_d X(r,d) Y(d,q),
// d ascending from 0), accumulating from 0.  Nine lanes per output block,
// one per entry (3 blocks per warp): the nine walk the same k and take the
// same branches, so the FP64 work runs on full lane groups.
template <int B>
__global__ void k_spgemm(int nr, const int *__restrict__ xr, const int *__restrict__ xc, const double *__restrict__ xv,
                         const int *__restrict__ yr, const int *__restrict__ yc, const double *__restrict__ yv,
                         const int *__restrict__ zr, const int *__restrict__ zc, double *__restrict__ zv, int nnz) {
  pdl_wait();
  constexpr int BB = B * B, PER = 32 / BB;  // output blocks per warp
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (lane >= PER * BB) return;
  const long ql = PER * w + lane / BB;
  if (ql >= nnz) return;
  const int q = (int)ql, e = lane % BB, r = e / B, qq = e - B * r;
  int lo = 0, hi = nr - 1;
  while (lo < hi) {  // row of entry q: last row with zr[row] <= q
    const int mid = (lo + hi + 1) >> 1;
    if (zr[mid] <= q) lo = mid; else hi = mid - 1;
  }
  const int i = lo, c = zc[q];
  double acc = 0.0;
  for (int kx = xr[i]; kx < xr[i + 1]; ++kx) {
    const int k = xc[kx];
    int a = yr[k], b = yr[k + 1] - 1, ky = -1;
    while (a <= b) {
      const int mid = (a + b) >> 1;
      if (yc[mid] == c) { ky = mid; break; }
      if (yc[mid] < c) a = mid + 1; else b = mid - 1;
    }
    if (ky < 0) continue;
    const double *x = xv + (size_t)kx * BB, *y = yv + (size_t)ky * BB;
    double sv = 0.0;
    for (int d = 0; d < B; ++d) sv = fma(x[r * B + d], y[d * B + qq], sv);
    acc = acc + sv;
  }
  zv[(size_t)q * BB + e] = acc;
}

// The same products by rows of Z (Gustavson's order): one warp per row i.
// The row's accumulators (one per entry of its blocks, from 0) and its
// column list sit in shared memory.  The entries (i, k) of X's row are taken
// 32 at a time; their terms -- the triples (k, j, e) of Y's row k, entry e of
// block j -- are numbered in that order and the lanes take 32 consecutive
// triples at once: each forms the FMA chain over d of its entry and finds
// the position of Y's column in Z's row; then the terms are added to their
// accumulators entry by entry, k ascending.  So every accumulator receives
// the terms of the k that contain its column, in ascending k, the additions
// of k_spgemm (same bits), while the FP64 instructions run on nearly full
// warps and no (k, column) pair is searched for in vain.
template <int B>
__global__ void __launch_bounds__(32) k_spgemm_rows(const int *__restrict__ xr, const int *__restrict__ xc,
                                                    const double *__restrict__ xv, const int *__restrict__ yr,
                                                    const int *__restrict__ yc, const double *__restrict__ yv,
                                                    const int *__restrict__ zr, const int *__restrict__ zc,
                                                    double *__restrict__ zv) {
  pdl_wait();
  constexpr int BB = B * B;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ double sacc[];  // len * BB accumulators, then len columns
  const int i = blockIdx.x, lane = threadIdx.x;
  const int z0 = zr[i], len = zr[i + 1] - z0;
  int *scol = reinterpret_cast<int *>(sacc + (size_t)len * BB);
  for (int q = lane; q < len * BB; q += 32) sacc[q] = 0.0;
  for (int q = lane; q < len; q += 32) scol[q] = zc[z0 + q];
  __syncwarp();
  const int xe = xr[i + 1];
  for (int kb = xr[i]; kb < xe; kb += 32) {
    // lane l: entry kb + l of X's row, the start of Y's row and its triple count
    int y0 = 0, cnt = 0;
    if (kb + lane < xe) {
      const int k = xc[kb + lane];
      y0 = yr[k];
      cnt = (yr[k + 1] - y0) * BB;
    }
    int pre = cnt;  // inclusive prefix over the lanes
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(FULL, pre, 31);
    for (int f0 = 0; f0 < total; f0 += 32) {
      const int f = f0 + lane;
      const bool valid = f < total;
      int u = 0;  // the entry whose triples hold f: the number of lanes with pre <= f
      for (int st = 16; st; st >>= 1)
        if (__shfl_sync(FULL, pre, u + st - 1) <= f) u += st;
      u = min(u, 31);
      const int first = __shfl_sync(FULL, pre - cnt, u), yb0 = __shfl_sync(FULL, y0, u);
      int pos = -1, e = 0;
      double sv = 0.0;
      if (valid) {
        const int t = f - first, j = t / BB;
        e = t - BB * j;
        const int r = e / B, qq = e - B * r;
        const int c = yc[yb0 + j];
        const double *xb = xv + (size_t)(kb + u) * BB, *yb = yv + (size_t)(yb0 + j) * BB;
#pragma unroll
        for (int d = 0; d < B; ++d) sv = fma(xb[r * B + d], yb[d * B + qq], sv);
        int lo = 0, hi = len - 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (scol[mid] < c) lo = mid + 1;
          else hi = mid;
        }
        if (len > 0 && scol[lo] == c) pos = lo;
      }
      const int ulo = __shfl_sync(FULL, u, 0), uhi = __reduce_max_sync(FULL, valid ? u : 0);
      for (int w = ulo; w <= uhi; ++w) {  // k ascending
        if (valid && u == w && pos >= 0) sacc[pos * BB + e] = sacc[pos * BB + e] + sv;
        __syncwarp();
      }
    }
  }
  __syncwarp();
  for (int q = lane; q < len * BB; q += 32) zv[(size_t)z0 * BB + q] = sacc[q];
}

int spgemm_numeric(const DevBsr &X, const DevBsr &Y, DevBsr &Z, cudaStream_t s) {
  if (Z.nnzb == 0) return AMG_OK;
  int ml = 0;
  AMG_TRY(Z.row_max(s, &ml));
  const size_t shm = (size_t)ml * (Z.b * Z.b * sizeof(double) + sizeof(int));
  // by rows when there are rows enough to fill the GPU and each fits the
  // default shared-memory window (measured on the beam's Galerkin products:
  // products of 139k, 30k and 6.2k rows faster by rows -- level 0's R A P
  // 1.37 -> 0.64 ms --, of 1.3k and 263 rows faster with nine lanes per
  // output block)
  if (Z.nr >= 4096 && shm <= 48 * 1024) {
    if (Z.b == 1)
      launch_k(k_spgemm_rows<1>, Z.nr, 32, shm, s, X.rowptr.p, X.col.p, X.val.p, Y.rowptr.p, Y.col.p, Y.val.p,
                                                       Z.rowptr.p, Z.col.p, Z.val.p);
    else
      launch_k(k_spgemm_rows<3>, Z.nr, 32, shm, s, X.rowptr.p, X.col.p, X.val.p, Y.rowptr.p, Y.col.p, Y.val.p,
                                                       Z.rowptr.p, Z.col.p, Z.val.p);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  }
  if (Z.b == 1)
    launch_k(k_spgemm<1>, nblk(32L * ((Z.nnzb + 31) / 32), 128), 128, 0, s, Z.nr, X.rowptr.p, X.col.p, X.val.p, Y.rowptr.p, Y.col.p, Y.val.p, Z.rowptr.p, Z.col.p, Z.val.p, Z.nnzb);
  else
    launch_k(k_spgemm<3>, nblk(32L * ((Z.nnzb + 2) / 3), 128), 128, 0, s, Z.nr, X.rowptr.p, X.col.p, X.val.p, Y.rowptr.p, Y.col.p, Y.val.p, Z.rowptr.p, Z.col.p, Z.val.p, Z.nnzb);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace det
}  // namespace amg
