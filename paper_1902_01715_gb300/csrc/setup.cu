// Hierarchy set-up (Algorithm 1 of the paper): per level the aFSAI smoother
// (Algorithm 3), the SRQCG test space (Algorithm 4), the affinity C/F split
// (Sec. 3.3), DPLS prolongation (Algorithm 5) and the Galerkin product.
// Floating-point work runs in the kernels of det.cu, the integer pattern work
// in those of graph.cu and of this file (maximal independent set, candidate
// sets, pattern compaction); the host keeps the control flow and reads back
// only sizes and status words.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "amg_internal.h"

namespace amg {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

const char *last_error() { return g_err; }

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local cudaStream_t t_stream = nullptr;
cudaStream_t current_stream() { return t_stream; }
StreamScope::StreamScope(cudaStream_t s) : prev(t_stream) { t_stream = s; }
StreamScope::~StreamScope() { t_stream = prev; }
static thread_local bool t_pdl = false;
bool pdl_enabled() { return t_pdl; }
PdlScope::PdlScope(bool on) : prev(t_pdl) { t_pdl = on && getenv("AMG_NO_PDL") == nullptr; }
PdlScope::~PdlScope() { t_pdl = prev; }

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
  // once per device: keep freed pool memory (the default threshold returns
  // it to the driver at every synchronisation)
  static std::mutex mu;
  static bool init[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(mu);
    if (!init[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        // memory freed on one stream is not handed to another by making the
        // second wait for the first (the set-up runs two streams at once)
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
      }
      init[dev] = true;
    }
  }
  return cudaMallocAsync(p, bytes, s);
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Set-up phase trace on stderr when the environment sets AMG_TRACE (phases
// end with a stream synchronisation, so host time is device time).
static bool trace_on() {
  static const bool on = getenv("AMG_TRACE") != nullptr;
  return on;
}

static void trace(const char *what, int level, double t0) {
  if (trace_on()) fprintf(stderr, "[amg] level %d %-18s %9.3f ms\n", level, what, 1e3 * (now_s() - t0));
}

// ---------------------------------------------------------------- kernels
// Copy rows stored with a fixed capacity into a compact BSR (values only,
// B x B blocks).
template <int B>
__global__ void k_compact_vals(int n, int cap, const int *__restrict__ rowptr, const double *__restrict__ src,
                               double *__restrict__ dst) {
  pdl_wait();
  constexpr int BB = B * B;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int I = (int)(t / (cap * BB));
  if (I >= n) return;
  const int rem = (int)(t - (long)I * cap * BB);
  const int j = rem / BB, e = rem % BB;
  const int len = rowptr[I + 1] - rowptr[I];
  if (j >= len) return;
  dst[((size_t)rowptr[I] + j) * BB + e] = src[((size_t)I * cap + j) * BB + e];
}

// P values: identity for coarse rows, DPLS blocks for fine rows.
template <int B>
__global__ void k_p_vals(int n, const int *__restrict__ rowptr, const int *__restrict__ fidx, int cap,
                         const double *__restrict__ fval, double *__restrict__ pv) {
  pdl_wait();
  constexpr int BB = B * B;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int I = (int)(t / (cap * BB));
  if (I >= n) return;
  const int rem = (int)(t - (long)I * cap * BB);
  const int j = rem / BB, e = rem % BB;
  const int len = rowptr[I + 1] - rowptr[I];
  if (j >= len) return;
  const int f = fidx[I];
  const double v = (f < 0) ? ((e % (B + 1) == 0) ? 1.0 : 0.0) : fval[((size_t)f * cap + j) * BB + e];
  pv[((size_t)rowptr[I] + j) * BB + e] = v;
}

// dense copy of a BSR matrix (row-major m x m, m = B nr); block I of the grid
// copies block row I, BB threads per block
template <int B>
__global__ void k_to_dense(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                           const double *__restrict__ val, double *__restrict__ D) {
  pdl_wait();
  constexpr int BB = B * B;
  const int I = blockIdx.x;
  const long m = (long)B * nr;
  for (int k = rp[I] + threadIdx.x / BB; k < rp[I + 1]; k += blockDim.x / BB) {
    if ((int)threadIdx.x >= (blockDim.x / BB) * BB) break;
    const int e = threadIdx.x % BB, r = e / B, c = e % B;
    D[(size_t)((long)B * I + r) * m + (long)B * col[k] + c] = val[(size_t)k * BB + e];
  }
}

// Explicit inverse of the last level's matrix by blocked sweeps (the
// symmetric form of Gauss-Jordan elimination), in place in a dense row-major
// m x m array of which only the lower triangle (i >= j) is kept current.
// Sweeping the pivot block K (indices [k0, k0+nb)) of a symmetric matrix:
// D = A_KK^{-1}; A_IJ -= A_IK D A_KJ for I, J outside K; A_IK = A_IK D;
// A_KJ = D A_KJ; A_KK = -D.  The matrix stays symmetric, and once every
// block has been swept it holds -A^{-1}; each pivot block is then a Schur
// complement of an SPD matrix, hence SPD (no pivoting).  With the pivot
// column C_J = A_JK (read from the lower triangle) and V_J = D C_J^T, step K
// is A_IJ -= C_I V_J on the lower tiles, A_IK = V_I^T, A_KJ = V_J and
// A_KK = -D; a last pass negates the lower triangle and mirrors it.  Half
// the multiply-adds of Gauss-Jordan on the full array.  The coarse solve is
// then one dense product with the inverse.
constexpr int CB = 32;
constexpr int SW_THREADS = 544;  // 17 warps: one thread per lower entry of a 32 x 32 block

// Scalar sweeps of an nb x nb SPD block whose lower triangle is in b0, by
// the NT threads of a CTA, thread t taking the lower entries t, t + NT, ...
// (row order: (r, c), c <= r).  Two buffers (a step reads one and writes the
// other: one barrier per step); the thread of the next pivot forms its
// reciprocal as soon as it has the pivot, while the others update their
// entries.  Leaves P = block^{-1} (both triangles), or sets status if a
// pivot is not positive.  Every thread of the CTA must call it.
template <int NT>
__device__ void sweep_block(double (*b0)[CB + 1], double (*b1)[CB + 1], int nb, double *__restrict__ P,
                            int *__restrict__ status) {
  constexpr int NE = (CB * (CB + 1) / 2 + NT - 1) / NT;
  __shared__ double rcp[2];
  __shared__ int bad;
  const int t = threadIdx.x;
  int rr[NE], cc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int u = t + e * NT;
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    rr[e] = r;
    cc[e] = u - r * (r + 1) / 2;
  }
  if (t == 0) {
    const double pv = b0[0][0];
    bad = !(pv > 0.0);
    rcp[0] = 1.0 / pv;
  }
  __syncthreads();
  for (int j = 0; j < nb && !bad; ++j) {
    double (*cur)[CB + 1] = (j & 1) ? b1 : b0;
    double (*nxt)[CB + 1] = (j & 1) ? b0 : b1;
    const double d = rcp[j & 1];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int r = rr[e], c = cc[e];
      if (r >= nb) continue;
      // column j of the current matrix: entry x is stored at (max(x, j), min(x, j))
      const double gr = r >= j ? cur[r][j] : cur[j][r];
      const double gc = c >= j ? cur[c][j] : cur[j][c];
      double nv;
      if (r == j && c == j) nv = -d;
      else if (r == j) nv = gc * d;
      else if (c == j) nv = gr * d;
      else nv = fma(-(gr * d), gc, cur[r][c]);
      nxt[r][c] = nv;
      if (r == j + 1 && c == j + 1 && j + 1 < nb) {  // the next pivot
        if (!(nv > 0.0)) bad = 1;
        rcp[(j + 1) & 1] = 1.0 / nv;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicMin(status, AMG_ERR_NOT_SPD);
    return;
  }
  double (*fin)[CB + 1] = (nb & 1) ? b1 : b0;
#pragma unroll
  for (int e = 0; e < NE; ++e) {  // the sweeps leave -block^{-1}
    const int r = rr[e], c = cc[e];
    if (r >= nb) continue;
    const double v = -fin[r][c];
    P[r * CB + c] = v;
    P[c * CB + r] = v;
  }
}

// P = A_KK^{-1} of the first pivot block (the later ones come from the
// update kernel of the step before)
__global__ void __launch_bounds__(SW_THREADS) k_sw_pivot(int m, int k0, int nb, const double *__restrict__ D,
                                                        double *__restrict__ P, int *__restrict__ status) {
  pdl_wait();
  __shared__ double a[2][CB][CB + 1];
  const int t = threadIdx.x;
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  const int c = t - r * (r + 1) / 2;
  if (r < nb) a[0][r][c] = D[(size_t)(k0 + r) * m + k0 + c];
  __syncthreads();
  sweep_block<SW_THREADS>(a[0], a[1], nb, P, status);
}

// C[x][q] = A[x][k0+q] (pivot column, from the lower triangle) and
// V[q][x] = sum_p P[q][p] C[x][p], for every row x outside the pivot block
__global__ void k_sw_panels(int m, int k0, int nb, const double *__restrict__ D, const double *__restrict__ P,
                            double *__restrict__ V, double *__restrict__ C) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)CB * m) return;
  const int q = (int)(t / m), x = (int)(t % m);
  if (q >= nb || (x >= k0 && x < k0 + nb)) return;
  const bool below = x >= k0 + nb;
  double s = 0.0;
  for (int p = 0; p < nb; ++p) {
    const double cx = below ? D[(size_t)x * m + k0 + p] : D[(size_t)(k0 + p) * m + x];
    s = fma(P[q * CB + p], cx, s);
  }
  V[(size_t)q * m + x] = s;
  C[(size_t)x * CB + q] = below ? D[(size_t)x * m + k0 + q] : D[(size_t)(k0 + q) * m + x];
}

// one lower tile (I >= J) per CTA, 32 x 32, 256 threads (4 rows each):
// A_IJ -= C_I V_J; the pivot row and column tiles take V_J and V_I^T, the
// pivot tile -P.  Look-ahead: when Pn is given, the CTA of the next pivot
// tile (K+1, K+1) runs first (block 0) and, once its tile is updated, sweeps
// it into Pn = A_{K+1,K+1}^{-1} (block size nbn), so the next step needs no
// pivot kernel and that inversion overlaps this step's other tiles.
__global__ void __launch_bounds__(256) k_sw_update(int m, int k0, int nb, double *__restrict__ D,
                                                   const double *__restrict__ P, const double *__restrict__ V,
                                                   const double *__restrict__ C, double *__restrict__ Pn, int nbn,
                                                   int *__restrict__ status) {
  pdl_wait();
  __shared__ double ct[CB][CB + 1], vt[CB][CB + 1];
  const int Kt = k0 / CB, lt = (Kt + 1) * (Kt + 2) / 2 + (Kt + 1);  // index of tile (K+1, K+1)
  int b = blockIdx.x;
  if (Pn) b = b == 0 ? lt : (b - 1 >= lt ? b : b - 1);
  int I = 0;  // lower tile b in row order: (I, J), J <= I
  while ((I + 1) * (I + 2) / 2 <= b) ++I;
  const int J = b - I * (I + 1) / 2;
  const int i0 = I * CB, j0 = J * CB;
  const bool kr = i0 == k0, kc = j0 == k0;
  const int tx = threadIdx.x % CB, ty = threadIdx.x / CB;  // column, first row
  if (!kr && !kc) {
    for (int e = threadIdx.x; e < CB * CB; e += 256) {
      const int a = e / CB, q = e % CB;
      ct[a][q] = (i0 + a < m && q < nb) ? C[(size_t)(i0 + a) * CB + q] : 0.0;
      vt[a][q] = (a < nb && j0 + q < m) ? V[(size_t)a * m + j0 + q] : 0.0;
    }
    __syncthreads();
  }
  const int j = j0 + tx;
  if (j < m)
    for (int rr = ty; rr < CB; rr += 8) {
      const int i = i0 + rr;
      if (i >= m) break;
      double *dij = D + (size_t)i * m + j;
      if (kr && kc) *dij = -P[rr * CB + tx];      // pivot tile
      else if (kr) *dij = V[(size_t)rr * m + j];  // A_KJ = V_J
      else if (kc) *dij = V[(size_t)tx * m + i];  // A_IK = V_I^T
      else {
        double s = 0.0;
        for (int q = 0; q < nb; ++q) s = fma(ct[rr][q], vt[q][tx], s);
        *dij -= s;
      }
    }
  if (!Pn || b != lt) return;  // the same for the whole CTA
  __syncthreads();  // the tile's new values (global, written by this CTA) and ct, vt free
  for (int u = threadIdx.x; u < CB * (CB + 1) / 2; u += 256) {
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    const int c = u - r * (r + 1) / 2;
    if (r < nbn) ct[r][c] = D[(size_t)(i0 + r) * m + j0 + c];
  }
  __syncthreads();
  sweep_block<256>(ct, vt, nbn, Pn, status);
}

// A^{-1} from the swept array: the lower triangle negated and mirrored
__global__ void k_sw_final(int m, double *__restrict__ D) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)m * m) return;
  const int i = (int)(t / m), j = (int)(t % m);
  if (j > i) return;
  const double v = -D[(size_t)i * m + j];
  D[(size_t)i * m + j] = v;
  if (j < i) D[(size_t)j * m + i] = v;
}

// ---------------------------------------------------------------- graph work
// Maximal independent set of the strong graph, the one the greedy visit by
// (degree descending, index ascending) gives: a visited undecided node
// becomes coarse and its strong neighbours fine.  The same set comes out of
// rounds in which every undecided node that outranks all its undecided strong
// neighbours becomes coarse and the undecided neighbours of the new coarse
// nodes become fine (the greedy order restricted to the undecided nodes puts
// such a node first among its neighbours), so the GPU runs rounds.
__device__ __forceinline__ bool mis_beats(int di, int i, int dj, int j) { return di > dj || (di == dj && i < j); }

__global__ void k_mis_deg(int n, const int *__restrict__ rp, const int *__restrict__ col,
                          const unsigned char *__restrict__ strong, int *__restrict__ deg, int *__restrict__ state) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int d = 0;
  for (int k = rp[I]; k < rp[I + 1]; ++k) d += (strong[k] && col[k] != I);
  deg[I] = d;
  state[I] = -1;
}

// flag = undecided nodes that outrank every undecided strong neighbour
__global__ void k_mis_select(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const unsigned char *__restrict__ strong, const int *__restrict__ deg,
                             const int *__restrict__ state, unsigned char *__restrict__ flag, int *__restrict__ left) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  unsigned char f = 0;
  if (state[I] == -1) {
    atomicAdd(left, 1);
    f = 1;
    const int di = deg[I];
    for (int k = rp[I]; k < rp[I + 1] && f; ++k) {
      const int J = col[k];
      if (strong[k] && J != I && state[J] == -1 && !mis_beats(di, I, deg[J], J)) f = 0;
    }
  }
  flag[I] = f;
}

__global__ void k_mis_apply(int n, const int *__restrict__ rp, const int *__restrict__ col,
                            const unsigned char *__restrict__ strong, const unsigned char *__restrict__ flag,
                            int *__restrict__ state) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n || state[I] != -1) return;
  if (flag[I]) {
    state[I] = 1;
    return;
  }
  for (int k = rp[I]; k < rp[I + 1]; ++k)
    if (strong[k] && col[k] != I && flag[col[k]]) {
      state[I] = 0;
      return;
    }
}

// The C/F split into L.cf (1 coarse, 0 fine) on the device.
static int mis_gpu(Level &L, const unsigned char *d_strong, cudaStream_t s) {
  const DevBsr &A = L.A;
  const int n = A.nr;
  AMG_TRY(L.cf.alloc(n));
  if (n == 0) return AMG_OK;
  DBuf<int> deg, left;
  DBuf<unsigned char> flag;
  int *state = L.cf.p;
  AMG_TRY(deg.alloc(n));
  AMG_TRY(flag.alloc(n));
  AMG_TRY(left.alloc(1));
  const int nb = nblk(n, 256);
  launch_k(k_mis_deg, nb, 256, 0, s, n, A.rowptr.p, A.col.p, d_strong, deg.p, state);
  AMG_LAUNCH_CHECK();
  // rounds are queued four at a time between read-backs of the undecided
  // count of the last one (rounds after the last decision change nothing)
  constexpr int kBatch = 4;
  for (int round = 0;; round += kBatch) {
    for (int q = 0; q < kBatch; ++q) {
      AMG_TRY(left.zero(s));
      launch_k(k_mis_select, nb, 256, 0, s, n, A.rowptr.p, A.col.p, d_strong, deg.p, state, flag.p, left.p);
      launch_k(k_mis_apply, nb, 256, 0, s, n, A.rowptr.p, A.col.p, d_strong, flag.p, state);
    }
    AMG_LAUNCH_CHECK();
    int hl = 0;
    AMG_TRY(read_int(left.p, &hl, s));
    if (hl == 0) break;
    if (round > n) {  // every round decides at least the top-ranked undecided node
      set_error("MIS: no progress");
      return AMG_ERR_CUDA;
    }
  }
  return AMG_OK;
}

// flag[I] = (cf[I] == want)
__global__ void k_cf_flag(int n, const int *__restrict__ cf, int want, int *__restrict__ flag) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < n) flag[I] = cf[I] == want;
}

// From the prefix sums of the coarse and fine flags: cidx[I] = coarse index
// of I (or -1), fidx[I] = fine index of I (or -1), fnodes[fine index] = I.
__global__ void k_cf_split(int n, const int *__restrict__ cf, const int *__restrict__ cs, const int *__restrict__ fs,
                           int *__restrict__ cidx, int *__restrict__ fidx, int *__restrict__ fnodes) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const bool c = cf[I] == 1;
  cidx[I] = c ? cs[I] : -1;
  fidx[I] = c ? -1 : fs[I];
  if (!c) fnodes[fs[I]] = I;
}

// rows of the next level's starting test space: the B dofs of each coarse node
__global__ void k_coarse_src(int n, int B, const int *__restrict__ cidx, int *__restrict__ src) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n || cidx[I] < 0) return;
  for (int c = 0; c < B; ++c) src[B * cidx[I] + c] = B * I + c;
}

// Galerkin product A_c = R (A P): patterns by pattern products on the GPU,
// values in fixed order (det::spgemm_numeric).
static int galerkin(const DevBsr &A, const DevBsr &P, const DevBsr &R, DevBsr &Ac, cudaStream_t s) {
  DevBsr AP;
  double tt = now_s();
  AMG_TRY(symbolic_product(A, P, AP, A.b, s));
  trace("AP symbolic", -1, tt);
  tt = now_s();
  AMG_TRY(det::spgemm_numeric(A, P, AP, s));
  AMG_TRY(symbolic_product(R, AP, Ac, A.b, s));
  trace("RAP symbolic", -1, tt);
  tt = now_s();
  AMG_TRY(det::spgemm_numeric(R, AP, Ac, s));
  AMG_CU(cudaStreamSynchronize(s));
  trace("RAP numeric", -1, tt);
  return AMG_OK;
}

// G column indices from the aFSAI output: row I holds its pattern nodes
// (ascending, below I), then I.  A row that breaks this sets *bad (the
// set-up then stops with an error instead of handing on the pattern).
__global__ void k_fsai_cols(int n, int maxg, const int *__restrict__ np, const int *__restrict__ pat,
                            const int *__restrict__ rp, int *__restrict__ col, int *__restrict__ bad) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int I = (int)(t / (maxg + 1)), j = (int)(t % (maxg + 1));
  if (I >= n || j > np[I]) return;
  int c = I;
  if (j < np[I]) {
    c = pat[(size_t)I * maxg + j];
    const int nx = j + 1 < np[I] ? pat[(size_t)I * maxg + j + 1] : I;
    if (c < 0 || c >= nx) {
      atomicExch(bad, 1);
      c = I;
    }
  }
  col[rp[I] + j] = c;
}

// aFSAI(A, G_s, k, rho, eps) into a compact G.
static int run_fsai(const DevBsr &A, const DevBsr *Gs, int k, int rho, double eps, int maxg, DevBsr &G,
                    cudaStream_t s) {
  const int n = A.nr;
  int maxdeg = 0;
  AMG_TRY(A.row_max(s, &maxdeg));
  DBuf<int> np, pat, status;
  DBuf<double> val;
  const int bb = A.b * A.b;
  AMG_TRY(np.alloc(n));
  AMG_TRY(pat.alloc((size_t)n * maxg));
  AMG_TRY(val.alloc((size_t)n * (maxg + 1) * bb));
  AMG_TRY(status.alloc(1));
  AMG_TRY(status.zero(s));
  det::FsaiOut out{np.p, pat.p, val.p};
  AMG_TRY(det::fsai(A, Gs, k, rho, eps, maxg, maxdeg, out, status.p, s));
  int st = 0;
  AMG_TRY(read_int(status.p, &st, s));
  if (st) {
    set_error("aFSAI: non-positive pivot in a row system (matrix not SPD)");
    return st;
  }
  DBuf<int> rp;
  AMG_TRY(rp.alloc(n + 1));
  AMG_TRY(dev_scan(n, np.p, 1, rp.p, s));
  int nnz = 0;
  AMG_TRY(read_int(rp.p + n, &nnz, s));
  AMG_TRY(G.alloc(n, n, nnz, A.b));
  AMG_CU(cudaMemcpyAsync(G.rowptr.p, rp.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  const long nt = (long)n * (maxg + 1);
  AMG_TRY(status.zero(s));
  if (n) launch_k(k_fsai_cols, nblk(nt, 256), 256, 0, s, n, maxg, np.p, pat.p, G.rowptr.p, G.col.p, status.p);
  if (A.b == 1)
    launch_k(k_compact_vals<1>, nblk(nt, 256), 256, 0, s, n, maxg + 1, G.rowptr.p, val.p, G.val.p);
  else
    launch_k(k_compact_vals<3>, nblk(nt * 9, 256), 256, 0, s, n, maxg + 1, G.rowptr.p, val.p, G.val.p);
  AMG_LAUNCH_CHECK();
  AMG_TRY(read_int(status.p, &st, s));
  if (st) {
    set_error("aFSAI: a row pattern is not ascending below its diagonal");
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

// Average time of one first aFSAI pass (k_g steps from the identity pattern,
// the launch of Algorithm 3 that every set-up makes) on level `lev`, timed
// with CUDA events on the handle's stream; the pattern is not compacted.
int bench_fsai(Handle *h, int lev, int reps, double *ms) {
  const Level &L = *h->lev[lev];
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  const int n = L.A.nr, maxg = p.max_g_nodes;
  int maxdeg = 0;
  AMG_TRY(L.A.row_max(s, &maxdeg));
  DBuf<int> np, pat, status;
  DBuf<double> val;
  AMG_TRY(np.alloc(n));
  AMG_TRY(pat.alloc((size_t)n * maxg));
  AMG_TRY(val.alloc((size_t)n * (maxg + 1) * L.A.b * L.A.b));
  AMG_TRY(status.alloc(1));
  AMG_TRY(status.zero(s));
  det::FsaiOut out{np.p, pat.p, val.p};
  AMG_TRY(det::fsai(L.A, nullptr, p.k_g, p.rho_g, p.eps_g, maxg, maxdeg, out, status.p, s));
  cudaEvent_t e0, e1;
  AMG_CU(cudaEventCreate(&e0));
  AMG_CU(cudaEventCreate(&e1));
  AMG_CU(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) AMG_TRY(det::fsai(L.A, nullptr, p.k_g, p.rho_g, p.eps_g, maxg, maxdeg, out, status.p, s));
  AMG_CU(cudaEventRecord(e1, s));
  AMG_CU(cudaEventSynchronize(e1));
  float t = 0.f;
  AMG_CU(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return AMG_OK;
}

// Algorithm 3, first part: the aFSAI factor G of the level, then the
// Lanczos estimate of lambda_max(G A G^T) queued on the second stream into
// `out` (3 doubles); smoother_finish waits for it.  The test space of the
// level (S = G A G^T, no omega) is generated on the main stream meanwhile.
static int smoother_start(Handle *h, Level &L, int level, DBuf<double> &out) {
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  double tt = now_s();
  AMG_TRY(run_fsai(L.A, nullptr, p.k_g, p.rho_g, p.eps_g, p.max_g_nodes, L.G, s));
  trace("aFSAI", level, tt);
  tt = now_s();
  AMG_TRY(transpose_bsr(L.G, L.GT, s));
  trace("G transpose", level, tt);
  AMG_TRY(out.alloc(3));
  if (!h->aux) {
    AMG_CU(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    AMG_CU(cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming));
    AMG_CU(cudaEventCreateWithFlags(&h->ev_aux, cudaEventDisableTiming));
  }
  // A, G, G^T and out are ready in the order of s
  AMG_CU(cudaEventRecord(h->ev_main, s));
  AMG_CU(cudaStreamWaitEvent(h->aux, h->ev_main, 0));
  {
    StreamScope scope(h->aux);
    AMG_TRY(det::lanczos(L.A, L.G, L.GT, p.lanczos_m, p.seed, level, p.omega_safety, out.p, h->aux, false));
  }
  AMG_CU(cudaEventRecord(h->ev_aux, h->aux));
  return AMG_OK;
}

// Algorithm 3, second part: omega from the estimate; while the smoother is
// too weak and G not yet too dense, refine G (each refinement re-estimates
// on the main stream).  refined tells the caller that G changed.
static int smoother_finish(Handle *h, Level &L, int level, DBuf<double> &out, bool &refined) {
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  double ho[3];
  double tt = now_s();
  AMG_CU(cudaEventSynchronize(h->ev_aux));
  trace("Lanczos wait", level, tt);
  AMG_CU(cudaMemcpy(ho, out.p, sizeof ho, cudaMemcpyDeviceToHost));
  int passes = 0;
  while (ho[1] < p.omega_bar && (double)L.G.nnzb / (double)L.G.nr < p.rho_bar && passes < p.max_refine) {
    DevBsr G2;
    AMG_TRY(run_fsai(L.A, &L.G, p.k_i, p.rho_i, p.eps_i, p.max_g_nodes, G2, s));
    L.G = std::move(G2);
    L.GT = DevBsr();
    AMG_TRY(transpose_bsr(L.G, L.GT, s));
    AMG_TRY(det::lanczos(L.A, L.G, L.GT, p.lanczos_m, p.seed, level, p.omega_safety, out.p, s));
    AMG_CU(cudaMemcpy(ho, out.p, sizeof ho, cudaMemcpyDeviceToHost));
    ++passes;
  }
  L.lmax = ho[0];
  L.omega = ho[2];
  L.npasses = passes;
  refined = passes > 0;
  return AMG_OK;
}

// Candidate sets of the fine nodes on the GPU (d_p <= 2): the coarse nodes
// within d_p strong edges of node I are the union of the strong coarse
// neighbours of I and, for d_p = 2, of each strong neighbour of I; one warp
// per fine node merges these sorted lists (as in k_sym_merge), skipping
// entries that are not strong, not coarse or the row's own node.  Pass 0
// counts, pass 1 writes.
__device__ __forceinline__ int cand_next(int pos, int end, int row, const int *__restrict__ col,
                                         const unsigned char *__restrict__ strong, const int *__restrict__ cf) {
  while (pos < end && !(strong[pos] && col[pos] != row && cf[col[pos]] == 1)) ++pos;
  return pos;
}

__global__ void __launch_bounds__(128) k_dpls_cand(int nf, const int *__restrict__ fnodes, int d_p,
                                                   const int *__restrict__ rp, const int *__restrict__ col,
                                                   const unsigned char *__restrict__ strong,
                                                   const int *__restrict__ cf, const int *__restrict__ cptr,
                                                   int *__restrict__ cand, int *__restrict__ cnt) {
  pdl_wait();
  constexpr int PER = 8, MAXL = 32 * PER;
  __shared__ int nbr[4][MAXL];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (f >= nf) return;
  const int I = fnodes[f];
  // lists: 0 = row I; 1 + q = row of the q-th strong neighbour of I
  int nl = 1;
  if (d_p >= 2) {
    for (int b = rp[I]; b < rp[I + 1]; b += 32) {
      const int k = b + lane;
      const bool sn = k < rp[I + 1] && strong[k] && col[k] != I;
      const unsigned bal = __ballot_sync(0xffffffffu, sn);
      const int at = nl - 1 + __popc(bal & ((1u << lane) - 1u));
      if (sn && at < MAXL) nbr[w][at] = col[k];
      nl += __popc(bal);
    }
    __syncwarp();
  }
  if (d_p <= 0) nl = 0;
  int row[PER], pos[PER], end[PER];
  for (int u = 0; u < PER; ++u) {
    const int q = lane + 32 * u;
    row[u] = -1;
    pos[u] = end[u] = 0;
    if (q < nl && q <= MAXL) {
      row[u] = q == 0 ? I : nbr[w][q - 1];
      end[u] = rp[row[u] + 1];
      pos[u] = cand_next(rp[row[u]], end[u], row[u], col, strong, cf);
    }
  }
  int out = cand ? cptr[f] : 0, n = 0;
  for (;;) {
    int h = 0x7fffffff;
    for (int u = 0; u < PER; ++u)
      if (pos[u] < end[u]) h = min(h, col[pos[u]]);
    for (int off = 16; off >= 1; off >>= 1) h = min(h, __shfl_xor_sync(0xffffffffu, h, off));
    if (h == 0x7fffffff) break;
    if (lane == 0 && cand) cand[out + n] = h;
    ++n;
    for (int u = 0; u < PER; ++u)
      if (pos[u] < end[u] && col[pos[u]] == h) pos[u] = cand_next(pos[u] + 1, end[u], row[u], col, strong, cf);
  }
  if (lane == 0 && !cand) cnt[f] = n;
}

// P row lengths: 1 for a coarse node, its DPLS count for a fine node
__global__ void k_p_len(int n, const int *__restrict__ fidx, const int *__restrict__ cnt, int *__restrict__ len) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < n) len[I] = fidx[I] < 0 ? 1 : cnt[fidx[I]];
}

// P columns: the coarse index of a coarse node, the DPLS columns of a fine one
__global__ void k_p_cols(int n, int cap, const int *__restrict__ cidx, const int *__restrict__ fidx,
                         const int *__restrict__ fcol, const int *__restrict__ rp, int *__restrict__ col) {
  pdl_wait();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int I = (int)(t / cap), j = (int)(t % cap);
  if (I >= n || j >= rp[I + 1] - rp[I]) return;
  col[rp[I] + j] = cidx[I] >= 0 ? cidx[I] : fcol[(size_t)fidx[I] * cap + j];
}

// Node numbering of the C/F split of a level (device arrays).
struct CfSplit {
  DBuf<int> cidx, fidx, fnodes;
  int nc = 0, nf = 0;
};

static int split_nodes(const Level &L, CfSplit &c, cudaStream_t s) {
  const int n = L.n;
  DBuf<int> flag, cs, fs;
  AMG_TRY(flag.alloc(n));
  AMG_TRY(cs.alloc(n + 1));
  AMG_TRY(fs.alloc(n + 1));
  const int nb = nblk(n, 256);
  if (n) launch_k(k_cf_flag, nb, 256, 0, s, n, L.cf.p, 1, flag.p);
  AMG_TRY(dev_scan(n, flag.p, 0, cs.p, s));
  if (n) launch_k(k_cf_flag, nb, 256, 0, s, n, L.cf.p, 0, flag.p);
  AMG_TRY(dev_scan(n, flag.p, 0, fs.p, s));
  AMG_TRY(read_int(cs.p + n, &c.nc, s));
  c.nf = n - c.nc;
  AMG_TRY(c.cidx.alloc(n));
  AMG_TRY(c.fidx.alloc(n));
  AMG_TRY(c.fnodes.alloc(c.nf));
  if (n) launch_k(k_cf_split, nb, 256, 0, s, n, L.cf.p, cs.p, fs.p, c.cidx.p, c.fidx.p, c.fnodes.p);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int build_P(Handle *h, Level &L, const unsigned char *d_strong, const CfSplit &c) {
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  const int n = L.n, t = p.n_tv, nf = c.nf;
  L.nc = c.nc;
  double tt = now_s();
  const int B = L.A.b, BB = B * B;
  const int cap = std::max(1, std::min(p.n_max, t / B));
  DBuf<int> d_cptr, d_cand, d_cnt, d_col;
  DBuf<double> d_val;
  AMG_TRY(d_cptr.alloc(nf + 1));
  AMG_TRY(d_cnt.alloc(nf));
  AMG_TRY(d_col.alloc((size_t)nf * cap));
  AMG_TRY(d_val.alloc((size_t)nf * cap * BB));
  int maxdeg = 0;
  AMG_TRY(L.A.row_max(s, &maxdeg));
  if (nf && p.d_p <= 2 && maxdeg < 256) {
    const int nb = nblk(32L * nf, 128);
    launch_k(k_dpls_cand, nb, 128, 0, s, nf, c.fnodes.p, p.d_p, L.A.rowptr.p, L.A.col.p, d_strong, L.cf.p,
                                              nullptr, nullptr, d_cnt.p);
    AMG_LAUNCH_CHECK();
    AMG_TRY(dev_scan(nf, d_cnt.p, 0, d_cptr.p, s));
    int ncand = 0;
    AMG_TRY(read_int(d_cptr.p + nf, &ncand, s));
    AMG_TRY(d_cand.alloc(ncand));
    launch_k(k_dpls_cand, nb, 128, 0, s, nf, c.fnodes.p, p.d_p, L.A.rowptr.p, L.A.col.p, d_strong, L.cf.p,
                                              d_cptr.p, d_cand.p, nullptr);
    AMG_LAUNCH_CHECK();
  } else if (nf) {  // longer rows or a larger distance: products of patterns
    AMG_TRY(dpls_candidates_gpu(L.A, d_strong, L.cf.p, c.fnodes.p, nf, p.d_p, d_cptr.p, d_cand, s));
  }
  trace("DPLS candidates", -1, tt);
  tt = now_s();
  if (nf) {
    AMG_TRY(det::dpls(L.A, nullptr, nullptr, c.cidx.p, c.fnodes.p, nf, d_cptr.p, d_cand.p, t, L.V.p, p.n_max,
                      p.kappa_p, d_cnt.p, d_col.p, d_val.p, nullptr, s));
  }
  trace("DPLS kernel", -1, tt);
  DBuf<int> len, rp;
  AMG_TRY(len.alloc(n));
  AMG_TRY(rp.alloc(n + 1));
  if (n) launch_k(k_p_len, nblk(n, 256), 256, 0, s, n, c.fidx.p, d_cnt.p, len.p);
  AMG_TRY(dev_scan(n, len.p, 0, rp.p, s));
  int nnz = 0;
  AMG_TRY(read_int(rp.p + n, &nnz, s));
  AMG_TRY(L.P.alloc(n, c.nc, nnz, B));
  AMG_CU(cudaMemcpyAsync(L.P.rowptr.p, rp.p, (n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (n)
    launch_k(k_p_cols, nblk((long)n * cap, 256), 256, 0, s, n, cap, c.cidx.p, c.fidx.p, d_col.p, L.P.rowptr.p,
                                                                  L.P.col.p);
  if (B == 1)
    launch_k(k_p_vals<1>, nblk((long)n * cap, 256), 256, 0, s, n, L.P.rowptr.p, c.fidx.p, cap, d_val.p,
                                                                     L.P.val.p);
  else
    launch_k(k_p_vals<3>, nblk((long)n * cap * 9, 256), 256, 0, s, n, L.P.rowptr.p, c.fidx.p, cap, d_val.p,
                                                                      L.P.val.p);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

static int coarse_factor(Handle *h, Level &L) {
  cudaStream_t s = h->stream;
  const int m = L.A.b * L.n;
  if (m > 6000) {
    set_error("last level has %d dofs; the dense coarse solve supports at most 6000", m);
    return AMG_ERR_COARSENING;
  }
  h->nL = m;
  DBuf<double> Pk, V, C;
  DBuf<int> st;
  AMG_TRY(st.alloc(1));
  AMG_TRY(st.zero(s));
  AMG_TRY(h->Cinv.alloc((size_t)m * m));
  AMG_TRY(h->Cinv.zero(s));
  if (L.n > 0) {
    AMG_TRY(Pk.alloc(2 * CB * CB));
    AMG_TRY(V.alloc((size_t)CB * m));
    AMG_TRY(C.alloc((size_t)m * CB));
    double *D = h->Cinv.p;
    if (L.A.b == 1) launch_k(k_to_dense<1>, L.n, 128, 0, s, L.n, L.A.rowptr.p, L.A.col.p, L.A.val.p, D);
    else launch_k(k_to_dense<3>, L.n, 288, 0, s, L.n, L.A.rowptr.p, L.A.col.p, L.A.val.p, D);
    const int nt = (m + CB - 1) / CB;
    // the pivot inverses alternate between two buffers: step K reads its own
    // while its update kernel writes the next one
    double *Pb[2] = {Pk.p, Pk.p + CB * CB};
    launch_k(k_sw_pivot, 1, SW_THREADS, 0, s, m, 0, m < CB ? m : CB, (const double *)D, Pb[0], st.p);
    for (int k0 = 0, K = 0; k0 < m; k0 += CB, ++K) {
      const int nb = m - k0 < CB ? m - k0 : CB;
      const int k1 = k0 + CB, nbn = k1 < m ? (m - k1 < CB ? m - k1 : CB) : 0;
      double *Pc = Pb[K & 1], *Pn = nbn > 0 ? Pb[(K + 1) & 1] : nullptr;
      launch_k(k_sw_panels, nblk((long)CB * m, 256), 256, 0, s, m, k0, nb, (const double *)D, (const double *)Pc,
               V.p, C.p);
      launch_k(k_sw_update, nt * (nt + 1) / 2, 256, 0, s, m, k0, nb, D, (const double *)Pc, (const double *)V.p,
               (const double *)C.p, Pn, nbn, st.p);
    }
    launch_k(k_sw_final, nblk((long)m * m, 256), 256, 0, s, m, D);
    AMG_LAUNCH_CHECK();
  }
  int hs = 0;
  AMG_CU(cudaMemcpyAsync(&hs, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  if (hs) {
    set_error("coarse-level inverse: non-positive pivot");
    return hs;
  }
  return AMG_OK;
}

// First invalid row of a level-0 pattern (else *bad stays n): row pointers
// start at 0, do not decrease and stay within [0, nnzb]; columns lie in
// [0, n) and increase strictly along a row.  Columns are read only between
// valid row pointers.
__global__ void k_check_pattern(int n, int nnzb, const int *__restrict__ rp, const int *__restrict__ col,
                                int *__restrict__ bad) {
  pdl_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > n) return;
  if (I == n) {
    if (rp[n] != nnzb) atomicMin(bad, n > 0 ? n - 1 : 0);
    return;
  }
  const int b = rp[I], e = rp[I + 1];
  if ((I == 0 && b != 0) || b < 0 || e < b || e > nnzb) {
    atomicMin(bad, I);
    return;
  }
  for (int k = b; k < e; ++k) {
    const int J = col[k];
    if (J < 0 || J >= n || (k > b && col[k - 1] >= J)) {
      atomicMin(bad, I);
      return;
    }
  }
}

void free_hierarchy(Handle *h) {
  h->lev.clear();
  h->nlev = 0;
  h->Cinv.release();
  h->nL = 0;
}

int build_hierarchy(Handle *h, const int *rowptr, const int *col, const double *vals, int mem, int ntv0,
                    const double *V0, int memV, bool keep_pattern) {
  PdlScope pdl;
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  const int t = p.n_tv;
  const double t_start = now_s();
  double T_sm = 0, T_ts = 0, T_cs = 0, T_pl = 0, T_rap = 0;
  const cudaMemcpyKind kind = mem == AMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  auto L0 = std::make_unique<Level>();
  if (keep_pattern && !h->lev.empty() && h->lev[0]->A.nr == h->n) {
    // new values on the pattern already held (checked when it was set up)
    L0->A = std::move(h->lev[0]->A);
    L0->n = L0->A.nr;
    free_hierarchy(h);
    AMG_CU(cudaMemcpyAsync(L0->A.val.p, vals, (size_t)L0->A.nnzb * h->b * h->b * sizeof(double), kind, s));
  } else {
    free_hierarchy(h);
    if (!rowptr || !col) {
      set_error("no level-0 pattern to reuse");
      return AMG_ERR_ARG;
    }
    const int n = h->n;
    int nnzb = 0;
    if (mem == AMG_MEM_HOST) nnzb = rowptr[n];
    else AMG_TRY(read_int(rowptr + n, &nnzb, s));
    if (nnzb < 0) {
      set_error("K pattern: negative entry count %d", nnzb);
      return AMG_ERR_ARG;
    }
    AMG_TRY(L0->A.alloc(n, n, nnzb, h->b));
    AMG_CU(cudaMemcpyAsync(L0->A.rowptr.p, rowptr, (n + 1) * sizeof(int), kind, s));
    if (nnzb) AMG_CU(cudaMemcpyAsync(L0->A.col.p, col, (size_t)nnzb * sizeof(int), kind, s));
    DBuf<int> bad;
    AMG_TRY(bad.alloc(1));
    AMG_CU(cudaMemcpyAsync(bad.p, &n, sizeof(int), cudaMemcpyHostToDevice, s));
    launch_k(k_check_pattern, nblk(n + 1, 256), 256, 0, s, n, nnzb, L0->A.rowptr.p, L0->A.col.p, bad.p);
    AMG_LAUNCH_CHECK();
    int hb = n;
    AMG_TRY(read_int(bad.p, &hb, s));
    if (hb < n) {
      set_error("K pattern: row %d has an invalid row pointer or an invalid or unsorted column index", hb);
      return AMG_ERR_ARG;
    }
    AMG_CU(cudaMemcpyAsync(L0->A.val.p, vals, (size_t)nnzb * h->b * h->b * sizeof(double), kind, s));
    L0->n = n;
  }
  // starting test space: V0 padded with counter-generator columns
  DBuf<double> Vin;
  {
    const int n3 = h->b * h->n;
    AMG_TRY(Vin.alloc((size_t)n3 * t));
    if (ntv0 > 0)
      AMG_CU(cudaMemcpyAsync(Vin.p, V0, (size_t)n3 * ntv0 * sizeof(double),
                             memV == AMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (ntv0 > 0 && V0 != h->V0keep.p) {
      AMG_TRY(h->V0keep.alloc((size_t)n3 * ntv0));
      AMG_CU(cudaMemcpyAsync(h->V0keep.p, Vin.p, (size_t)n3 * ntv0 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    h->ntv0 = ntv0;
    AMG_TRY(det::uniform_fill(Vin.p, n3, ntv0, t - ntv0, p.seed, s));
  }
  h->lev.push_back(std::move(L0));
  DBuf<unsigned char> d_strong;
  for (int k = 0;; ++k) {
    Level &L = *h->lev[k];
    const int B = h->b;
    const int n3 = B * L.n;
    if (n3 <= p.n_coarse || k == p.max_levels - 1 || k == 31) break;
    double t0 = now_s();
    DBuf<double> om;
    // on every way out of this level (errors included) the second stream has
    // finished writing om before om is freed
    struct AuxDone {
      Handle *h;
      ~AuxDone() {
        if (h->aux) cudaStreamSynchronize(h->aux);
      }
    } aux_done{h};
    AMG_TRY(smoother_start(h, L, k, om));
    double t1 = now_s();
    T_sm += t1 - t0;
    AMG_TRY(L.V.alloc((size_t)n3 * t));
    DBuf<int> st;
    AMG_TRY(st.alloc(1));
    double tw = 0.0;
    for (int attempt = 0;; ++attempt) {
      AMG_TRY(st.zero(s));
      AMG_TRY(det::srqcg(L.A, L.G, L.GT, p.n_rq, p.k_ritz, t, Vin.p, L.V.p, st.p, s));
      trace("SRQCG", k, t1);
      if (attempt > 0) break;
      // the test space used G as first built; a refined G needs a new one
      bool refined = false;
      const double tf = now_s();
      AMG_TRY(smoother_finish(h, L, k, om, refined));
      tw = now_s() - tf;
      if (!refined) break;
    }
    int hs = 0;
    AMG_CU(cudaMemcpy(&hs, st.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (hs) {
      set_error("SRQCG: Ritz step lost rank");
      return hs;
    }
    double t2 = now_s();
    T_sm += tw;
    T_ts += t2 - t1 - tw;
    AMG_TRY(d_strong.alloc(L.A.nnzb));
    AMG_TRY(det::soc_filter(L.A, t, L.V.p, p.theta, d_strong.p, s));
    trace("SoC filter", k, t2);
    double tm = now_s();
    AMG_TRY(mis_gpu(L, d_strong.p, s));
    CfSplit split;
    AMG_TRY(split_nodes(L, split, s));
    trace("MIS", k, tm);
    const int nc = split.nc;
    double t3 = now_s();
    T_cs += t3 - t2;
    if (nc == 0 || (double)nc > p.max_coarse_ratio * (double)L.n) {
      L.G = DevBsr();
      L.GT = DevBsr();
      L.V.release();
      L.cf.release();
      break;
    }
    AMG_TRY(build_P(h, L, d_strong.p, split));
    AMG_TRY(transpose_bsr(L.P, L.R, s));
    double t4 = now_s();
    T_pl += t4 - t3;
    auto Ln = std::make_unique<Level>();
    AMG_TRY(galerkin(L.A, L.P, L.R, Ln->A, s));
    Ln->n = Ln->A.nr;
    double t5 = now_s();
    T_rap += t5 - t4;
    // next level's starting test space: rows of the coarse nodes
    {
      DBuf<int> dsrc;
      AMG_TRY(dsrc.alloc((size_t)B * nc));
      launch_k(k_coarse_src, nblk(L.n, 256), 256, 0, s, L.n, B, split.cidx.p, dsrc.p);
      AMG_LAUNCH_CHECK();
      DBuf<double> Vn;
      AMG_TRY(Vn.alloc((size_t)B * nc * t));
      AMG_TRY(det::gather_rows(dsrc.p, B * nc, n3, t, L.V.p, Vn.p, s));
      AMG_CU(cudaStreamSynchronize(s));
      Vin = std::move(Vn);
    }
    h->lev.push_back(std::move(Ln));
    T_ts += now_s() - t5;
  }
  h->nlev = (int)h->lev.size();
  const double t6 = now_s();
  AMG_TRY(coarse_factor(h, *h->lev[h->nlev - 1]));
  trace("coarse inverse", h->nlev - 1, t6);
  const double t7 = now_s();
  AMG_TRY(prepare_solve(h));
  AMG_CU(cudaStreamSynchronize(s));
  trace("solve layout", -1, t7);
  const double t_end = now_s();
  amg_stats &st = h->stats;
  st.nlev = h->nlev;
  st.T_sm = T_sm;
  st.T_ts = T_ts;
  st.T_cs = T_cs;
  st.T_pl = T_pl;
  st.T_rap = T_rap + (t_end - t6);
  st.T_p = t_end - t_start;
  double rows = 0, nnz = 0, gnnz = 0;
  for (int k = 0; k < h->nlev && k < 32; ++k) {
    const Level &L = *h->lev[k];
    rows += L.n;
    nnz += L.A.nnzb;
    gnnz += L.G.nnzb;
    st.level_nodes[k] = L.n;
    st.level_nnzb[k] = L.A.nnzb;
    st.level_g_nnzb[k] = L.G.nnzb;
    st.level_omega[k] = L.omega;
  }
  const Level &L0r = *h->lev[0];
  st.C_gd = rows / (double)L0r.n;
  st.C_op = nnz / (double)L0r.A.nnzb;
  st.C_fs = gnnz / (double)L0r.A.nnzb;
  return AMG_OK;
}

}  // namespace amg
