// Hierarchy set-up (Algorithm 1 of the paper): per level the aFSAI smoother
// (Algorithm 3), the SRQCG test space (Algorithm 4), the affinity C/F split
// (Sec. 3.3), DPLS prolongation (Algorithm 5) and the Galerkin product.
// Floating-point work runs in the kernels of det.cu; this file does the
// control flow and the integer graph work (pattern compaction and
// transposition, DPLS candidate sets and the symbolic Galerkin pattern) on
// the host; the maximal independent set runs in rounds on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>

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

// T.val[dst] = transpose(A.val[perm[dst]])
template <int B>
__global__ void k_transpose_vals(int nnzb, const int *__restrict__ perm, const double *__restrict__ src,
                                 double *__restrict__ dst) {
  constexpr int BB = B * B;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)BB * nnzb) return;
  const int q = (int)(t / BB), e = (int)(t % BB), r = e / B, c = e % B;
  dst[(size_t)q * BB + c * B + r] = src[(size_t)perm[q] * BB + e];
}

// P values: identity for coarse rows, DPLS blocks for fine rows.
template <int B>
__global__ void k_p_vals(int n, const int *__restrict__ rowptr, const int *__restrict__ fidx, int cap,
                         const double *__restrict__ fval, double *__restrict__ pv) {
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
  constexpr int BB = B * B;
  const int I = blockIdx.x;
  const long m = (long)B * nr;
  for (int k = rp[I] + threadIdx.x / BB; k < rp[I + 1]; k += blockDim.x / BB) {
    if ((int)threadIdx.x >= (blockDim.x / BB) * BB) break;
    const int e = threadIdx.x % BB, r = e / B, c = e % B;
    D[(size_t)((long)B * I + r) * m + (long)B * col[k] + c] = val[(size_t)k * BB + e];
  }
}

// Explicit inverse of the last level's matrix by blocked Gauss-Jordan
// elimination, in place in a dense row-major m x m array, pivot blocks of CB
// columns.  No pivoting is needed: every pivot block is a Schur complement of
// an SPD matrix, hence SPD.  Step k (block rows/columns [k0, k0+nb)):
// P = A_kk^{-1}; R = P A_kj and C = A_ik (copies of the pivot row and column
// panels); then A_ij -= C_i R_j for i, j outside the block, A_ik = -C_i P,
// A_kj = R_j and A_kk = P.  The coarse solve is then one dense product with
// the (symmetric) inverse.  Each step's update is m^2 CB independent
// multiply-adds spread over all SMs; only the CB x CB pivot inversion is
// serial.
constexpr int CB = 32;

// P = A_kk^{-1} by scalar Gauss-Jordan in shared memory (one CTA, one
// thread per entry); a pivot that is not positive sets status
__global__ void __launch_bounds__(CB *CB) k_gj_pivot(int m, int k0, int nb, const double *__restrict__ D,
                                                     double *__restrict__ P, int *__restrict__ status) {
  __shared__ double a[CB][CB + 1];
  __shared__ double rinv;
  __shared__ int bad;
  const int r = threadIdx.x / CB, c = threadIdx.x % CB;
  if (threadIdx.x == 0) bad = 0;
  if (r < nb && c < nb) a[r][c] = D[(size_t)(k0 + r) * m + k0 + c];
  for (int j = 0; j < nb; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const double pv = a[j][j];
      if (!(pv > 0.0)) bad = 1;
      rinv = 1.0 / pv;
    }
    __syncthreads();
    if (bad) break;
    if (r == j && c < nb) a[j][c] = (c == j) ? rinv : a[j][c] * rinv;
    __syncthreads();
    double f = 0.0, rowj = 0.0;
    if (r < nb && c < nb && r != j) {
      f = a[r][j];
      rowj = a[j][c];
    }
    __syncthreads();
    if (r < nb && c < nb && r != j) a[r][c] = (c == j) ? -f * rinv : fma(-f, rowj, a[r][c]);
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicMin(status, AMG_ERR_NOT_SPD);
    return;
  }
  if (r < nb && c < nb) P[r * CB + c] = a[r][c];
}

// R[q][j] = sum_p P[q][p] A[k0+p][j] (pivot row panel times P) and
// C[i][q] = A[i][k0+q] (pivot column panel), for every i, j of the matrix
__global__ void k_gj_panels(int m, int k0, int nb, const double *__restrict__ D, const double *__restrict__ P,
                            double *__restrict__ R, double *__restrict__ C) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)CB * m) return;
  const int q = (int)(t / m), j = (int)(t % m);
  if (q >= nb) return;
  double s = 0.0;
  for (int p = 0; p < nb; ++p) s = fma(P[q * CB + p], D[(size_t)(k0 + p) * m + j], s);
  R[(size_t)q * m + j] = s;
  C[(size_t)j * CB + q] = D[(size_t)j * m + k0 + q];
}

// every entry of the matrix for step k, 32 x 32 tiles, 256 threads (4 rows each)
__global__ void __launch_bounds__(256) k_gj_update(int m, int k0, int nb, double *__restrict__ D,
                                                   const double *__restrict__ P, const double *__restrict__ R,
                                                   const double *__restrict__ C) {
  __shared__ double ct[CB][CB + 1], rt[CB][CB + 1];
  const int i0 = blockIdx.y * CB, j0 = blockIdx.x * CB;
  const bool kr = i0 == k0, kc = j0 == k0;
  const int tx = threadIdx.x % CB, ty = threadIdx.x / CB;  // column, first row
  for (int e = threadIdx.x; e < CB * CB; e += 256) {
    const int a = e / CB, b = e % CB;
    // C rows of this tile; R columns of this tile (P for the pivot column)
    ct[a][b] = (i0 + a < m && b < nb) ? C[(size_t)(i0 + a) * CB + b] : 0.0;
    rt[a][b] = (a < nb && j0 + b < m) ? (kc ? (b < nb ? P[a * CB + b] : 0.0) : R[(size_t)a * m + j0 + b]) : 0.0;
  }
  __syncthreads();
  const int j = j0 + tx;
  if (j >= m) return;
  for (int rr = ty; rr < CB; rr += 8) {
    const int i = i0 + rr;
    if (i >= m) break;
    double *dij = D + (size_t)i * m + j;
    if (kr) {
      if (tx < CB) *dij = kc ? (tx < nb && rr < nb ? P[rr * CB + tx] : *dij) : R[(size_t)rr * m + j];
      continue;
    }
    double s = 0.0;
    for (int q = 0; q < nb; ++q) s = fma(ct[rr][q], rt[q][tx], s);
    *dij = kc ? -s : *dij - s;
  }
}

// ---------------------------------------------------------------- host graph work
int transpose_bsr(const DevBsr &A, DevBsr &T, cudaStream_t s) {
  const int nnzb = A.nnzb;
  AMG_TRY(T.alloc(A.nc, A.nr, nnzb, A.b));
  T.h_rowptr.assign(A.nc + 1, 0);
  T.h_col.resize(nnzb);
  std::vector<int> perm(nnzb > 0 ? nnzb : 1);
  for (int k = 0; k < nnzb; ++k) T.h_rowptr[A.h_col[k] + 1]++;
  for (int i = 0; i < A.nc; ++i) T.h_rowptr[i + 1] += T.h_rowptr[i];
  std::vector<int> next(T.h_rowptr.begin(), T.h_rowptr.end() - 1);
  for (int I = 0; I < A.nr; ++I)
    for (int k = A.h_rowptr[I]; k < A.h_rowptr[I + 1]; ++k) {
      const int dst = next[A.h_col[k]]++;
      T.h_col[dst] = I;
      perm[dst] = k;
    }
  AMG_TRY(T.upload_pattern(s));
  if (nnzb) {
    DBuf<int> dperm;
    AMG_TRY(dperm.alloc(nnzb));
    AMG_CU(cudaMemcpyAsync(dperm.p, perm.data(), nnzb * sizeof(int), cudaMemcpyHostToDevice, s));
    if (A.b == 1)
      AMG_KCOUNT k_transpose_vals<1><<<nblk((long)nnzb, 256), 256, 0, s>>>(nnzb, dperm.p, A.val.p, T.val.p);
    else
      AMG_KCOUNT k_transpose_vals<3><<<nblk(9L * nnzb, 256), 256, 0, s>>>(nnzb, dperm.p, A.val.p, T.val.p);
    AMG_LAUNCH_CHECK();
    AMG_CU(cudaStreamSynchronize(s));
  }
  return AMG_OK;
}

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

static int mis_gpu(const DevBsr &A, const unsigned char *d_strong, std::vector<int> &cf, cudaStream_t s) {
  const int n = A.nr;
  cf.assign(n, 0);
  if (n == 0) return AMG_OK;
  DBuf<int> deg, state, left;
  DBuf<unsigned char> flag;
  AMG_TRY(deg.alloc(n));
  AMG_TRY(state.alloc(n));
  AMG_TRY(flag.alloc(n));
  AMG_TRY(left.alloc(1));
  const int nb = nblk(n, 256);
  AMG_KCOUNT k_mis_deg<<<nb, 256, 0, s>>>(n, A.rowptr.p, A.col.p, d_strong, deg.p, state.p);
  AMG_LAUNCH_CHECK();
  for (int round = 0;; ++round) {
    AMG_TRY(left.zero(s));
    AMG_KCOUNT k_mis_select<<<nb, 256, 0, s>>>(n, A.rowptr.p, A.col.p, d_strong, deg.p, state.p, flag.p, left.p);
    AMG_KCOUNT k_mis_apply<<<nb, 256, 0, s>>>(n, A.rowptr.p, A.col.p, d_strong, flag.p, state.p);
    AMG_LAUNCH_CHECK();
    int hl = 0;
    AMG_CU(cudaMemcpyAsync(&hl, left.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
    if (hl == 0) break;
    if (round > n) {  // every round decides at least the top-ranked undecided node
      set_error("MIS: no progress");
      return AMG_ERR_CUDA;
    }
  }
  AMG_CU(cudaMemcpy(cf.data(), state.p, n * sizeof(int), cudaMemcpyDeviceToHost));
  return AMG_OK;
}

// Host worker pool for the row-parallel graph work: rows are cut into
// contiguous ranges, each range produces its own output in row order, and the
// ranges are concatenated in order, so the result does not depend on the
// number of threads.
static int host_threads() {
  static const int n = [] {
    const char *e = getenv("AMG_HOST_THREADS");
    int v = e ? atoi(e) : (int)std::thread::hardware_concurrency();
    return v < 1 ? 1 : (v > 64 ? 64 : v);
  }();
  return n;
}

// Persistent workers: parallel_ranges hands each worker one contiguous range
// and waits for all of them (threads are created once per process).
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool(host_threads());
    return pool;
  }
  void run(int nt, const std::function<void(int)> &job) {
    std::lock_guard<std::mutex> one_at_a_time(run_mu_);  // callers from several host threads
    std::unique_lock<std::mutex> lock(mu_);
    job_ = &job;
    njobs_ = nt;
    next_ = 1;
    done_ = 0;
    ++epoch_;
    cv_.notify_all();
    lock.unlock();
    job(0);  // the caller takes range 0
    lock.lock();
    ++done_;
    done_cv_.wait(lock, [&] { return done_ == njobs_; });
    job_ = nullptr;
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lock(mu_);
      stop_ = true;
      ++epoch_;
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }

 private:
  explicit HostPool(int n) {
    for (int i = 1; i < n; ++i) th_.emplace_back([this] { loop(); });
  }
  void loop() {
    long seen = 0;
    std::unique_lock<std::mutex> lock(mu_);
    for (;;) {
      cv_.wait(lock, [&] { return stop_ || (epoch_ != seen && job_ && next_ < njobs_); });
      if (stop_) return;
      seen = epoch_;
      while (job_ && next_ < njobs_) {
        const int id = next_++;
        const std::function<void(int)> *job = job_;
        lock.unlock();
        (*job)(id);
        lock.lock();
        if (++done_ == njobs_) done_cv_.notify_all();
      }
    }
  }
  std::vector<std::thread> th_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)> *job_ = nullptr;
  int njobs_ = 0, next_ = 0, done_ = 0;
  long epoch_ = 0;
  bool stop_ = false;
};

template <class F>
static void parallel_ranges(int n, F f) {
  const int nt = std::min(host_threads(), std::max(1, n / 2048));
  if (nt <= 1) {
    f(0, 0, n);
    return;
  }
  const std::function<void(int)> job = [&](int t) {
    const int lo = (int)((long)n * t / nt), hi = (int)((long)n * (t + 1) / nt);
    f(t, lo, hi);
  };
  HostPool::get().run(nt, job);
}

// Concatenates per-range outputs in range order: row lengths into a row
// pointer starting at rp[0], entries into out (both filled in parallel).
static void concat_ranges(const std::vector<std::vector<int>> &len, const std::vector<std::vector<int>> &ent,
                          std::vector<int> &rp, std::vector<int> &out) {
  const int nt = (int)len.size();
  std::vector<long> row0(nt + 1, 0), e0(nt + 1, 0);
  for (int t = 0; t < nt; ++t) {
    row0[t + 1] = row0[t] + (long)len[t].size();
    e0[t + 1] = e0[t] + (long)ent[t].size();
  }
  rp.assign(row0[nt] + 1, 0);
  out.resize(e0[nt]);
  const std::function<void(int)> job = [&](int t) {
    std::copy(ent[t].begin(), ent[t].end(), out.begin() + e0[t]);
    long r = row0[t], acc = e0[t];
    for (int l : len[t]) {
      acc += l;
      rp[++r] = (int)acc;
    }
  };
  if (nt > 1) HostPool::get().run(nt, job);
  else if (nt == 1) job(0);
}

// Coarse nodes within d_p strong edges of every fine node, ascending.
static void dpls_candidates(const DevBsr &A, const std::vector<unsigned char> &strong, const std::vector<int> &cf,
                            int d_p, std::vector<int> &fnodes, std::vector<int> &cptr, std::vector<int> &cand) {
  const int n = A.nr;
  const int nt = std::min(host_threads(), std::max(1, n / 2048));
  std::vector<std::vector<int>> pf(nt), pl(nt), pc(nt);
  parallel_ranges(n, [&](int t, int lo, int hi) {
    std::vector<int> dist(n, -1), front;
    std::vector<int> &fn = pf[t], &len = pl[t], &cd = pc[t];
    for (int I = lo; I < hi; ++I) {
      if (cf[I] == 1) continue;
      fn.push_back(I);
      front.assign(1, I);
      dist[I] = 0;
      const size_t c0 = cd.size();
      for (size_t q = 0; q < front.size(); ++q) {
        const int K = front[q];
        if (dist[K] >= d_p) continue;
        for (int k = A.h_rowptr[K]; k < A.h_rowptr[K + 1]; ++k) {
          const int J = A.h_col[k];
          if (!strong[k] || J == K || dist[J] >= 0) continue;
          dist[J] = dist[K] + 1;
          front.push_back(J);
          if (cf[J] == 1) cd.push_back(J);
        }
      }
      for (int K : front) dist[K] = -1;
      std::sort(cd.begin() + c0, cd.end());
      len.push_back((int)(cd.size() - c0));
    }
  });
  fnodes.clear();
  for (int t = 0; t < (int)pf.size(); ++t) fnodes.insert(fnodes.end(), pf[t].begin(), pf[t].end());
  concat_ranges(pl, pc, cptr, cand);
}

// Pattern of Z = X Y (columns ascending).
static void symbolic_product(const DevBsr &X, const DevBsr &Y, DevBsr &Z) {
  const int nr = X.nr, nc = Y.nc;
  const int nt = std::min(host_threads(), std::max(1, nr / 2048));
  std::vector<std::vector<int>> pcols(nt), plen(nt);
  parallel_ranges(nr, [&](int t, int lo, int hi) {
    std::vector<int> mark(nc, -1), cols;
    std::vector<int> &out = pcols[t], &len = plen[t];
    for (int i = lo; i < hi; ++i) {
      cols.clear();
      for (int kx = X.h_rowptr[i]; kx < X.h_rowptr[i + 1]; ++kx) {
        const int k = X.h_col[kx];
        for (int ky = Y.h_rowptr[k]; ky < Y.h_rowptr[k + 1]; ++ky) {
          const int c = Y.h_col[ky];
          if (mark[c] != i) {
            mark[c] = i;
            cols.push_back(c);
          }
        }
      }
      std::sort(cols.begin(), cols.end());
      out.insert(out.end(), cols.begin(), cols.end());
      len.push_back((int)cols.size());
    }
  });
  concat_ranges(plen, pcols, Z.h_rowptr, Z.h_col);
  Z.nr = nr;
  Z.nc = nc;
  Z.nnzb = (int)Z.h_col.size();
}

// Pattern of Z = X Y on the GPU: row i of Z is the union of the (sorted)
// rows of Y named by row i of X.  One warp per row merges them: lane l holds
// the heads of lists l, l+32, ...; each step takes the warp minimum, emits it
// once and advances every list whose head equals it, so the output is
// ascending and duplicate-free.  Pass 0 counts, pass 1 writes.
__global__ void k_sym_merge(int nr, const int *__restrict__ xr, const int *__restrict__ xc,
                            const int *__restrict__ yr, const int *__restrict__ yc, const int *__restrict__ zr,
                            int *__restrict__ zc, int *__restrict__ cnt) {
  const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nr) return;
  const int l0 = xr[i], nl = xr[i + 1] - l0;
  constexpr int PER = 8;  // lists per lane held in registers
  int pos[PER], end[PER];
  for (int u = 0; u < PER; ++u) {
    const int q = lane + 32 * u;
    if (q < nl) {
      const int k = xc[l0 + q];
      pos[u] = yr[k];
      end[u] = yr[k + 1];
    } else {
      pos[u] = end[u] = 0;
    }
  }
  int out = zc ? zr[i] : 0, n = 0;
  for (;;) {
    int h = 0x7fffffff;
    for (int u = 0; u < PER; ++u)
      if (pos[u] < end[u]) h = min(h, yc[pos[u]]);
    for (int off = 16; off >= 1; off >>= 1) h = min(h, __shfl_xor_sync(0xffffffffu, h, off));
    if (h == 0x7fffffff) break;
    if (lane == 0 && zc) zc[out + n] = h;
    ++n;
    for (int u = 0; u < PER; ++u)
      if (pos[u] < end[u] && yc[pos[u]] == h) ++pos[u];
  }
  if (lane == 0 && !zc) cnt[i] = n;
}

// exclusive prefix sum of n ints into out[0..n] (one block; the host checks
// that n is small enough, else the scan runs on the host)
__global__ void __launch_bounds__(1024) k_scan1(int n, const int *__restrict__ in, int *__restrict__ out) {
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int acc = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    out[i] = acc;
    acc += in[i];
  }
  if (threadIdx.x == 1023) out[n] = part[1023];
}

// Z's pattern on the device (Z.rowptr, Z.col, Z.val allocated); the host
// mirror only when want_host.
static int symbolic_product_gpu(const DevBsr &X, const DevBsr &Y, DevBsr &Z, bool want_host, cudaStream_t s) {
  const int nr = X.nr;
  int maxlen = 0;
  for (int i = 0; i < nr; ++i) maxlen = std::max(maxlen, X.h_rowptr[i + 1] - X.h_rowptr[i]);
  if (maxlen > 32 * 8) return AMG_ERR_ARG;  // caller falls back to the host product
  DBuf<int> cnt, rp;
  AMG_TRY(cnt.alloc(nr));
  AMG_TRY(rp.alloc(nr + 1));
  const int nb = nblk(32L * nr, 256);
  if (nr) AMG_KCOUNT k_sym_merge<<<nb, 256, 0, s>>>(nr, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, nullptr, nullptr, cnt.p);
  AMG_KCOUNT k_scan1<<<1, 1024, 0, s>>>(nr, cnt.p, rp.p);
  AMG_LAUNCH_CHECK();
  int nnz = 0;
  AMG_CU(cudaMemcpyAsync(&nnz, rp.p + nr, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  AMG_TRY(Z.alloc(nr, Y.nc, nnz, X.b));
  AMG_CU(cudaMemcpyAsync(Z.rowptr.p, rp.p, (nr + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (nr) AMG_KCOUNT k_sym_merge<<<nb, 256, 0, s>>>(nr, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, rp.p, Z.col.p, nullptr);
  AMG_LAUNCH_CHECK();
  if (want_host) AMG_TRY(Z.download_pattern(s));
  return AMG_OK;
}

static int galerkin(const DevBsr &A, const DevBsr &P, const DevBsr &R, DevBsr &Ac, cudaStream_t s) {
  DevBsr AP;
  double tt = now_s();
  // AP's pattern stays on the device (its host mirror is only needed when
  // R's rows are too long for the GPU merge)
  int rc = symbolic_product_gpu(A, P, AP, false, s);
  bool ap_host = false;
  if (rc == AMG_ERR_ARG) {
    symbolic_product(A, P, AP);
    AMG_TRY(AP.alloc(AP.nr, AP.nc, AP.nnzb, A.b));
    AMG_TRY(AP.upload_pattern(s));
    ap_host = true;
  } else if (rc) {
    return rc;
  }
  trace("AP symbolic", -1, tt);
  tt = now_s();
  AMG_TRY(det::spgemm_numeric(A, P, AP, s));
  AMG_CU(cudaStreamSynchronize(s));
  trace("AP numeric", -1, tt);
  tt = now_s();
  rc = symbolic_product_gpu(R, AP, Ac, true, s);
  if (rc == AMG_ERR_ARG) {
    if (!ap_host) AMG_TRY(AP.download_pattern(s));
    symbolic_product(R, AP, Ac);
    AMG_TRY(Ac.alloc(Ac.nr, Ac.nc, Ac.nnzb, A.b));
    AMG_TRY(Ac.upload_pattern(s));
  } else if (rc) {
    return rc;
  }
  trace("RAP symbolic", -1, tt);
  tt = now_s();
  AMG_TRY(det::spgemm_numeric(R, AP, Ac, s));
  AMG_CU(cudaStreamSynchronize(s));
  trace("RAP numeric", -1, tt);
  return AMG_OK;
}

// aFSAI(A, G_s, k, rho, eps) into a compact G.
static int run_fsai(const DevBsr &A, const DevBsr *Gs, int k, int rho, double eps, int maxg, DevBsr &G,
                    cudaStream_t s) {
  const int n = A.nr;
  int maxdeg = 0;
  for (int I = 0; I < n; ++I) maxdeg = std::max(maxdeg, A.h_rowptr[I + 1] - A.h_rowptr[I]);
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
  AMG_CU(cudaMemcpy(&st, status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    set_error("aFSAI: non-positive pivot in a row system (matrix not SPD)");
    return st;
  }
  std::vector<int> hnp(n), hpat((size_t)n * maxg);
  AMG_CU(cudaMemcpy(hnp.data(), np.p, n * sizeof(int), cudaMemcpyDeviceToHost));
  AMG_CU(cudaMemcpy(hpat.data(), pat.p, (size_t)n * maxg * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<int> rp(n + 1, 0);
  for (int I = 0; I < n; ++I) rp[I + 1] = rp[I] + hnp[I] + 1;
  std::vector<int> cl(rp[n]);
  parallel_ranges(n, [&](int, int lo, int hi) {
    for (int I = lo; I < hi; ++I) {
      int *o = cl.data() + rp[I];
      for (int j = 0; j < hnp[I]; ++j) o[j] = hpat[(size_t)I * maxg + j];
      o[hnp[I]] = I;
    }
  });
  AMG_TRY(G.alloc(n, n, (int)cl.size(), A.b));
  G.h_rowptr = std::move(rp);
  G.h_col = std::move(cl);
  AMG_TRY(G.upload_pattern(s));
  if (A.b == 1)
    AMG_KCOUNT k_compact_vals<1><<<nblk((long)n * (maxg + 1), 256), 256, 0, s>>>(n, maxg + 1, G.rowptr.p, val.p, G.val.p);
  else
    AMG_KCOUNT k_compact_vals<3><<<nblk((long)n * (maxg + 1) * 9, 256), 256, 0, s>>>(n, maxg + 1, G.rowptr.p, val.p,
                                                                                   G.val.p);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
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
  for (int I = 0; I < n; ++I) maxdeg = std::max(maxdeg, L.A.h_rowptr[I + 1] - L.A.h_rowptr[I]);
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

static int build_P(Handle *h, Level &L, const std::vector<unsigned char> &strong, const unsigned char *d_strong) {
  const amg_params &p = h->prm;
  cudaStream_t s = h->stream;
  const int n = L.n, t = p.n_tv;
  std::vector<int> cidx(n, -1), fnodes;
  int nc = 0;
  for (int I = 0; I < n; ++I) {
    if (L.cf[I] == 1) cidx[I] = nc++;
    else fnodes.push_back(I);
  }
  L.nc = nc;
  double tt = now_s();
  const int nf = (int)fnodes.size();
  const int B = L.A.b, BB = B * B;
  const int cap = std::max(1, std::min(p.n_max, t / B));
  DBuf<int> d_cidx, d_f, d_cptr, d_cand, d_cnt, d_col, d_cf;
  DBuf<double> d_val;
  AMG_TRY(d_cidx.alloc(n));
  AMG_TRY(d_f.alloc(nf));
  AMG_TRY(d_cptr.alloc(nf + 1));
  AMG_TRY(d_cnt.alloc(nf));
  AMG_TRY(d_col.alloc((size_t)nf * cap));
  AMG_TRY(d_val.alloc((size_t)nf * cap * BB));
  AMG_CU(cudaMemcpyAsync(d_cidx.p, cidx.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nf) AMG_CU(cudaMemcpyAsync(d_f.p, fnodes.data(), nf * sizeof(int), cudaMemcpyHostToDevice, s));
  int maxdeg = 0;
  for (int I = 0; I < n; ++I) maxdeg = std::max(maxdeg, L.A.h_rowptr[I + 1] - L.A.h_rowptr[I]);
  if (nf && p.d_p <= 2 && maxdeg < 256) {
    AMG_TRY(d_cf.alloc(n));
    AMG_CU(cudaMemcpyAsync(d_cf.p, L.cf.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    const int nb = nblk(32L * nf, 128);
    AMG_KCOUNT k_dpls_cand<<<nb, 128, 0, s>>>(nf, d_f.p, p.d_p, L.A.rowptr.p, L.A.col.p, d_strong, d_cf.p,
                                              nullptr, nullptr, d_cnt.p);
    AMG_KCOUNT k_scan1<<<1, 1024, 0, s>>>(nf, d_cnt.p, d_cptr.p);
    AMG_LAUNCH_CHECK();
    int ncand = 0;
    AMG_CU(cudaMemcpyAsync(&ncand, d_cptr.p + nf, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
    AMG_TRY(d_cand.alloc(ncand));
    AMG_KCOUNT k_dpls_cand<<<nb, 128, 0, s>>>(nf, d_f.p, p.d_p, L.A.rowptr.p, L.A.col.p, d_strong, d_cf.p,
                                              d_cptr.p, d_cand.p, nullptr);
    AMG_LAUNCH_CHECK();
  } else if (nf) {
    std::vector<int> fn2, cptr, cand;
    dpls_candidates(L.A, strong, L.cf, p.d_p, fn2, cptr, cand);
    AMG_TRY(d_cand.alloc(cand.size()));
    AMG_CU(cudaMemcpyAsync(d_cptr.p, cptr.data(), (nf + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!cand.empty())
      AMG_CU(cudaMemcpyAsync(d_cand.p, cand.data(), cand.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    AMG_CU(cudaStreamSynchronize(s));
  }
  trace("DPLS candidates", -1, tt);
  tt = now_s();
  if (nf) {
    AMG_TRY(det::dpls(L.A, nullptr, nullptr, d_cidx.p, d_f.p, nf, d_cptr.p, d_cand.p, t, L.V.p, p.n_max,
                      p.kappa_p, d_cnt.p, d_col.p, d_val.p, nullptr, s));
  }
  trace("DPLS kernel", -1, tt);
  std::vector<int> hcnt(nf), hcol((size_t)nf * cap), fidx(n, -1);
  if (nf) {
    AMG_CU(cudaMemcpy(hcnt.data(), d_cnt.p, nf * sizeof(int), cudaMemcpyDeviceToHost));
    AMG_CU(cudaMemcpy(hcol.data(), d_col.p, (size_t)nf * cap * sizeof(int), cudaMemcpyDeviceToHost));
  }
  for (int f = 0; f < nf; ++f) fidx[fnodes[f]] = f;
  std::vector<int> rp(n + 1, 0), cl;
  for (int I = 0; I < n; ++I) {
    if (L.cf[I] == 1) cl.push_back(cidx[I]);
    else {
      const int f = fidx[I];
      for (int u = 0; u < hcnt[f]; ++u) cl.push_back(hcol[(size_t)f * cap + u]);
    }
    rp[I + 1] = (int)cl.size();
  }
  AMG_TRY(L.P.alloc(n, nc, (int)cl.size(), B));
  L.P.h_rowptr = std::move(rp);
  L.P.h_col = std::move(cl);
  AMG_TRY(L.P.upload_pattern(s));
  DBuf<int> d_fidx;
  AMG_TRY(d_fidx.alloc(n));
  AMG_CU(cudaMemcpyAsync(d_fidx.p, fidx.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  if (B == 1)
    AMG_KCOUNT k_p_vals<1><<<nblk((long)n * cap, 256), 256, 0, s>>>(n, L.P.rowptr.p, d_fidx.p, cap, d_val.p, L.P.val.p);
  else
    AMG_KCOUNT k_p_vals<3><<<nblk((long)n * cap * 9, 256), 256, 0, s>>>(n, L.P.rowptr.p, d_fidx.p, cap, d_val.p,
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
  DBuf<double> Pk, R, C;
  DBuf<int> st;
  AMG_TRY(st.alloc(1));
  AMG_TRY(st.zero(s));
  AMG_TRY(h->Cinv.alloc((size_t)m * m));
  AMG_TRY(h->Cinv.zero(s));
  if (L.n > 0) {
    AMG_TRY(Pk.alloc(CB * CB));
    AMG_TRY(R.alloc((size_t)CB * m));
    AMG_TRY(C.alloc((size_t)m * CB));
    double *D = h->Cinv.p;
    if (L.A.b == 1) AMG_KCOUNT k_to_dense<1><<<L.n, 128, 0, s>>>(L.n, L.A.rowptr.p, L.A.col.p, L.A.val.p, D);
    else AMG_KCOUNT k_to_dense<3><<<L.n, 288, 0, s>>>(L.n, L.A.rowptr.p, L.A.col.p, L.A.val.p, D);
    const int nt = (m + CB - 1) / CB;
    for (int k0 = 0; k0 < m; k0 += CB) {
      const int nb = m - k0 < CB ? m - k0 : CB;
      AMG_KCOUNT k_gj_pivot<<<1, CB * CB, 0, s>>>(m, k0, nb, D, Pk.p, st.p);
      AMG_KCOUNT k_gj_panels<<<nblk((long)CB * m, 256), 256, 0, s>>>(m, k0, nb, D, Pk.p, R.p, C.p);
      AMG_KCOUNT k_gj_update<<<dim3(nt, nt), 256, 0, s>>>(m, k0, nb, D, Pk.p, R.p, C.p);
    }
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

void free_hierarchy(Handle *h) {
  h->lev.clear();
  h->nlev = 0;
  h->Cinv.release();
  h->nL = 0;
}

int build_hierarchy(Handle *h, const int *rowptr, const int *col, const double *vals, int mem, int ntv0,
                    const double *V0, int memV, bool keep_pattern) {
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
    std::vector<int> hrp(n + 1);
    if (mem == AMG_MEM_HOST) memcpy(hrp.data(), rowptr, (n + 1) * sizeof(int));
    else AMG_CU(cudaMemcpy(hrp.data(), rowptr, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    const int nnzb = hrp[n];
    AMG_TRY(L0->A.alloc(n, n, nnzb, h->b));
    L0->A.h_rowptr = std::move(hrp);
    L0->A.h_col.resize(nnzb);
    if (mem == AMG_MEM_HOST) memcpy(L0->A.h_col.data(), col, nnzb * sizeof(int));
    else AMG_CU(cudaMemcpy(L0->A.h_col.data(), col, nnzb * sizeof(int), cudaMemcpyDeviceToHost));
    for (int I = 0; I < n; ++I) {
      for (int k = L0->A.h_rowptr[I]; k < L0->A.h_rowptr[I + 1]; ++k) {
        const int J = L0->A.h_col[k];
        if (J < 0 || J >= n || (k > L0->A.h_rowptr[I] && L0->A.h_col[k - 1] >= J)) {
          set_error("K pattern: row %d has an invalid or unsorted column index %d", I, J);
          return AMG_ERR_ARG;
        }
      }
    }
    AMG_TRY(L0->A.upload_pattern(s));
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
    std::vector<unsigned char> strong(L.A.nnzb);
    if (L.A.nnzb)
      AMG_CU(cudaMemcpy(strong.data(), d_strong.p, L.A.nnzb, cudaMemcpyDeviceToHost));
    trace("SoC filter", k, t2);
    double tm = now_s();
    AMG_TRY(mis_gpu(L.A, d_strong.p, L.cf, s));
    trace("MIS", k, tm);
    int nc = 0;
    for (int I = 0; I < L.n; ++I) nc += (L.cf[I] == 1);
    double t3 = now_s();
    T_cs += t3 - t2;
    if (nc == 0 || (double)nc > p.max_coarse_ratio * (double)L.n) {
      L.G = DevBsr();
      L.GT = DevBsr();
      L.V.release();
      L.cf.clear();
      break;
    }
    AMG_TRY(build_P(h, L, strong, d_strong.p));
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
      std::vector<int> src((size_t)B * nc);
      int q = 0;
      for (int I = 0; I < L.n; ++I)
        if (L.cf[I] == 1) {
          for (int c = 0; c < B; ++c) src[(size_t)B * q + c] = B * I + c;
          ++q;
        }
      DBuf<int> dsrc;
      AMG_TRY(dsrc.alloc((size_t)B * nc));
      AMG_CU(cudaMemcpyAsync(dsrc.p, src.data(), (size_t)B * nc * sizeof(int), cudaMemcpyHostToDevice, s));
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
