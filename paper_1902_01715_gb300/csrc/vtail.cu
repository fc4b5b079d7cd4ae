// The coarse end of the V(1,1)-cycle (Algorithm 2 below a start level, down to
// the dense coarse solve and back) as one persistent kernel.  On the coarse
// levels every product is a few microseconds of work, and as separate
// launches each one costs a launch, a ramp-up and a tail; here the products
// run one after another inside one cooperatively launched grid (one or two
// 16-warp CTAs per SM), separated by a grid barrier.
//
// The arithmetic of every row is the standalone product's (spmv.cu): the same
// sliced layout and permutation, the same warps per slice (the size rule's
// WPS, which fixes the summation order), the same partial-sum merge through
// shared memory; the coarse product is k_coarse_mv's.  So the fused V-cycle
// gives the same bits as the launch-per-product one.
//
// Every barrier wait is bounded (about two seconds of SM clock); a wait that
// runs out sets the error word (read after the solve like the bulk-copy
// product's) and the kernel returns.
#include <cstdlib>

#include "amg_internal.h"

namespace amg {

constexpr int VT_WARPS = 16;
constexpr int VT_THREADS = 32 * VT_WARPS;
constexpr int VT_MAXOPS = 128;

__device__ int g_vtail_err;

struct VtOp {
  int kind;  // 0 sparse product, 1 coarse product with the explicit inverse
  int ep, wps, nr, ns;
  const int *prow, *rp, *slp, *scol;
  const void *v;  // values (T)
  const void *x;
  void *y;
  const void *aux;
  double w;
  const double *Ci;  // kind 1
  int m;             // kind 1: order of the coarse level
};

struct VtProg {
  int nops;
  VtOp op[VT_MAXOPS];
};

// Grid barrier: arrival counter bar[0] and generation bar[1].  The last block
// to arrive resets the counter and bumps the generation; the others wait for
// the bump (bounded).  Returns false on a timeout (in every thread).
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned &gen, int *fail) {
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
        // another block gave up: leave at once instead of waiting out the limit
        if (*(volatile int *)&g_vtail_err || clock64() - t0 > (1LL << 32)) {
          atomicExch(&g_vtail_err, 1);
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

template <typename T, int B, int WPS>
__device__ __forceinline__ void vt_spmv(const VtOp &o, T (*red)[2 * B][32]) {
  constexpr int SPB = VT_WARPS / WPS, BB = B * B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = warp % WPS;
  // Vectors are written by earlier products of this kernel on other SMs:
  // they are read through L2 (__ldcg), never through the non-coherent L1 or
  // read-only paths; the matrices do not change while the kernel runs.
  const T *__restrict__ v = (const T *)o.v;
  const T *x = (const T *)o.x;
  const T *aux = (const T *)o.aux;
  T *y = (T *)o.y;
  const T w = (T)o.w;
  const int rounds = (o.ns + gridDim.x * SPB - 1) / (gridDim.x * SPB);
  for (int rd = 0; rd < rounds; ++rd) {
    const int sl = (rd * gridDim.x + blockIdx.x) * SPB + warp / WPS;
    const int pos = sl * 32 + lane;
    const int row = (sl < o.ns && pos < o.nr) ? (o.prow ? o.prow[pos] : pos) : -1;
    const bool valid = row >= 0;
    const int len = valid ? o.rp[row + 1] - o.rp[row] : 0;
    const long base = valid ? (long)o.slp[sl] : 0L;
    RowAcc<T> acc;
    for (int j0 = part; j0 < len; j0 += WPS * 2) {
      int c[2];
      T m[2][BB];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u * WPS;
        if (j < len) {
          const long slot = base + 32L * j;
          c[u] = o.scol[slot + lane];
          const T *vp = v + BB * slot + lane;
#pragma unroll
          for (int e = 0; e < BB; ++e) m[u][e] = vp[32 * e];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = j0 + u * WPS;
        if (j < len) {
          const T *xp = x + (long)B * c[u];
          if constexpr (B == 3) {
            const T x0 = __ldcg(xp), x1 = __ldcg(xp + 1), x2 = __ldcg(xp + 2);
#pragma unroll
            for (int r = 0; r < 3; ++r) acc.add(r, m[u][3 * r], m[u][3 * r + 1], m[u][3 * r + 2], x0, x1, x2);
          } else {
            acc.add1(0, m[u][0], __ldcg(xp));
          }
        }
      }
    }
    if (WPS > 1) {
#pragma unroll
      for (int r = 0; r < B; ++r) {
        red[warp][r][lane] = acc.hi(r);
        red[warp][B + r][lane] = acc.lo(r);
      }
      __syncthreads();
      if (part == 0) {
#pragma unroll
        for (int p = 1; p < WPS; ++p)
#pragma unroll
          for (int r = 0; r < B; ++r) acc.merge(r, red[warp + p][r][lane], red[warp + p][B + r][lane]);
      }
      __syncthreads();
    }
    if (valid && part == 0) {
      const long ob = (long)B * row;
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const T a = acc.get(r);
        if (o.ep == EP_SET) y[ob + r] = a;
        else if (o.ep == EP_SCALE) y[ob + r] = w * a;
        else if (o.ep == EP_RESID) y[ob + r] = __ldcg(aux + ob + r) - a;
        else if (o.ep == EP_SADD) y[ob + r] = __ldcg(aux + ob + r) + w * a;
        else y[ob + r] = __ldcg(y + ob + r) + a;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void vt_coarse(const VtOp &o) {
  const T *yv = (const T *)o.x;  // written by the restriction before: read through L2
  T *z = (T *)o.y;
  const int lane = threadIdx.x & 31;
  const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long row = gw; row < o.m; row += nw) {
    double s = 0.0;
    const double *Cr = o.Ci + (size_t)row * o.m;
    for (int k = lane; k < o.m; k += 32) s = fma(Cr[k], (double)__ldcg(yv + k), s);
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) z[row] = (T)s;
  }
}

template <typename T, int B>
__global__ void __launch_bounds__(VT_THREADS) k_vtail(const VtProg *__restrict__ prog, unsigned *bar,
                                                      const int *__restrict__ done) {
  if (done && *done) return;
  __shared__ T red[VT_WARPS][2 * B][32];
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  unsigned gen = ((volatile unsigned *)bar)[1];
  __syncthreads();
  const int nops = prog->nops;
  for (int i = 0; i < nops; ++i) {
    const VtOp &o = prog->op[i];
    if (o.kind == 1) vt_coarse<T>(o);
    else {
      switch (o.wps) {
        case 1: vt_spmv<T, B, 1>(o, red); break;
        case 2: vt_spmv<T, B, 2>(o, red); break;
        case 4: vt_spmv<T, B, 4>(o, red); break;
        case 8: vt_spmv<T, B, 8>(o, red); break;
        default: vt_spmv<T, B, 16>(o, red); break;
      }
    }
    if (i + 1 < nops && !grid_sync(bar, gen, &fail)) return;
  }
}

}  // namespace amg

namespace amg {

static int nsm_of_device() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

template <typename T, int B>
static void *vt_kernel() {
  return (void *)k_vtail<T, B>;
}

static void *vt_kernel_for(bool f64, int b) {
  if (f64) return b == 1 ? vt_kernel<double, 1>() : vt_kernel<double, 3>();
  return b == 1 ? vt_kernel<float, 1>() : vt_kernel<float, 3>();
}

// Level vectors and value arrays in the V-cycle's storage.
template <typename T> static T *vy(Level &L);
template <typename T> static T *vz(Level &L);
template <typename T> static T *vs(Level &L);
template <typename T> static T *vr(Level &L);
template <typename T> static T *vt(Level &L);
template <> double *vy<double>(Level &L) { return L.y64.p; }
template <> double *vz<double>(Level &L) { return L.z64.p; }
template <> double *vs<double>(Level &L) { return L.s64.p; }
template <> double *vr<double>(Level &L) { return L.r64.p; }
template <> double *vt<double>(Level &L) { return L.t64.p; }
template <> float *vy<float>(Level &L) { return L.y32.p; }
template <> float *vz<float>(Level &L) { return L.z32.p; }
template <> float *vs<float>(Level &L) { return L.s32.p; }
template <> float *vr<float>(Level &L) { return L.r32.p; }
template <> float *vt<float>(Level &L) { return L.t32.p; }
template <typename T> static const T *vals_of(const SolveMat &M);
template <> const double *vals_of<double>(const SolveMat &M) { return M.v64.p; }
template <> const float *vals_of<float>(const SolveMat &M) { return M.v32.p; }

template <typename T>
static void add_op(VtProg &P, const SolveMat &M, int ep, const void *x, void *y, const void *aux, double w, bool f64) {
  VtOp &o = P.op[P.nops++];
  o = VtOp{};
  o.kind = 0;
  o.ep = ep;
  o.wps = mapping_wps(M, f64);
  o.nr = M.nr;
  o.ns = M.ns;
  o.prow = M.prow.p;
  o.rp = M.rowptr;
  o.slp = M.slp.p;
  o.scol = M.scol.p;
  o.v = vals_of<T>(M);
  o.x = x;
  o.y = y;
  o.aux = aux;
  o.w = w;
}

// The program of the V-cycle below level `start` (Algorithm 2): per level the
// pre-smoothing, residual and restriction, the coarse product, then per level
// (coarse to fine) prolongation, residual and post-smoothing.
template <typename T>
static void build_prog(Handle *h, int start, VtProg &P, bool f64) {
  P.nops = 0;
  const int L = h->nlev - 1;
  for (int k = start; k < L; ++k) {
    Level &A = *h->lev[k], &C = *h->lev[k + 1];
    add_op<T>(P, A.sG, EP_SET, vy<T>(A), vt<T>(A), nullptr, 0.0, f64);
    add_op<T>(P, A.sGT, EP_SCALE, vt<T>(A), vs<T>(A), nullptr, A.omega, f64);
    add_op<T>(P, A.sA, EP_RESID, vs<T>(A), vr<T>(A), vy<T>(A), 0.0, f64);
    add_op<T>(P, A.sR, EP_SET, vr<T>(A), vy<T>(C), nullptr, 0.0, f64);
  }
  {
    VtOp &o = P.op[P.nops++];
    o = VtOp{};
    o.kind = 1;
    o.x = vy<T>(*h->lev[L]);
    o.y = vz<T>(*h->lev[L]);
    o.Ci = h->Cinv.p;
    o.m = h->nL;
  }
  for (int k = L - 1; k >= start; --k) {
    Level &A = *h->lev[k], &C = *h->lev[k + 1];
    add_op<T>(P, A.sP, EP_ACC, vz<T>(C), vs<T>(A), nullptr, 0.0, f64);
    add_op<T>(P, A.sA, EP_RESID, vs<T>(A), vr<T>(A), vy<T>(A), 0.0, f64);
    add_op<T>(P, A.sG, EP_SET, vr<T>(A), vt<T>(A), nullptr, 0.0, f64);
    add_op<T>(P, A.sGT, EP_SADD, vt<T>(A), vz<T>(A), vs<T>(A), A.omega, f64);
  }
}

static int vt_launch(Handle *h, const int *done, cudaStream_t s) {
  AMG_CU(cudaMemsetAsync(h->vt_bar.p, 0, 2 * sizeof(unsigned), s));
  const VtProg *prog = (const VtProg *)h->vt_prog.p;
  unsigned *bar = h->vt_bar.p;
  void *args[] = {(void *)&prog, (void *)&bar, (void *)&done};
  count_launches(1);
  AMG_CU(cudaLaunchCooperativeKernel(h->vt_func, dim3(h->vt_grid), dim3(VT_THREADS), args, 0, s));
  return AMG_OK;
}

// Decide whether (and from which level) the V-cycle's coarse end runs as one
// persistent kernel, and build its program.  Off unless AMG_VTAIL_LEVEL=<k>
// names the start level: measured on the 128x32x32 beam (fused from level 2,
// 17 products), the solve took 85.5 ms against 68.7 ms with one launch per
// product replayed from the CUDA graph -- the grid barriers cost more than the
// launches they replace.  FP64 and FP32 V-cycles (not bf16-stored G, P).  A
// trial capture checks that the cooperative launch can go into a CUDA graph
// on this system; otherwise the products stay separate launches.
int vtail_prepare(Handle *h) {
  h->vt_level = -1;
  const int prec = h->prm.vcycle_prec;
  const char *e = getenv("AMG_VTAIL_LEVEL");
  if (!e || prec == AMG_FP32_BF16GP || h->nlev < 3) return AMG_OK;
  const int start = atoi(e);
  if (start < 1 || start > h->nlev - 2) return AMG_OK;
  const bool f64 = prec == AMG_FP64;
  int coop = 0, dev = 0;
  AMG_CU(cudaGetDevice(&dev));
  AMG_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return AMG_OK;
  void *fn = vt_kernel_for(f64, h->b);
  int per = 0;
  AMG_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, VT_THREADS, 0));
  if (per < 1) return AMG_OK;
  per = per > 2 ? 2 : per;
  VtProg P;
  if (f64) build_prog<double>(h, start, P, true);
  else build_prog<float>(h, start, P, false);
  if (P.nops > VT_MAXOPS) return AMG_OK;
  cudaStream_t s = h->stream;
  AMG_TRY(h->vt_prog.alloc(sizeof(VtProg)));
  AMG_TRY(h->vt_bar.alloc(4));
  AMG_TRY(h->vt_flag.alloc(1));
  AMG_CU(cudaMemcpyAsync(h->vt_prog.p, &P, sizeof(VtProg), cudaMemcpyHostToDevice, s));
  const int one = 1;
  AMG_CU(cudaMemcpyAsync(h->vt_flag.p, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  AMG_CU(cudaStreamSynchronize(s));
  h->vt_func = fn;
  h->vt_grid = per * nsm_of_device();
  // trial: capture one launch (its done flag is set: it returns at once)
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const int rc = vt_launch(h, h->vt_flag.p, s);
    count_launches(-1);
    ok = cudaStreamEndCapture(s, &g) == cudaSuccess && rc == AMG_OK;
  }
  if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
  if (ok) ok = cudaGraphLaunch(ge, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!ok) return AMG_OK;
  h->vt_level = start;
  if (getenv("AMG_TRACE"))
    fprintf(stderr, "[amg] fused V-cycle from level %d: %d products, grid %d x %d threads\n", start, P.nops,
            h->vt_grid, VT_THREADS);
  return AMG_OK;
}

int vtail_run(Handle *h, const int *done, cudaStream_t s) { return vt_launch(h, done, s); }

int vtail_error() {
  int e = 0;
  AMG_CU(cudaMemcpyFromSymbol(&e, g_vtail_err, sizeof(int)));
  if (e) {
    const int z = 0;
    cudaMemcpyToSymbol(g_vtail_err, &z, sizeof(int));
    set_error("a grid barrier of the fused V-cycle kernel did not complete in time");
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

}  // namespace amg
