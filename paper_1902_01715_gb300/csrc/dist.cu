// Kernels of the row-partitioned solve (paper_1902_01715_gb300/dist.py): each
// rank applies the level products to its own block rows, updates its own
// entries of the PCG vectors, forms partial inner products over them and
// moves halo entries between its vectors and the exchange buffers.  The
// hierarchy is the handle's (every rank builds the same one); products use
// the FP64 storage of the level matrices.
#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// Partial inner product over entries [n0, n1) in a fixed order: one block of
// 256 threads, thread j sums entries n0 + j, n0 + j + 256, ... in order, then
// the 256 partial sums are combined by a fixed binary tree.
__global__ void __launch_bounds__(256) k_range_dot(long n0, long n1, const double *__restrict__ x,
                                                   const double *__restrict__ y, double *__restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long i = n0 + threadIdx.x; i < n1; i += 256) s = fma(x[i], y[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// y = a x + b y on [n0, n1)
__global__ void k_range_axpby(long n0, long n1, double a, const double *__restrict__ x, double b,
                              double *__restrict__ y) {
  const long i = n0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) y[i] = fma(a, x[i], b * y[i]);
}

__global__ void k_gather(long m, const long long *__restrict__ idx, const double *__restrict__ x,
                         double *__restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = x[idx[i]];
}

__global__ void k_scatter(long m, const long long *__restrict__ idx, const double *__restrict__ in,
                          double *__restrict__ x) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) x[idx[i]] = in[i];
}

// z = Cinv y with the explicit inverse of the last level, one warp per row
__global__ void k_coarse_full(int m, const double *__restrict__ Ci, const double *__restrict__ y,
                              double *__restrict__ z) {
  const int row = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double s = 0.0;
  const double *Cr = Ci + (size_t)row * m;
  for (int k = lane; k < m; k += 32) s = fma(Cr[k], y[k], s);
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) z[row] = s;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_level_apply(amg_handle hh, int lev, int which, int ep, int row0, int row1, const double *x,
                               double *y, const double *aux, double w) {
  Handle *h = (Handle *)hh;
  if (!h || lev < 0 || lev >= h->nlev || which < 0 || which > 4 || ep < EP_SET || ep > EP_ACC || !x || !y ||
      ((ep == EP_RESID || ep == EP_SADD) && !aux)) {
    set_error("amg_level_apply: invalid argument");
    return AMG_ERR_ARG;
  }
  Level &L = *h->lev[lev];
  const SolveMat &M = which == 0 ? L.sA : which == 1 ? L.sG : which == 2 ? L.sGT : which == 3 ? L.sP : L.sR;
  if (M.nr == 0 || !M.v64.p) {
    set_error("amg_level_apply: level %d has no FP64 copy of matrix %d (FP64 V-cycle only, or level-0 A)", lev,
              which);
    return AMG_ERR_ARG;
  }
  if (row0 < 0 || row1 > M.nr || row0 > row1) {
    set_error("amg_level_apply: rows [%d, %d) outside [0, %d)", row0, row1, M.nr);
    return AMG_ERR_ARG;
  }
  bsrmv_rows(ep, M, x, y, aux, w, row0, row1, h->stream);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

extern "C" int amg_coarse_apply(amg_handle hh, const double *y, double *z) {
  Handle *h = (Handle *)hh;
  if (!h || !y || !z) return AMG_ERR_ARG;
  const int m = h->nL;
  if (m > 0) AMG_KCOUNT k_coarse_full<<<nblk(32L * m, 256), 256, 0, h->stream>>>(m, h->Cinv.p, y, z);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

extern "C" int amg_range_dot(long long n0, long long n1, const double *x, const double *y, double *out,
                             void *stream) {
  if (n0 < 0 || n1 < n0 || !x || !y || !out) return AMG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_range_dot<<<1, 256, 0, s>>>(n0, n1, x, y, out);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

extern "C" int amg_range_axpby(long long n0, long long n1, double a, const double *x, double b, double *y,
                               void *stream) {
  if (n0 < 0 || n1 < n0 || !x || !y) return AMG_ERR_ARG;
  if (n1 == n0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_range_axpby<<<nblk(n1 - n0, 256), 256, 0, s>>>(n0, n1, a, x, b, y);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

extern "C" int amg_gather(long long m, const long long *idx, const double *x, double *out, void *stream) {
  if (m < 0 || (m > 0 && (!idx || !x || !out))) return AMG_ERR_ARG;
  if (m == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_gather<<<nblk(m, 256), 256, 0, s>>>(m, idx, x, out);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

extern "C" int amg_scatter(long long m, const long long *idx, const double *in, double *x, void *stream) {
  if (m < 0 || (m > 0 && (!idx || !in || !x))) return AMG_ERR_ARG;
  if (m == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_scatter<<<nblk(m, 256), 256, 0, s>>>(m, idx, in, x);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}
