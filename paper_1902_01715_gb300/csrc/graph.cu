// Integer pattern work of the set-up on the GPU: prefix sums, longest rows,
// transposes (G^T of Algorithm 3's factor, R = P^T of Algorithm 5's
// prolongation), patterns of sparse products with rows of any length (the
// Galerkin product P^T A P, Sec. 3.5, and the distance-d_p neighbourhoods of
// Algorithm 5's candidate sets) and row compaction by a predicate.  Every
// output is a function of its input alone: atomics only count entries or
// claim slots, whose contents are then put in a fixed order.
#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- prefix sums
// out[i] = sum over j < i of (in[j] + add), out[n] = the total.  One block of
// 1024 threads: each sums a contiguous chunk, the chunk sums are scanned in
// shared memory, then each thread writes its chunk.
__global__ void __launch_bounds__(1024) k_scan(int n, const int *__restrict__ in, int add, int *__restrict__ out) {
  pdl_wait();
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024;
  const int lo = (int)min((long)n, (long)threadIdx.x * per), hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += in[i] + add;
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
    acc += in[i] + add;
  }
  if (threadIdx.x == 1023) out[n] = part[1023];
}

int dev_scan(int n, const int *in, int add, int *out, cudaStream_t s) {
  launch_k(k_scan, 1, 1024, 0, s, n, in, add, out);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int read_int(const int *d, int *h, cudaStream_t s) {
  AMG_CU(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ---------------------------------------------------------------- longest row
__global__ void k_row_max(int n, const int *__restrict__ rp, int *__restrict__ out) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int v = i < n ? rp[i + 1] - rp[i] : 0;
  for (int off = 16; off; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(out, v);
}

int dev_row_max(int n, const int *rp, int *out, cudaStream_t s) {
  *out = 0;
  if (n <= 0) return AMG_OK;
  DBuf<int> d;
  AMG_TRY(d.alloc(1));
  AMG_TRY(d.zero(s));
  launch_k(k_row_max, nblk(n, 256), 256, 0, s, n, rp, d.p);
  AMG_LAUNCH_CHECK();
  return read_int(d.p, out, s);
}

int DevBsr::row_max(cudaStream_t s, int *out) const {
  if (maxlen < 0) AMG_TRY(dev_row_max(nr, rowptr.p, &maxlen, s));
  *out = maxlen;
  return AMG_OK;
}

// ---------------------------------------------------------------- transpose
// T = A^T: entries counted per column, column starts by a prefix sum; each
// entry claims a slot in its column (atomic counter), then moves to its rank
// among the rows of that column (the rows of a column are distinct), so the
// rows of T come out ascending whatever order the claims took.
__global__ void k_tr_count(int nnzb, const int *__restrict__ col, int *__restrict__ cnt) {
  pdl_wait();
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnzb) atomicAdd(&cnt[col[k]], 1);
}

// one warp per row of A
__global__ void k_tr_place(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                           const int *__restrict__ trp, int *__restrict__ fill, int *__restrict__ trow,
                           int *__restrict__ tsrc) {
  pdl_wait();
  const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (I >= nr) return;
  for (int k = rp[I] + lane; k < rp[I + 1]; k += 32) {
    const int c = col[k];
    const int at = trp[c] + atomicAdd(&fill[c], 1);
    trow[at] = I;
    tsrc[at] = k;
  }
}

// one warp per column of A (row of T)
__global__ void k_tr_rank(int nc, const int *__restrict__ trp, const int *__restrict__ trow,
                          const int *__restrict__ tsrc, int *__restrict__ tcol, int *__restrict__ perm) {
  pdl_wait();
  const int c = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (c >= nc) return;
  const int b = trp[c], e = trp[c + 1];
  for (int q = b + lane; q < e; q += 32) {
    const int r = trow[q];
    int rank = 0;
    for (int u = b; u < e; ++u) rank += trow[u] < r;
    tcol[b + rank] = r;
    perm[b + rank] = tsrc[q];
  }
}

// T.val[q] = transpose(A.val[perm[q]])
template <int B>
__global__ void k_transpose_vals(int nnzb, const int *__restrict__ perm, const double *__restrict__ src,
                                 double *__restrict__ dst) {
  pdl_wait();
  constexpr int BB = B * B;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)BB * nnzb) return;
  const int q = (int)(t / BB), e = (int)(t % BB), r = e / B, c = e % B;
  dst[(size_t)q * BB + c * B + r] = src[(size_t)perm[q] * BB + e];
}

int transpose_bsr(const DevBsr &A, DevBsr &T, cudaStream_t s) {
  const int nnzb = A.nnzb;
  AMG_TRY(T.alloc(A.nc, A.nr, nnzb, A.b));
  DBuf<int> cnt, fill, trow, tsrc, perm;
  AMG_TRY(cnt.alloc(A.nc));
  AMG_TRY(fill.alloc(A.nc));
  AMG_TRY(cnt.zero(s));
  AMG_TRY(fill.zero(s));
  if (nnzb) launch_k(k_tr_count, nblk(nnzb, 256), 256, 0, s, nnzb, A.col.p, cnt.p);
  AMG_LAUNCH_CHECK();
  AMG_TRY(dev_scan(A.nc, cnt.p, 0, T.rowptr.p, s));
  if (!nnzb) return AMG_OK;
  AMG_TRY(trow.alloc(nnzb));
  AMG_TRY(tsrc.alloc(nnzb));
  AMG_TRY(perm.alloc(nnzb));
  launch_k(k_tr_place, nblk(32L * A.nr, 256), 256, 0, s, A.nr, A.rowptr.p, A.col.p, T.rowptr.p, fill.p,
                                                              trow.p, tsrc.p);
  launch_k(k_tr_rank, nblk(32L * A.nc, 256), 256, 0, s, A.nc, T.rowptr.p, trow.p, tsrc.p, T.col.p, perm.p);
  if (A.b == 1)
    launch_k(k_transpose_vals<1>, nblk((long)nnzb, 256), 256, 0, s, nnzb, perm.p, A.val.p, T.val.p);
  else if (A.b == 3)
    launch_k(k_transpose_vals<3>, nblk(9L * nnzb, 256), 256, 0, s, nnzb, perm.p, A.val.p, T.val.p);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// ---------------------------------------------------------------- pattern products
// Row i of Z = X Y is the union of the (ascending) rows of Y named by row i
// of X.  Rows of X with at most 256 entries: one warp merges the lists (lane
// l holds the heads of lists l, l + 32, ...; each step takes the warp minimum,
// emits it once and advances every list whose head equals it), so the output
// is ascending and duplicate-free.  Pass 0 counts, pass 1 writes.
constexpr int SYM_PER = 8;  // lists per lane held in registers
constexpr int SYM_MAXL = 32 * SYM_PER;

__global__ void k_sym_merge(int nr, const int *__restrict__ xr, const int *__restrict__ xc,
                            const int *__restrict__ yr, const int *__restrict__ yc, const int *__restrict__ zr,
                            int *__restrict__ zc, int *__restrict__ cnt) {
  pdl_wait();
  const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nr) return;
  const int l0 = xr[i], nl = xr[i + 1] - l0;
  if (nl > SYM_MAXL) return;  // k_sym_long
  int pos[SYM_PER], end[SYM_PER];
  for (int u = 0; u < SYM_PER; ++u) {
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
    for (int u = 0; u < SYM_PER; ++u)
      if (pos[u] < end[u]) h = min(h, yc[pos[u]]);
    for (int off = 16; off >= 1; off >>= 1) h = min(h, __shfl_xor_sync(0xffffffffu, h, off));
    if (h == 0x7fffffff) break;
    if (lane == 0 && zc) zc[out + n] = h;
    ++n;
    for (int u = 0; u < SYM_PER; ++u)
      if (pos[u] < end[u] && yc[pos[u]] == h) ++pos[u];
  }
  if (lane == 0 && !zc) cnt[i] = n;
}

// Rows of X with more than 256 entries: a CTA takes such rows one at a time
// and marks the union in a bitmap over Z's columns (global scratch, one per
// CTA); the set bits are then counted, or written in ascending order (a
// prefix sum of the per-thread counts over contiguous word ranges).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_sym_long(int nr, int nc, const int *__restrict__ xr,
                                                  const int *__restrict__ xc, const int *__restrict__ yr,
                                                  const int *__restrict__ yc, const int *__restrict__ zr,
                                                  int *__restrict__ zc, int *__restrict__ cnt,
                                                  unsigned *__restrict__ bm_all) {
  pdl_wait();
  __shared__ int part[256];
  const int words = (nc + 31) >> 5;
  unsigned *bm = bm_all + (size_t)blockIdx.x * words;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (words + 255) / 256;
  const int w0 = min(words, (int)threadIdx.x * per), w1 = min(words, w0 + per);
  for (int i = blockIdx.x; i < nr; i += gridDim.x) {
    const int l0 = xr[i], nl = xr[i + 1] - l0;
    if (nl <= SYM_MAXL) continue;  // the same for the whole CTA
    for (int w = threadIdx.x; w < words; w += 256) bm[w] = 0u;
    __syncthreads();
    for (int q = warp; q < nl; q += 8) {
      const int k = xc[l0 + q];
      for (int e = yr[k] + lane; e < yr[k + 1]; e += 32) {
        const int c = yc[e];
        atomicOr(&bm[c >> 5], 1u << (c & 31));
      }
    }
    __syncthreads();
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
    part[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (!WRITE) {
      if (threadIdx.x == 255) cnt[i] = part[255];
    } else {
      int o = zr[i] + (threadIdx.x ? part[threadIdx.x - 1] : 0);
      for (int w = w0; w < w1; ++w) {
        unsigned b = bm[w];
        while (b) {
          zc[o++] = (w << 5) + __ffs(b) - 1;
          b &= b - 1u;
        }
      }
    }
    __syncthreads();  // the bitmap is cleared for the next row only after every thread read it
  }
}

// Z = pattern of X Y on the device (row pointer, columns, and values for
// b x b blocks when b > 0, left unset).
int symbolic_product(const DevBsr &X, const DevBsr &Y, DevBsr &Z, int b, cudaStream_t s) {
  const int nr = X.nr;
  int maxlen = 0;
  AMG_TRY(X.row_max(s, &maxlen));
  const bool longrows = maxlen > SYM_MAXL;
  int nlong = 0;
  DBuf<unsigned> bm;
  if (longrows) {
    int dev = 0, nsm = 0;
    AMG_CU(cudaGetDevice(&dev));
    AMG_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    nlong = std::min(nr, 2 * nsm);
    AMG_TRY(bm.alloc((size_t)nlong * ((Y.nc + 31) / 32)));
  }
  DBuf<int> cnt, rp;
  AMG_TRY(cnt.alloc(nr));
  AMG_TRY(rp.alloc(nr + 1));
  const int nb = nblk(32L * nr, 256);
  if (nr) launch_k(k_sym_merge, nb, 256, 0, s, nr, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, nullptr, nullptr,
                                                    cnt.p);
  if (longrows)
    launch_k(k_sym_long<false>, nlong, 256, 0, s, nr, Y.nc, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, nullptr,
                                                       nullptr, cnt.p, bm.p);
  AMG_TRY(dev_scan(nr, cnt.p, 0, rp.p, s));
  // entry count and longest row of Z in one read-back
  DBuf<int> tail;
  AMG_TRY(tail.alloc(2));
  AMG_TRY(tail.zero(s));
  AMG_CU(cudaMemcpyAsync(tail.p, rp.p + nr, sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (nr) launch_k(k_row_max, nblk(nr, 256), 256, 0, s, nr, rp.p, tail.p + 1);
  AMG_LAUNCH_CHECK();
  int ht[2] = {0, 0};
  AMG_CU(cudaMemcpyAsync(ht, tail.p, sizeof ht, cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  const int nnz = ht[0];
  AMG_TRY(Z.alloc(nr, Y.nc, nnz, b));
  Z.maxlen = ht[1];
  AMG_CU(cudaMemcpyAsync(Z.rowptr.p, rp.p, (nr + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (nr) launch_k(k_sym_merge, nb, 256, 0, s, nr, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, rp.p, Z.col.p,
                                                    nullptr);
  if (longrows)
    launch_k(k_sym_long<true>, nlong, 256, 0, s, nr, Y.nc, X.rowptr.p, X.col.p, Y.rowptr.p, Y.col.p, rp.p,
                                                      Z.col.p, nullptr, bm.p);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// ---------------------------------------------------------------- row compaction
// Entries of each row kept in order by a predicate; one warp per row (ballot
// compaction).  MODE 0: entries strong or on the diagonal (the strong graph
// with self loops); MODE 1: entries that are coarse nodes other than the
// row's own node self[i].  Pass 0 counts (cnt), pass 1 writes (orp, ocol).
template <int MODE>
__global__ void k_keep(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                       const unsigned char *__restrict__ strong, const int *__restrict__ cf,
                       const int *__restrict__ self, const int *__restrict__ orp, int *__restrict__ ocol,
                       int *__restrict__ cnt) {
  pdl_wait();
  const int i = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= nr) return;
  int n = 0;
  const int o = ocol ? orp[i] : 0;
  for (int b = rp[i]; b < rp[i + 1]; b += 32) {
    const int k = b + lane;
    bool keep = false;
    if (k < rp[i + 1]) {
      const int c = col[k];
      keep = MODE == 0 ? (strong[k] || c == i) : (cf[c] == 1 && c != self[i]);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep && ocol) ocol[o + n + __popc(bal & ((1u << lane) - 1u))] = col[k];
    n += __popc(bal);
  }
  if (lane == 0 && !ocol) cnt[i] = n;
}

template <int MODE>
static int keep_rows(int nr, int nc, const int *rp, const int *col, const unsigned char *strong, const int *cf,
                     const int *self, DevBsr &Z, cudaStream_t s) {
  DBuf<int> cnt;
  AMG_TRY(cnt.alloc(nr));
  DBuf<int> zr;
  AMG_TRY(zr.alloc(nr + 1));
  const int nb = nblk(32L * nr, 256);
  if (nr) launch_k(k_keep<MODE>, nb, 256, 0, s, nr, rp, col, strong, cf, self, nullptr, nullptr, cnt.p);
  AMG_TRY(dev_scan(nr, cnt.p, 0, zr.p, s));
  int nnz = 0;
  AMG_TRY(read_int(zr.p + nr, &nnz, s));
  AMG_TRY(Z.alloc(nr, nc, nnz, 0));
  AMG_CU(cudaMemcpyAsync(Z.rowptr.p, zr.p, (nr + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (nr) launch_k(k_keep<MODE>, nb, 256, 0, s, nr, rp, col, strong, cf, self, Z.rowptr.p, Z.col.p, nullptr);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// Candidate sets of Algorithm 5 for any distance and row length: the coarse
// nodes within d_p strong edges of fine node fnodes[f], ascending.  With S1
// the strong graph plus self loops and E the selection of the fine rows,
// the ball of radius d around each fine node is the pattern of E S1^d
// (d pattern products); the candidates are its coarse entries other than the
// node itself.
int dpls_candidates_gpu(const DevBsr &A, const unsigned char *strong, const int *cf, const int *fnodes, int nf,
                        int d_p, int *cptr, DBuf<int> &cand, cudaStream_t s) {
  const int n = A.nr;
  DevBsr S1, ball;
  AMG_TRY(keep_rows<0>(n, n, A.rowptr.p, A.col.p, strong, nullptr, nullptr, S1, s));
  // E: row f holds the column fnodes[f]
  AMG_TRY(ball.alloc(nf, n, nf, 0));
  {
    DBuf<int> ones;
    AMG_TRY(ones.alloc(nf));
    AMG_CU(cudaMemsetAsync(ones.p, 0, (size_t)nf * sizeof(int), s));
    AMG_TRY(dev_scan(nf, ones.p, 1, ball.rowptr.p, s));
    AMG_CU(cudaMemcpyAsync(ball.col.p, fnodes, (size_t)nf * sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  for (int d = 0; d < d_p; ++d) {
    DevBsr next;
    AMG_TRY(symbolic_product(ball, S1, next, 0, s));
    ball = std::move(next);
  }
  DevBsr C;
  AMG_TRY(keep_rows<1>(nf, n, ball.rowptr.p, ball.col.p, nullptr, cf, fnodes, C, s));
  AMG_CU(cudaMemcpyAsync(cptr, C.rowptr.p, (nf + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  cand = std::move(C.col);
  return AMG_OK;
}

}  // namespace amg
