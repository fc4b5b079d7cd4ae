// Solve-phase sparse products y = epilogue(A x) over 3x3-block matrices
// (the level matrices A_k, the smoother factors G_k and G_k^T, P_k and
// R_k = P_k^T of the V-cycle, Algorithm 2), in a sliced layout built for
// coalesced streaming from HBM.
//
// Layout ("SELL-32" over block rows).  Block rows are grouped in slices of 32
// consecutive rows.  Slice s owns the slot range [slp[s], slp[s+1]), whose
// length is 32 x (longest row of the slice).  Slot slp[s] + 32 j + l holds
// block j of row 32 s + l: its column in scol[slot] and its 9 entries
// (row-major within the block) at v[9 (slp[s] + 32 j) + 32 e + l], e = 0..8.
// So the 32 lanes of a warp, one block row each, read every entry of their
// j-th blocks with one fully used 32-element load per entry, and a slice is
// one contiguous run of memory.  Padding slots (rows shorter than the
// slice's longest) are never read: each lane stops at its own row length.
// Rows are placed in the slices in order of decreasing length inside windows
// of SIGMA consecutive rows (ties keep row order; prow[position] = row), so
// the rows of a slice have nearly equal lengths and the lanes of a warp
// finish together (FP64 instructions cost the same with idle lanes); the
// window keeps the rows a warp reads and writes close together.  A row is
// still summed by the same lanes in the same order, whatever its position.
//
// Mapping.  WPS warps share one slice (warp p of the slice takes blocks
// j = p, p + WPS, ...) and their partial sums are added in warp order through
// shared memory, so small coarse levels with long rows still spread over the
// SMs; a CTA holds 4 warps (WPS <= 4) or one slice's WPS warps (8, 16).  In FP64 every product is one fused
// multiply-add into the row's accumulator (9 per block): FP64 arithmetic is
// the scarce resource of this GPU (about 0.63e12 FP64 FMA/s against
// 6.7 TB/s of HBM, i.e. 10.6 bytes per FMA, while an FP64 block brings 8.4
// bytes per FMA), so the FP64 product is bounded by the FP64 pipe and must
// spend nothing else there; FP32 and bf16 storage are HBM-bound.  Each
// warp issues the loads of U blocks before it uses any of them.  (WPS, U)
// is picked per matrix by timing the candidates on the matrix itself.
#include <mutex>
#include <type_traits>
#include <vector>

#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ double cvs(double v, double) { return v; }
__device__ __forceinline__ float cvs(float v, float) { return v; }
__device__ __forceinline__ float cvs(__nv_bfloat16 v, float) { return __bfloat162float(v); }

struct Mapping {
  int wps, u;
  bool w1;  // one warp per CTA (k_sellmv_w)
};
// entry 8 is the bulk-copy variant below (FP32 and bf16 storage); 9.. put
// every warp in a CTA of its own (14.. with four blocks in flight per lane)
constexpr int SELL_SIGMA = 1024;  // rows per sorting window (a multiple of 32)
static const Mapping kMaps[] = {{1, 2, false}, {1, 4, false}, {2, 2, false}, {2, 4, false}, {4, 2, false},
                                {4, 4, false}, {8, 2, false}, {16, 2, false}, {0, 0, false}, {1, 2, true},
                                {2, 2, true},  {4, 2, true},  {8, 2, true},  {16, 2, true}, {1, 4, true},
                                {2, 4, true},  {4, 4, true}};
constexpr int kNumMaps = (int)(sizeof(kMaps) / sizeof(kMaps[0]));

// CTA size: 4 warps, or one slice of WPS warps when WPS > 4
template <int WPS> struct SellCta {
  static constexpr int warps = WPS > 4 ? WPS : 4;
  static constexpr int threads = 32 * warps;
  static constexpr int slices = warps / WPS;
};

// the column indices and entries of blocks j0, j0 + WPS, ..., j0 + (U-1) WPS
// of a lane's row (those below the row length len)
template <typename TM, int BB, int WPS, int U>
__device__ __forceinline__ void sell_load(int j0, int len, long base, int lane, const int *__restrict__ scol,
                                          const TM *__restrict__ v, int (&c)[U], TM (&m)[U][BB]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int j = j0 + u * WPS;
    if (j < len) {
      const long slot = base + 32L * j;
      c[u] = scol[slot + lane];
      const TM *vp = v + BB * slot + lane;
#pragma unroll
      for (int e = 0; e < BB; ++e) m[u][e] = vp[32 * e];
    }
  }
}

template <typename TM, typename TX, int B, int EP, int WPS, int U>
__global__ void __launch_bounds__(SellCta<WPS>::threads) k_sellmv(int s0, int r0, int r1, int nr,
                                                                  const int *__restrict__ prow,
                                                                  const int *__restrict__ rp,
                                                                  const int *__restrict__ slp,
                                                                  const int *__restrict__ scol,
                                                                  const TM *__restrict__ v,
                                                                  const TX *__restrict__ x, TX *__restrict__ y,
                                                                  const TX *__restrict__ aux, TX w,
                                                                  const int *__restrict__ done) {
  constexpr int SPB = SellCta<WPS>::slices, BB = B * B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sl = s0 + blockIdx.x * SPB + warp / WPS;
  const int part = warp % WPS;
  const int pos = sl * 32 + lane;
  const int row = pos < nr ? (prow ? prow[pos] : pos) : -1;
  const bool valid = row >= r0 && row < r1;  // rows [r0, r1) only
  const int len = valid ? rp[row + 1] - rp[row] : 0;
  const long base = valid ? (long)slp[sl] : 0L;
  // the row data and the first U blocks (solve layout) are loaded before
  // the wait for the preceding kernel; x, the flag and y after it
  int c[U];
  TM m[U][BB];
  sell_load<TM, BB, WPS, U>(part, len, base, lane, scol, v, c, m);
  pdl_wait();
  if (done && *done) return;  // the same for the whole grid
  RowAcc<TX> acc;
  for (int j0 = part; j0 < len; j0 += WPS * U) {
    if (j0 != part) sell_load<TM, BB, WPS, U>(j0, len, base, lane, scol, v, c, m);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * WPS;
      if (j < len) {
        const TX *xp = x + (long)B * c[u];
        if constexpr (B == 3) {
          const TX x0 = xp[0], x1 = xp[1], x2 = xp[2];
#pragma unroll
          for (int r = 0; r < 3; ++r)
            acc.add(r, cvs(m[u][3 * r], TX(0)), cvs(m[u][3 * r + 1], TX(0)), cvs(m[u][3 * r + 2], TX(0)), x0, x1,
                    x2);
        } else {
          acc.add1(0, cvs(m[u][0], TX(0)), xp[0]);
        }
      }
    }
  }
  pdl_trigger();
  if (WPS > 1) {
    __shared__ TX red[SellCta<WPS>::warps][2 * B][32];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      red[warp][r][lane] = acc.hi(r);
      red[warp][B + r][lane] = acc.lo(r);
    }
    __syncthreads();
    if (part != 0) return;
#pragma unroll
    for (int p = 1; p < WPS; ++p)
#pragma unroll
      for (int r = 0; r < B; ++r) acc.merge(r, red[warp + p][r][lane], red[warp + p][B + r][lane]);
  }
  if (!valid) return;
  const long o = (long)B * row;
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const TX a = acc.get(r);
    if (EP == EP_SET) y[o + r] = a;
    if (EP == EP_SCALE) y[o + r] = w * a;
    if (EP == EP_RESID) y[o + r] = aux[o + r] - a;
    if (EP == EP_SADD) y[o + r] = aux[o + r] + w * a;
    if (EP == EP_ACC) y[o + r] += a;
  }
}

// The same product with one warp per CTA, for matrices whose slices are too
// few to give every SM a CTA of the kernel above: the CTAs then spread over
// all SMs (a small level's FP64 product is bounded by the FP64 pipes of the
// SMs it reaches).  The WPS warps of a slice are CTAs of their own; each
// stores its partial row sums, and the last to arrive (an arrival counter
// per slice) rebuilds the partial of warp 0 and adds those of warps 1,
// 2, ... in order -- the additions, in the order, of the shared-memory merge
// above, so both kernels give the same bits -- then writes the rows and
// clears the counter for the next launch.
template <typename TM, typename TX, int B, int EP, int WPS, int U>
__global__ void __launch_bounds__(32) k_sellmv_w(int s0, int r0, int r1, int nr, const int *__restrict__ prow,
                                                 const int *__restrict__ rp, const int *__restrict__ slp,
                                                 const int *__restrict__ scol, const TM *__restrict__ v,
                                                 const TX *__restrict__ x, TX *__restrict__ y,
                                                 const TX *__restrict__ aux, TX w, const int *__restrict__ done,
                                                 TX *__restrict__ wpart, unsigned *__restrict__ wtick) {
  constexpr int BB = B * B;
  const int lane = threadIdx.x;
  const int sl = s0 + (int)(blockIdx.x / WPS);
  const int part = (int)(blockIdx.x % WPS);
  const int pos = sl * 32 + lane;
  const int row = pos < nr ? (prow ? prow[pos] : pos) : -1;
  const bool valid = row >= r0 && row < r1;
  const int len = valid ? rp[row + 1] - rp[row] : 0;
  const long base = valid ? (long)slp[sl] : 0L;
  int c[U];
  TM m[U][BB];
  sell_load<TM, BB, WPS, U>(part, len, base, lane, scol, v, c, m);  // before the wait, as above
  pdl_wait();
  if (done && *done) return;
  RowAcc<TX> acc;
  for (int j0 = part; j0 < len; j0 += WPS * U) {
    if (j0 != part) sell_load<TM, BB, WPS, U>(j0, len, base, lane, scol, v, c, m);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * WPS;
      if (j < len) {
        const TX *xp = x + (long)B * c[u];
        if constexpr (B == 3) {
          const TX x0 = xp[0], x1 = xp[1], x2 = xp[2];
#pragma unroll
          for (int r = 0; r < 3; ++r)
            acc.add(r, cvs(m[u][3 * r], TX(0)), cvs(m[u][3 * r + 1], TX(0)), cvs(m[u][3 * r + 2], TX(0)), x0, x1,
                    x2);
        } else {
          acc.add1(0, cvs(m[u][0], TX(0)), xp[0]);
        }
      }
    }
  }
  pdl_trigger();
  if (WPS > 1) {
    TX *mine = wpart + ((size_t)sl * WPS + part) * (2 * B * 32);
#pragma unroll
    for (int r = 0; r < B; ++r) {
      mine[r * 32 + lane] = acc.hi(r);
      mine[(B + r) * 32 + lane] = acc.lo(r);
    }
    __threadfence();
    __syncwarp();
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(&wtick[sl], 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t != (unsigned)(WPS - 1)) return;
    __threadfence();
    const TX *sp = wpart + (size_t)sl * WPS * (2 * B * 32);
#pragma unroll
    for (int r = 0; r < B; ++r) acc.set(r, __ldcg(sp + r * 32 + lane), __ldcg(sp + (B + r) * 32 + lane));
#pragma unroll
    for (int p = 1; p < WPS; ++p) {
      const TX *pp = sp + (size_t)p * (2 * B * 32);
#pragma unroll
      for (int r = 0; r < B; ++r) acc.merge(r, __ldcg(pp + r * 32 + lane), __ldcg(pp + (B + r) * 32 + lane));
    }
    if (lane == 0) wtick[sl] = 0u;
  }
  if (!valid) return;
  const long o = (long)B * row;
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const TX a = acc.get(r);
    if (EP == EP_SET) y[o + r] = a;
    if (EP == EP_SCALE) y[o + r] = w * a;
    if (EP == EP_RESID) y[o + r] = aux[o + r] - a;
    if (EP == EP_SADD) y[o + r] = aux[o + r] + w * a;
    if (EP == EP_ACC) y[o + r] += a;
  }
}

// positions holding rows [r0, r1): the same range without a permutation, else
// the SIGMA windows that contain them
static void row_slices(const SolveMat &M, int r0, int r1, int &s0, int &s1) {
  int p0 = r0, p1 = r1;
  if (M.prow.p) {
    p0 = (r0 / SELL_SIGMA) * SELL_SIGMA;
    p1 = std::min(M.nr, ((r1 + SELL_SIGMA - 1) / SELL_SIGMA) * SELL_SIGMA);
  }
  s0 = p0 >> 5;
  s1 = ((p1 - 1) >> 5) + 1;
}

template <typename TM, typename TX, int B, int WPS, int U>
static void launch_map(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w,
                       const int *done, cudaStream_t s, int r0 = 0, int r1 = -1) {
  if (r1 < 0) r1 = M.nr;
  if (r1 <= r0) return;
  int s0, s1;
  row_slices(M, r0, r1, s0, s1);
  const int nb = nblk(s1 - s0, SellCta<WPS>::slices);
  constexpr int T = SellCta<WPS>::threads;
  if (nb == 0) return;
#define AMG_SELL_ARGS s0, r0, r1, M.nr, M.prow.p, M.rowptr, M.slp.p, M.scol.p, v, x, y, aux, w, done
  switch (ep) {
    case EP_SET: launch_k(k_sellmv<TM, TX, B, EP_SET, WPS, U>, nb, T, 0, s, AMG_SELL_ARGS); break;
    case EP_SCALE: launch_k(k_sellmv<TM, TX, B, EP_SCALE, WPS, U>, nb, T, 0, s, AMG_SELL_ARGS); break;
    case EP_RESID: launch_k(k_sellmv<TM, TX, B, EP_RESID, WPS, U>, nb, T, 0, s, AMG_SELL_ARGS); break;
    case EP_SADD: launch_k(k_sellmv<TM, TX, B, EP_SADD, WPS, U>, nb, T, 0, s, AMG_SELL_ARGS); break;
    default: launch_k(k_sellmv<TM, TX, B, EP_ACC, WPS, U>, nb, T, 0, s, AMG_SELL_ARGS); break;
  }
#undef AMG_SELL_ARGS
}

template <typename TM, typename TX, int B, int WPS, int U = 2>
static void launch_w(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w,
                     const int *done, cudaStream_t s, int r0 = 0, int r1 = -1) {
  if (r1 < 0) r1 = M.nr;
  if (r1 <= r0) return;
  int s0, s1;
  row_slices(M, r0, r1, s0, s1);
  const long nb = (long)(s1 - s0) * WPS;
  if (nb == 0) return;
  TX *wp = reinterpret_cast<TX *>(M.wpart.p);
  unsigned *wt = M.wtick.p;
#define AMG_SELL_ARGS s0, r0, r1, M.nr, M.prow.p, M.rowptr, M.slp.p, M.scol.p, v, x, y, aux, w, done, wp, wt
  switch (ep) {
    case EP_SET: launch_k(k_sellmv_w<TM, TX, B, EP_SET, WPS, U>, (unsigned)nb, 32, 0, s, AMG_SELL_ARGS); break;
    case EP_SCALE: launch_k(k_sellmv_w<TM, TX, B, EP_SCALE, WPS, U>, (unsigned)nb, 32, 0, s, AMG_SELL_ARGS); break;
    case EP_RESID: launch_k(k_sellmv_w<TM, TX, B, EP_RESID, WPS, U>, (unsigned)nb, 32, 0, s, AMG_SELL_ARGS); break;
    case EP_SADD: launch_k(k_sellmv_w<TM, TX, B, EP_SADD, WPS, U>, (unsigned)nb, 32, 0, s, AMG_SELL_ARGS); break;
    default: launch_k(k_sellmv_w<TM, TX, B, EP_ACC, WPS, U>, (unsigned)nb, 32, 0, s, AMG_SELL_ARGS); break;
  }
#undef AMG_SELL_ARGS
}

// ---------------------------------------------------------------- bulk-copy variant
// For FP32 and bf16 storage (HBM-bound): each warp runs its own pipeline of
// BK_ST shared-memory stages; lane 0 fills a stage with one chunk of a slice
// (the values and column indices of BK_JC consecutive block columns, which
// are contiguous in the slice layout) by two asynchronous bulk copies
// completing on the stage's mbarrier, while the lanes compute on the stages
// filled before.  Loads of the matrix then cost two instructions per chunk
// and the bytes in flight no longer depend on registers.  Every wait is
// bounded: a stage that does not complete within the limit sets the error
// word and ends the warp's work.
constexpr int BK_JC = 4;   // block columns per chunk
constexpr int BK_ST = 2;   // stages per warp
constexpr int BK_WARPS = 4;
__device__ int g_bulk_err;
// Test knob: when set, the first warp that reads it skips filling one stage
// (once), so its wait runs out and the timeout path is exercised without any
// fault.  Set from the environment (AMG_BULK_STALL_ONCE) at the first launch.
__device__ int g_bulk_stall;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait: gives up after about two seconds of SM clock
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > (1LL << 32)) return false;
  return true;
}

template <typename TM>
struct BulkStage {
  TM v[9 * 32 * BK_JC];
  int c[32 * BK_JC];
};

template <typename TM, typename TX, int EP>
__global__ void __launch_bounds__(32 * BK_WARPS) k_sellmv_bulk(int nr, int ns, const int *__restrict__ prow,
                                                               const int *__restrict__ rp,
                                                               const int *__restrict__ slp,
                                                               const int *__restrict__ scol,
                                                               const TM *__restrict__ v, const TX *__restrict__ x,
                                                               TX *__restrict__ y, const TX *__restrict__ aux, TX w,
                                                               const int *__restrict__ done) {
  pdl_wait();
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char bk_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BulkStage<TM> *st = reinterpret_cast<BulkStage<TM> *>(bk_smem) + warp * BK_ST;
  __shared__ __align__(8) unsigned long long bars[BK_WARPS][BK_ST];
  const int gw = blockIdx.x * BK_WARPS + warp, nw = gridDim.x * BK_WARPS;
  if (lane == 0) {
    for (int q = 0; q < BK_ST; ++q) mbar_init(smem_u32(&bars[warp][q]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // chunk stream of this warp: slices gw, gw + nw, ...; chunk c of a slice
  // covers block columns [c BK_JC, (c+1) BK_JC)
  int ps = gw, pc = 0;      // next chunk to fill (producer)
  unsigned pending = 0;     // lane 0: stages with copies in flight
  auto fill = [&](int q) {  // lane 0: start the next chunk into stage q
    while (ps < ns) {
      const int len = (slp[ps + 1] - slp[ps]) >> 5;
      if (pc * BK_JC < len) break;
      ps += nw;
      pc = 0;
    }
    if (ps >= ns) return;
    const int len = (slp[ps + 1] - slp[ps]) >> 5;
    const int nb = min(BK_JC, len - pc * BK_JC);
    const long slot = (long)slp[ps] + 32L * BK_JC * pc;
    const unsigned vb = (unsigned)(9 * 32 * nb * sizeof(TM)), cb = (unsigned)(32 * nb * sizeof(int));
    const unsigned bar = smem_u32(&bars[warp][q]);
    ++pc;
    if (g_bulk_stall && atomicExch(&g_bulk_stall, 0)) return;  // test knob: leave this stage empty
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(bar, vb + cb);
    bulk_g2s(smem_u32(st[q].v), v + 9 * slot, vb, bar);
    bulk_g2s(smem_u32(st[q].c), scol + slot, cb, bar);
    pending |= 1u << q;
  };
  if (lane == 0)
    for (int q = 0; q < BK_ST; ++q) fill(q);
  __syncwarp();
  unsigned phase[BK_ST];
  for (int q = 0; q < BK_ST; ++q) phase[q] = 0;
  int q = 0;
  bool failed = false;
  for (int sl = gw; sl < ns && !failed; sl += nw) {
    const int len_s = (slp[sl + 1] - slp[sl]) >> 5;
    const int pos = sl * 32 + lane;
    const int row = pos < nr ? (prow ? prow[pos] : pos) : nr;
    const int len = row < nr ? rp[row + 1] - rp[row] : 0;
    RowAcc<TX> acc;
    for (int c = 0; c * BK_JC < len_s; ++c) {
      const bool got = mbar_wait(smem_u32(&bars[warp][q]), phase[q]);
      if (!__all_sync(0xffffffffu, got)) {  // the warp leaves together
        if (lane == 0) atomicExch(&g_bulk_err, 1);
        failed = true;
        break;
      }
      phase[q] ^= 1u;
      pending &= ~(1u << q);
      // the chunk's neighbour values are gathered before any is used
      TX xv[BK_JC][3];
#pragma unroll
      for (int jj = 0; jj < BK_JC; ++jj)
        if (c * BK_JC + jj < len) {
          const TX *xp = x + 3L * st[q].c[jj * 32 + lane];
          xv[jj][0] = xp[0];
          xv[jj][1] = xp[1];
          xv[jj][2] = xp[2];
        }
#pragma unroll
      for (int jj = 0; jj < BK_JC; ++jj)
        if (c * BK_JC + jj < len) {
          const TM *m = st[q].v + jj * 9 * 32 + lane;
#pragma unroll
          for (int r = 0; r < 3; ++r)
            acc.add(r, cvs(m[32 * (3 * r)], TX(0)), cvs(m[32 * (3 * r + 1)], TX(0)), cvs(m[32 * (3 * r + 2)], TX(0)),
                    xv[jj][0], xv[jj][1], xv[jj][2]);
        }
      __syncwarp();
      if (lane == 0) fill(q);
      __syncwarp();
      q = q + 1 == BK_ST ? 0 : q + 1;
    }
    if (failed || row >= nr) continue;
    const TX a0 = acc.get(0), a1 = acc.get(1), a2 = acc.get(2);
    const long o = 3L * row;
    if (EP == EP_SET) { y[o] = a0; y[o + 1] = a1; y[o + 2] = a2; }
    if (EP == EP_SCALE) { y[o] = w * a0; y[o + 1] = w * a1; y[o + 2] = w * a2; }
    if (EP == EP_RESID) { y[o] = aux[o] - a0; y[o + 1] = aux[o + 1] - a1; y[o + 2] = aux[o + 2] - a2; }
    if (EP == EP_SADD) { y[o] = aux[o] + w * a0; y[o + 1] = aux[o + 1] + w * a1; y[o + 2] = aux[o + 2] + w * a2; }
    if (EP == EP_ACC) { y[o] += a0; y[o + 1] += a1; y[o + 2] += a2; }
  }
  pdl_trigger();
  if (failed && lane == 0)  // let the copies still in flight land (bounded) before the warp leaves
    for (int k = 0; k < BK_ST; ++k)
      if (pending & (1u << k)) mbar_wait(smem_u32(&bars[warp][k]), phase[k]);
}

template <typename TM, typename TX>
static void launch_bulk(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w,
                        const int *done, cudaStream_t s) {
  static int nsm = 0;
  static bool attr = false;
  const size_t shm = sizeof(BulkStage<TM>) * BK_ST * BK_WARPS;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  if (!attr) {
    if (getenv("AMG_BULK_STALL_ONCE")) {
      const int one = 1;
      cudaMemcpyToSymbol(g_bulk_stall, &one, sizeof(int));
    }
    cudaFuncSetAttribute(k_sellmv_bulk<TM, TX, EP_SET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_sellmv_bulk<TM, TX, EP_SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_sellmv_bulk<TM, TX, EP_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_sellmv_bulk<TM, TX, EP_SADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_sellmv_bulk<TM, TX, EP_ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    attr = true;
  }
  int nb = (M.ns + BK_WARPS - 1) / BK_WARPS;
  const int cap = nsm * 5;  // five CTAs per SM
  if (nb > cap) nb = cap;
  if (nb == 0) return;
#define AMG_BULK_ARGS M.nr, M.ns, M.prow.p, M.rowptr, M.slp.p, M.scol.p, v, x, y, aux, w, done
  switch (ep) {
    case EP_SET: launch_k(k_sellmv_bulk<TM, TX, EP_SET>, nb, 32 * BK_WARPS, shm, s, AMG_BULK_ARGS); break;
    case EP_SCALE: launch_k(k_sellmv_bulk<TM, TX, EP_SCALE>, nb, 32 * BK_WARPS, shm, s, AMG_BULK_ARGS); break;
    case EP_RESID: launch_k(k_sellmv_bulk<TM, TX, EP_RESID>, nb, 32 * BK_WARPS, shm, s, AMG_BULK_ARGS); break;
    case EP_SADD: launch_k(k_sellmv_bulk<TM, TX, EP_SADD>, nb, 32 * BK_WARPS, shm, s, AMG_BULK_ARGS); break;
    default: launch_k(k_sellmv_bulk<TM, TX, EP_ACC>, nb, 32 * BK_WARPS, shm, s, AMG_BULK_ARGS); break;
  }
#undef AMG_BULK_ARGS
}

int bulk_copy_error() {
  int e = 0;
  AMG_CU(cudaMemcpyFromSymbol(&e, g_bulk_err, sizeof(int)));
  if (e) {
    const int z = 0;
    cudaMemcpyToSymbol(g_bulk_err, &z, sizeof(int));
    set_error("a bulk-copy stage of the sparse product did not complete in time");
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

template <typename TM, typename TX, int B>
static void bsrmv_b(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w, const int *done,
                    cudaStream_t s) {
  switch (std::is_same<TM, double>::value ? M.map64 : M.map) {
    case 0: launch_map<TM, TX, B, 1, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 1: launch_map<TM, TX, B, 1, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 2: launch_map<TM, TX, B, 2, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 3: launch_map<TM, TX, B, 2, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 4: launch_map<TM, TX, B, 4, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 5: launch_map<TM, TX, B, 4, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 6: launch_map<TM, TX, B, 8, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 7: launch_map<TM, TX, B, 16, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 9: launch_w<TM, TX, B, 1>(ep, M, v, x, y, aux, w, done, s); break;
    case 10: launch_w<TM, TX, B, 2>(ep, M, v, x, y, aux, w, done, s); break;
    case 11: launch_w<TM, TX, B, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 12: launch_w<TM, TX, B, 8>(ep, M, v, x, y, aux, w, done, s); break;
    case 13: launch_w<TM, TX, B, 16>(ep, M, v, x, y, aux, w, done, s); break;
    case 14: launch_w<TM, TX, B, 1, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 15: launch_w<TM, TX, B, 2, 4>(ep, M, v, x, y, aux, w, done, s); break;
    case 16: launch_w<TM, TX, B, 4, 4>(ep, M, v, x, y, aux, w, done, s); break;
    default:
      // the bulk-copy variant is written for 3x3 blocks in FP32/bf16
      if constexpr (std::is_same<TM, double>::value || B != 3) launch_map<TM, TX, B, 1, 2>(ep, M, v, x, y, aux, w, done, s);
      else launch_bulk<TM, TX>(ep, M, v, x, y, aux, w, done, s);
      break;
  }
}

template <typename TM, typename TX>
void bsrmv(int ep, const SolveMat &M, const TM *v, const TX *x, TX *y, const TX *aux, TX w, const int *done,
           cudaStream_t s) {
  if (M.b == 1) bsrmv_b<TM, TX, 1>(ep, M, v, x, y, aux, w, done, s);
  else bsrmv_b<TM, TX, 3>(ep, M, v, x, y, aux, w, done, s);
}

// rows [r0, r1) only, FP64 storage (the row-partitioned solve)
template <int B>
static void bsrmv_rows_b(int ep, const SolveMat &M, const double *x, double *y, const double *aux, double w, int r0,
                         int r1, cudaStream_t s) {
  const double *v = M.v64.p;
  switch (M.map64) {
    case 0: launch_map<double, double, B, 1, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 1: launch_map<double, double, B, 1, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 2: launch_map<double, double, B, 2, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 3: launch_map<double, double, B, 2, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 4: launch_map<double, double, B, 4, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 5: launch_map<double, double, B, 4, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 6: launch_map<double, double, B, 8, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 7: launch_map<double, double, B, 16, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 9: launch_w<double, double, B, 1>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 10: launch_w<double, double, B, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 11: launch_w<double, double, B, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 12: launch_w<double, double, B, 8>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 13: launch_w<double, double, B, 16>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 14: launch_w<double, double, B, 1, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 15: launch_w<double, double, B, 2, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    case 16: launch_w<double, double, B, 4, 4>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
    default: launch_map<double, double, B, 1, 2>(ep, M, v, x, y, aux, w, nullptr, s, r0, r1); break;
  }
}

void bsrmv_rows(int ep, const SolveMat &M, const double *x, double *y, const double *aux, double w, int r0, int r1,
                cudaStream_t s) {
  if (M.b == 1) bsrmv_rows_b<1>(ep, M, x, y, aux, w, r0, r1, s);
  else bsrmv_rows_b<3>(ep, M, x, y, aux, w, r0, r1, s);
}

template void bsrmv<double, double>(int, const SolveMat &, const double *, const double *, double *, const double *,
                                    double, const int *, cudaStream_t);
template void bsrmv<float, float>(int, const SolveMat &, const float *, const float *, float *, const float *, float,
                                  const int *, cudaStream_t);
template void bsrmv<__nv_bfloat16, float>(int, const SolveMat &, const __nv_bfloat16 *, const float *, float *,
                                          const float *, float, const int *, cudaStream_t);

// ---------------------------------------------------------------- layout
// One thread per block row copies its blocks into the slice layout (and, for
// the first value array, the column indices); lanes of a warp write
// consecutive slots.
template <typename T>
__device__ __forceinline__ T from_f64(double a);
template <> __device__ __forceinline__ double from_f64<double>(double a) { return a; }
template <> __device__ __forceinline__ float from_f64<float>(double a) { return (float)a; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double a) {
  return __float2bfloat16_rn((float)a);
}

template <typename T, int B>
__global__ void k_to_sell(int nr, const int *__restrict__ prow, const int *__restrict__ rp,
                          const int *__restrict__ col, const double *__restrict__ src, const int *__restrict__ slp,
                          int *__restrict__ scol, T *__restrict__ dst) {
  constexpr int BB = B * B;
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nr) return;
  const int row = prow ? prow[pos] : pos;
  const int sl = pos >> 5, lane = pos & 31;
  const int kb = rp[row], len = rp[row + 1] - kb;
  const long base = slp[sl];
  for (int j = 0; j < len; ++j) {
    const long slot = base + 32L * j;
    if (scol) scol[slot + lane] = col[kb + j];
    const double *b = src + (long)BB * (kb + j);
#pragma unroll
    for (int e = 0; e < BB; ++e) dst[BB * slot + 32 * e + lane] = from_f64<T>(b[e]);
  }
}

template <typename T>
static void to_sell(const DevBsr &A, const SolveMat &M, int *cols, T *dst, cudaStream_t s) {
  const int nb = nblk(A.nr, 128);
  if (!nb) return;
  if (A.b == 1)
    AMG_KCOUNT k_to_sell<T, 1><<<nb, 128, 0, s>>>(A.nr, M.prow.p, A.rowptr.p, A.col.p, A.val.p, M.slp.p, cols, dst);
  else
    AMG_KCOUNT k_to_sell<T, 3><<<nb, 128, 0, s>>>(A.nr, M.prow.p, A.rowptr.p, A.col.p, A.val.p, M.slp.p, cols, dst);
}

// Warps per slice: few slices of long rows leave SMs idle unless several
// warps share a slice, so the warps per slice double while the launch has
// fewer than 32 warps per SM and each warp keeps at least two blocks of an
// average row per chunk.  This fixes the order of every row sum.  (Measured
// on the beam, solve to 1e-8: with a bound of 16 warps per SM FP64 64.3 ms,
// FP32 47.1 ms; 32: 63.1 and 41.0 ms, where the FP32 sums' rounding also
// took the FP32 count from 103 to 93 iterations; 8: 69.0, 52.3; 64: 65.5,
// 44.5.)
static int rule_wps(const SolveMat &M) {
  const double avg = M.nr ? (double)M.nnzb / M.nr : 1.0;
  int wps = 1;
  while (wps < 16 && (long)M.ns * wps < 32L * 152 && avg / (2.0 * wps * 2) >= 1.0) wps *= 2;
  return wps;
}

// Mapping for matrices too small to time: CTAs of 4 warps (or of one slice),
// unless that gives fewer than two CTAs per SM; then one warp per CTA.
static int rule_map(const SolveMat &M) {
  const int wps = rule_wps(M);
  const long ctas = wps <= 4 ? ((long)M.ns * wps + 3) / 4 : (long)M.ns;
  const bool w1 = ctas < 2L * 152;
  switch (wps) {
    case 1: return w1 ? 9 : 0;    // WPS 1, U 2
    case 2: return w1 ? 10 : 2;   // WPS 2, U 2
    case 4: return w1 ? 11 : 4;   // WPS 4, U 2
    case 8: return w1 ? 12 : 6;   // WPS 8, U 2
    default: return w1 ? 13 : 7;  // WPS 16, U 2
  }
}

// Slice heights of the layout: h[s] = 32 x the longest row at positions
// [32 s, 32 s + 32) (row prow[pos], or pos); their sum into *tot.  One warp
// per slice.
__global__ void k_slice_h(int nr, int ns, const int *__restrict__ rp, const int *__restrict__ prow,
                          int *__restrict__ h, unsigned long long *__restrict__ tot) {
  const int sl = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (sl >= ns) return;
  const int pos = 32 * sl + lane;
  int len = 0;
  if (pos < nr) {
    const int r = prow ? prow[pos] : pos;
    len = rp[r + 1] - rp[r];
  }
  for (int off = 16; off; off >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, off));
  if (lane == 0) {
    h[sl] = 32 * len;
    atomicAdd(tot, 32ULL * (unsigned long long)len);
  }
}

// Rows by decreasing length inside windows of SELL_SIGMA rows, ties in row
// order: the position of row r in its window is the number of rows of the
// window that are longer, plus those before r that are as long.  One CTA of
// SELL_SIGMA threads per window sorts the keys (LMAX - length, index) -- all
// distinct -- with a bitonic network in shared memory; the unused keys of a
// short last window are all ones and sort behind the rows.
static_assert(SELL_SIGMA == 1024, "the sort key holds the index in a window in 10 bits");
__global__ void __launch_bounds__(SELL_SIGMA) k_sell_perm(int nr, const int *__restrict__ rp, int *__restrict__ prow) {
  constexpr unsigned LMAX = (1u << 22) - 1u;
  __shared__ unsigned key[SELL_SIGMA];
  const int w0 = blockIdx.x * SELL_SIGMA, q = threadIdx.x;
  const int wn = min(SELL_SIGMA, nr - w0);
  unsigned kq = 0xffffffffu;
  if (q < wn) {
    const unsigned len = min((unsigned)(rp[w0 + q + 1] - rp[w0 + q]), LMAX);
    kq = ((LMAX - len) << 10) | (unsigned)q;
  }
  key[q] = kq;
  for (int k = 2; k <= SELL_SIGMA; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      __syncthreads();
      const int p = q ^ j;
      if (p > q) {
        const unsigned a = key[q], b = key[p];
        if ((a > b) == ((q & k) == 0)) {
          key[q] = b;
          key[p] = a;
        }
      }
    }
  __syncthreads();
  if (q < wn) prow[w0 + q] = w0 + (int)(key[q] & 1023u);
}

// Sliced layouts of several matrices at once.  The slot counts decide the
// allocations, so they come back to the host: all matrices' slice heights
// are formed first and read back together, then those of the matrices that
// take the sorted row order, then every layout is filled -- two
// synchronisations for the whole hierarchy instead of one or two per matrix.
int make_solvemats(const std::vector<SolveJob> &jobs, cudaStream_t s) {
  const int nj = (int)jobs.size();
  if (nj == 0) return AMG_OK;
  std::vector<DBuf<int>> hsl(nj);
  DBuf<unsigned long long> tot;
  AMG_TRY(tot.alloc(2 * (size_t)nj));
  AMG_CU(cudaMemsetAsync(tot.p, 0, 2 * (size_t)nj * sizeof(unsigned long long), s));
  std::vector<unsigned long long> slots(2 * (size_t)nj, 0ULL);
  auto heights = [&](int i, const int *prow, unsigned long long *t) {
    const SolveMat &M = *jobs[i].M;
    if (M.ns)
      AMG_KCOUNT k_slice_h<<<nblk(32L * M.ns, 256), 256, 0, s>>>(M.nr, M.ns, M.rowptr, prow, hsl[i].p, t);
  };
  for (int i = 0; i < nj; ++i) {
    const DevBsr &A = *jobs[i].A;
    SolveMat &M = *jobs[i].M;
    M.nr = A.nr;
    M.nc = A.nc;
    M.nnzb = A.nnzb;
    M.b = A.b;
    M.rowptr = A.rowptr.p;
    M.col = A.col.p;
    M.ns = (A.nr + 31) / 32;
    M.prow.release();
    AMG_TRY(hsl[i].alloc(M.ns));
    heights(i, nullptr, tot.p + i);
  }
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaMemcpyAsync(slots.data(), tot.p, (size_t)nj * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  AMG_CU(cudaStreamSynchronize(s));
  // Rows by decreasing length inside each window of SELL_SIGMA rows (ties in
  // row order), for FP64 storage only and only where the natural order fills
  // the slices poorly: FP64 instructions cost the same with idle lanes, while
  // the bandwidth-bound FP32/bf16 products lose more to the scattered row
  // order than they gain.
  bool any = false;
  for (int i = 0; i < nj; ++i) {
    const SolveJob &J = jobs[i];
    SolveMat &M = *J.M;
    if (J.f64 && !J.f32 && !J.b16 && M.nr > 0 && slots[i] > 0 && (double)M.nnzb < 0.9 * (double)slots[i]) {
      AMG_TRY(M.prow.alloc(M.nr));
      AMG_KCOUNT k_sell_perm<<<nblk(M.nr, SELL_SIGMA), SELL_SIGMA, 0, s>>>(M.nr, M.rowptr, M.prow.p);
      heights(i, M.prow.p, tot.p + nj + i);
      any = true;
    }
  }
  AMG_LAUNCH_CHECK();
  if (any) {
    AMG_CU(cudaMemcpyAsync(slots.data() + nj, tot.p + nj, (size_t)nj * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    AMG_CU(cudaStreamSynchronize(s));
  }
  for (int i = 0; i < nj; ++i) {
    const SolveJob &J = jobs[i];
    const DevBsr &A = *J.A;
    SolveMat &M = *J.M;
    const unsigned long long sl = M.prow.p ? slots[nj + i] : slots[i];
    if (sl > 0x7fffffffULL) {
      set_error("matrix too large for 32-bit slot offsets (%llu slots)", sl);
      return AMG_ERR_ARG;
    }
    M.nslot = (long)sl;
    AMG_TRY(M.slp.alloc(M.ns + 1));
    AMG_TRY(dev_scan(M.ns, hsl[i].p, 0, M.slp.p, s));
    const long tot_slots = M.nslot;
    AMG_TRY(M.scol.alloc(tot_slots));
    M.map = M.map64 = rule_map(M);
    M.wps_rule = rule_wps(M);
    if (M.wps_rule > 1) {  // partial sums of the one-warp-CTA mappings
      AMG_TRY(M.wpart.alloc((size_t)M.ns * M.wps_rule * 2 * A.b * 32));
      AMG_TRY(M.wtick.alloc(M.ns));
      AMG_TRY(M.wtick.zero(s));
    } else {
      M.wpart.release();
      M.wtick.release();
    }
    const long n9 = (long)A.b * A.b * tot_slots;
    int *cols = M.scol.p;
    if (J.f64) {
      AMG_TRY(M.v64.alloc(n9));
      to_sell<double>(A, M, cols, M.v64.p, s);
      cols = nullptr;
    }
    if (J.f32) {
      AMG_TRY(M.v32.alloc(n9));
      to_sell<float>(A, M, cols, M.v32.p, s);
      cols = nullptr;
    }
    if (J.b16) {
      AMG_TRY(M.v16.alloc(n9));
      to_sell<__nv_bfloat16>(A, M, cols, M.v16.p, s);
    }
  }
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// ---------------------------------------------------------------- autotuner
// The mapping is chosen by timing candidates on the matrix itself (CUDA
// events, one warm-up and three timed launches each).  Only WPS decides the
// order in which a row's blocks are summed (warp p sums blocks p, p + WPS,
// ... in order whatever U, and the bulk-copy variant sums them in order like
// WPS = 1), so WPS is fixed by the size rule and the timing picks among the
// candidates with that WPS: the products, and with them the iteration count
// of a solve, do not depend on which candidate won on a given run.  The
// winner is cached per (storage type, slice count, average row length) so
// that later hierarchies of the same shape reuse it; matrices too small to
// time keep the rule.
static std::mutex g_tune_mu;
static std::vector<std::pair<long long, int>> g_tune_cache;

template <typename TM, typename TX>
static int tune_one(SolveMat &M, const TM *v, cudaStream_t s, int kind) {
  const double avg = M.nr ? (double)M.nnzb / M.nr : 1.0;
  const long long key = ((long long)kind << 56) | ((long long)M.ns << 20) | (long long)(avg * 16.0 + 0.5);
  int &map = std::is_same<TM, double>::value ? M.map64 : M.map;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &e : g_tune_cache)
      if (e.first == key) {
        map = e.second;
        return AMG_OK;
      }
  }
  DBuf<TX> x, y;
  AMG_TRY(x.alloc((size_t)M.b * M.nc));
  AMG_TRY(y.alloc((size_t)M.b * M.nr));
  AMG_TRY(x.zero(s));
  cudaEvent_t e0, e1;
  AMG_CU(cudaEventCreate(&e0));
  AMG_CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int bm = map;
  const int rule_wps = kMaps[rule_map(M)].wps;
  for (int c = 0; c < kNumMaps; ++c) {
    const int wps = kMaps[c].wps == 0 ? 1 : kMaps[c].wps;  // bulk copy: one warp per slice
    if (wps != rule_wps) continue;
    if (kMaps[c].wps == 0 && (std::is_same<TM, double>::value || M.b != 3)) continue;  // no bulk variant
    map = c;
    bsrmv<TM, TX>(EP_SET, M, v, x.p, y.p, (const TX *)nullptr, TX(0), nullptr, s);
    AMG_CU(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) bsrmv<TM, TX>(EP_SET, M, v, x.p, y.p, (const TX *)nullptr, TX(0), nullptr, s);
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
  map = bm;
  if (getenv("AMG_TRACE"))
    fprintf(stderr, "[amg] mapping kind %d rows %d avg %.1f -> %s (%.4f ms)\n", kind, M.nr, avg,
            mapping_name(M, std::is_same<TM, double>::value), best / 3.0);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.push_back({key, bm});
  return AMG_OK;
}

int tune_solvemat(SolveMat &M, int kind, cudaStream_t s) {
  // AMG_MAP=<0..16> pins the mapping of every matrix (for experiments);
  // one-warp-CTA mappings only with the matrix's own warps per slice
  if (const char *pin = getenv("AMG_MAP")) {
    const int m = atoi(pin);
    if (m >= 0 && m < kNumMaps && (!kMaps[m].w1 || kMaps[m].wps == M.wps_rule)) {
      (kind == 0 ? M.map64 : M.map) = m;
      return AMG_OK;
    }
  }
  if (M.nnzb < 100000 || getenv("AMG_NO_TUNE")) return AMG_OK;
  if (kind == 0) return tune_one<double, double>(M, M.v64.p, s, 0);
  if (kind == 1) return tune_one<float, float>(M, M.v32.p, s, 1);
  return tune_one<__nv_bfloat16, float>(M, M.v16.p, s, 2);
}

int mapping_wps(const SolveMat &M, bool f64) {
  const int m = f64 ? M.map64 : M.map;
  if (m < 0 || m >= kNumMaps) return 1;
  return kMaps[m].wps == 0 ? 1 : kMaps[m].wps;  // the bulk-copy variant sums like one warp per slice
}

const char *mapping_name(const SolveMat &M, bool f64) {
  static const char *names[kNumMaps] = {"wps1_u2",    "wps1_u4",    "wps2_u2",    "wps2_u4",   "wps4_u2",
                                        "wps4_u4",    "wps8_u2",    "wps16_u2",   "bulk_copy", "w1_wps1",
                                        "w1_wps2",    "w1_wps4",    "w1_wps8",    "w1_wps16",  "w1_wps1_u4",
                                        "w1_wps2_u4", "w1_wps4_u4"};
  const int m = f64 ? M.map64 : M.map;
  return (m >= 0 && m < kNumMaps) ? names[m] : "?";
}

}  // namespace amg
