// Structured Q1-hex linear elasticity (Sec. 1 of the paper: K is the
// integral of B^T D B, D isotropic and SPD for given E and nu).  Element
// matrix by 2x2x2 Gauss quadrature for E = 1 (upper triangle integrated and
// mirrored), K = sum_e E_e Ke0 summed over elements in increasing id, loads
// and rigid-body modes.  Compiled with -fmad=false: every entry is produced by
// the same sequence of rounded operations as the plain definition, so K is
// reproducible bit for bit (the hierarchy's structure depends on it).
// Element-sensitivity kernel for the adjoint: grad_e = -dEdp_e lam_e^T Ke0 u_e.
#include <cstring>
#include <vector>

#include "amg_internal.h"

namespace amg {

static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// B[k][col] of the trilinear element at natural point (xi, eta, zeta)
__device__ double bentry(int k, int col, double xi, double eta, double zeta, double sx, double sy, double sz) {
  const int a = col / 3, comp = col % 3;
  const double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0, za = (a & 4) ? 1.0 : -1.0;
  const double dxi = ((xa * (1.0 + ya * eta)) * (1.0 + za * zeta)) * 0.125;
  const double deta = ((ya * (1.0 + xa * xi)) * (1.0 + za * zeta)) * 0.125;
  const double dzeta = ((za * (1.0 + xa * xi)) * (1.0 + ya * eta)) * 0.125;
  const double Nx = dxi * sx, Ny = deta * sy, Nz = dzeta * sz;
  // Voigt rows xx, yy, zz, xy, yz, zx with engineering shear strains
  if (comp == 0) return k == 0 ? Nx : k == 3 ? Ny : k == 5 ? Nz : 0.0;
  if (comp == 1) return k == 1 ? Ny : k == 3 ? Nx : k == 4 ? Nz : 0.0;
  return k == 2 ? Nz : k == 4 ? Ny : k == 5 ? Nx : 0.0;
}

__global__ void k_ke0(double nu, double hx, double hy, double hz, double *__restrict__ Ke) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 576) return;
  const int p = tid / 24, s = tid % 24;
  if (s < p) return;
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  double D[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) D[i][j] = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) D[i][j] = lam;
    D[i][i] = lam + 2.0 * mu;
    D[3 + i][3 + i] = mu;
  }
  const double g = 1.0 / sqrt(3.0);
  const double sx = 2.0 / hx, sy = 2.0 / hy, sz = 2.0 / hz;
  const double wdet = ((0.5 * hx) * (0.5 * hy)) * (0.5 * hz);
  double acc = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xi = (q & 1) ? g : -g, eta = (q & 2) ? g : -g, zeta = (q & 4) ? g : -g;
    double t = 0.0;
    for (int k = 0; k < 6; ++k) {
      double db = 0.0;
      for (int l = 0; l < 6; ++l) db = db + D[k][l] * bentry(l, s, xi, eta, zeta, sx, sy, sz);
      t = t + bentry(k, p, xi, eta, zeta, sx, sy, sz) * db;
    }
    acc = acc + t * wdet;
  }
  Ke[p * 24 + s] = acc;
  Ke[s * 24 + p] = acc;
}

struct Mesh {
  int nx, ny, nz, clamp;
  std::vector<int> node_map, f2g, rowptr, col;
};

static bool clamped(int ix, int iz, int clamp) { return (clamp == 0 && ix == 0) || (clamp == 2 && iz == 0); }

static int build_mesh(int nx, int ny, int nz, int clamp, Mesh &m, bool pattern) {
  if (nx < 1 || ny < 1 || nz < 1 || (clamp != -1 && clamp != 0 && clamp != 2)) {
    set_error("mesh: invalid sizes or clamp");
    return AMG_ERR_ARG;
  }
  const long NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  if (NX * NY * NZ > 400000000L) {
    set_error("mesh: too many nodes");
    return AMG_ERR_ARG;
  }
  m.nx = nx; m.ny = ny; m.nz = nz; m.clamp = clamp;
  m.node_map.assign(NX * NY * NZ, -1);
  m.f2g.clear();
  for (long iz = 0; iz < NZ; ++iz)
    for (long iy = 0; iy < NY; ++iy)
      for (long ix = 0; ix < NX; ++ix) {
        const long gid = ix + NX * (iy + NY * iz);
        if (!clamped((int)ix, (int)iz, clamp)) {
          m.node_map[gid] = (int)m.f2g.size();
          m.f2g.push_back((int)gid);
        }
      }
  if (!pattern) return AMG_OK;
  const int nf = (int)m.f2g.size();
  m.rowptr.assign(nf + 1, 0);
  m.col.clear();
  m.col.reserve((size_t)nf * 27);
  for (int I = 0; I < nf; ++I) {
    const long g = m.f2g[I];
    const long ix = g % NX, iy = (g / NX) % NY, iz = g / (NX * NY);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const long jx = ix + dx, jy = iy + dy, jz = iz + dz;
          if (jx < 0 || jy < 0 || jz < 0 || jx >= NX || jy >= NY || jz >= NZ) continue;
          const int J = m.node_map[jx + NX * (jy + NY * jz)];
          if (J >= 0) m.col.push_back(J);
        }
    m.rowptr[I + 1] = (int)m.col.size();
  }
  return AMG_OK;
}

// Block (I,J): sum over the elements containing both nodes, increasing id.
__global__ void k_assemble(int nfree, long nnzb, int nx, int ny, int nz, const int *__restrict__ rp,
                           const int *__restrict__ col, const int *__restrict__ f2g, const double *__restrict__ E,
                           const double *__restrict__ Ke, double *__restrict__ val) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzb) return;
  int lo = 0, hi = nfree - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= q) lo = mid; else hi = mid - 1;
  }
  const long NX = nx + 1, NY = ny + 1;
  const long gi = f2g[lo], gj = f2g[col[q]];
  const int ix = (int)(gi % NX), iy = (int)((gi / NX) % NY), iz = (int)(gi / (NX * NY));
  const int jx = (int)(gj % NX), jy = (int)((gj / NX) % NY), jz = (int)(gj / (NX * NY));
  double acc[9];
  for (int e = 0; e < 9; ++e) acc[e] = 0.0;
  const int ex0 = max(max(ix, jx) - 1, 0), ex1 = min(min(ix, jx), nx - 1);
  const int ey0 = max(max(iy, jy) - 1, 0), ey1 = min(min(iy, jy), ny - 1);
  const int ez0 = max(max(iz, jz) - 1, 0), ez1 = min(min(iz, jz), nz - 1);
  for (int ez = ez0; ez <= ez1; ++ez)
    for (int ey = ey0; ey <= ey1; ++ey)
      for (int ex = ex0; ex <= ex1; ++ex) {
        const long e = ex + (long)nx * (ey + (long)ny * ez);
        const int a = (ix - ex) + 2 * (iy - ey) + 4 * (iz - ez);
        const int b = (jx - ex) + 2 * (jy - ey) + 4 * (jz - ez);
        const double Ee = E[e];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) acc[r * 3 + c] = acc[r * 3 + c] + Ee * Ke[(3 * a + r) * 24 + 3 * b + c];
      }
  for (int e = 0; e < 9; ++e) val[q * 9 + e] = acc[e];
}

__device__ __forceinline__ void node_xyz(long g, int nx, int ny, int &ix, int &iy, int &iz) {
  const long NX = nx + 1, NY = ny + 1;
  ix = (int)(g % NX);
  iy = (int)((g / NX) % NY);
  iz = (int)(g / (NX * NY));
}

// kind 0 body force, 1 top pressure, 2 end shear, 3 top nodal forces
__global__ void k_load(int nfree, int nx, int ny, int nz, double hx, double hy, double hz, int kind, double g0,
                       double g1, double g2, const double *__restrict__ p, const int *__restrict__ f2g,
                       double *__restrict__ f) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nfree) return;
  int ix, iy, iz;
  node_xyz(f2g[I], nx, ny, ix, iy, iz);
  const long o = 3L * I;
  if (kind == 0) {
    const double share = ((hx * hy) * hz) * 0.125;
    const double gg[3] = {g0, g1, g2};
    for (int ez = max(iz - 1, 0); ez <= min(iz, nz - 1); ++ez)
      for (int ey = max(iy - 1, 0); ey <= min(iy, ny - 1); ++ey)
        for (int ex = max(ix - 1, 0); ex <= min(ix, nx - 1); ++ex)
          for (int c = 0; c < 3; ++c) f[o + c] = f[o + c] + gg[c] * share;
  } else if (kind == 1) {
    if (iz != nz) return;
    const double area = hx * hy;
    for (int ey = max(iy - 1, 0); ey <= min(iy, ny - 1); ++ey)
      for (int ex = max(ix - 1, 0); ex <= min(ix, nx - 1); ++ex) {
        const double share = (p[ex + (long)nx * ey] * area) * 0.25;
        f[o + 2] = f[o + 2] - share;
      }
  } else if (kind == 2) {
    if (ix != nx) return;
    const double t = g0 / (((double)ny * hy) * ((double)nz * hz));
    const double share = (t * (hy * hz)) * 0.25;
    for (int ez = max(iz - 1, 0); ez <= min(iz, nz - 1); ++ez)
      for (int ey = max(iy - 1, 0); ey <= min(iy, ny - 1); ++ey) f[o + 2] = f[o + 2] + share;
  } else {
    if (iz != nz) return;
    const long tn = ix + (long)(nx + 1) * iy;
    for (int c = 0; c < 3; ++c) f[o + c] = f[o + c] + p[tn * 3 + c];
  }
}

__global__ void k_rbm(int nfree, int nx, int ny, int nz, double hx, double hy, double hz,
                      const int *__restrict__ f2g, double *__restrict__ V) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nfree) return;
  int ix, iy, iz;
  node_xyz(f2g[I], nx, ny, ix, iy, iz);
  const long n = 3L * nfree, u = 3L * I, v = u + 1, w = u + 2;
  const double X = (double)ix * hx - 0.5 * ((double)nx * hx);
  const double Y = (double)iy * hy - 0.5 * ((double)ny * hy);
  const double Z = (double)iz * hz - 0.5 * ((double)nz * hz);
  for (int c = 0; c < 6; ++c) {
    V[c * n + u] = 0.0;
    V[c * n + v] = 0.0;
    V[c * n + w] = 0.0;
  }
  V[0 * n + u] = 1.0;
  V[1 * n + v] = 1.0;
  V[2 * n + w] = 1.0;
  V[3 * n + u] = -Y;
  V[3 * n + v] = X;
  V[4 * n + v] = -Z;
  V[4 * n + w] = Y;
  V[5 * n + u] = Z;
  V[5 * n + w] = -X;
}

__global__ void k_conn(long ne, int nx, int ny, int nz, const int *__restrict__ node_map, int *__restrict__ conn) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((long)nx * ny));
  const long NX = nx + 1, NY = ny + 1;
  for (int a = 0; a < 8; ++a) {
    const long gx = ex + (a & 1), gy = ey + ((a >> 1) & 1), gz = ez + ((a >> 2) & 1);
    conn[e * 8 + a] = node_map[gx + NX * (gy + NY * gz)];
  }
}

// grad_e = -dEdp_e * lam_e^T Ke0 u_e (clamped dofs contribute zero)
__global__ void __launch_bounds__(128) k_elem_grad(long ne, const int *__restrict__ conn, const double *__restrict__ Ke,
                                                   const double *__restrict__ dEdp, const double *__restrict__ U,
                                                   const double *__restrict__ Lam, double *__restrict__ grad) {
  __shared__ double sK[576];
  for (int i = threadIdx.x; i < 576; i += blockDim.x) sK[i] = Ke[i];
  __syncthreads();
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double u[24], l[24];
  for (int a = 0; a < 8; ++a) {
    const int I = conn[e * 8 + a];
    for (int c = 0; c < 3; ++c) {
      u[3 * a + c] = I >= 0 ? U[3L * I + c] : 0.0;
      l[3 * a + c] = I >= 0 ? Lam[3L * I + c] : 0.0;
    }
  }
  double s = 0.0;
  for (int p = 0; p < 24; ++p) {
    double t = 0.0;
    for (int q = 0; q < 24; ++q) t += sK[p * 24 + q] * u[q];
    s += l[p] * t;
  }
  grad[e] = -dEdp[e] * s;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_fe_size(int nx, int ny, int nz, int clamp, int *nfree, int *nnzb) {
  Mesh m;
  AMG_TRY(build_mesh(nx, ny, nz, clamp, m, true));
  if (nfree) *nfree = (int)m.f2g.size();
  if (nnzb) *nnzb = (int)m.col.size();
  return AMG_OK;
}

extern "C" int amg_fe_assemble(int nx, int ny, int nz, double hx, double hy, double hz, double nu, const double *E,
                               int clamp, int *node_map, int *rowptr, int *colind, double *vals, double *Ke0,
                               void *stream) {
  if (!E || !rowptr || !colind || !vals || !Ke0 || !(hx > 0 && hy > 0 && hz > 0) || !(nu > -1.0 && nu < 0.5)) {
    set_error("amg_fe_assemble: invalid argument");
    return AMG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  StreamScope scope(s);  // temporaries are taken and returned on s
  Mesh m;
  AMG_TRY(build_mesh(nx, ny, nz, clamp, m, true));
  const int nf = (int)m.f2g.size();
  const long nnzb = (long)m.col.size();
  if (node_map) memcpy(node_map, m.node_map.data(), m.node_map.size() * sizeof(int));
  DBuf<int> f2g;
  AMG_TRY(f2g.alloc(nf));
  AMG_CU(cudaMemcpyAsync(f2g.p, m.f2g.data(), nf * sizeof(int), cudaMemcpyHostToDevice, s));
  AMG_CU(cudaMemcpyAsync(rowptr, m.rowptr.data(), (nf + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  AMG_CU(cudaMemcpyAsync(colind, m.col.data(), nnzb * sizeof(int), cudaMemcpyHostToDevice, s));
  AMG_KCOUNT k_ke0<<<3, 192, 0, s>>>(nu, hx, hy, hz, Ke0);
  AMG_KCOUNT k_assemble<<<nblk(nnzb, 128), 128, 0, s>>>(nf, nnzb, nx, ny, nz, rowptr, colind, f2g.p, E, Ke0, vals);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" int amg_fe_load(int nx, int ny, int nz, double hx, double hy, double hz, int clamp, int kind,
                           const double *g, const double *p, double *f, void *stream) {
  if (!f || kind < 0 || kind > 3 || ((kind == 1 || kind == 3) && !p) || ((kind == 0 || kind == 2) && !g)) {
    set_error("amg_fe_load: invalid argument");
    return AMG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  StreamScope scope(s);  // temporaries are taken and returned on s
  Mesh m;
  AMG_TRY(build_mesh(nx, ny, nz, clamp, m, false));
  const int nf = (int)m.f2g.size();
  DBuf<int> f2g;
  AMG_TRY(f2g.alloc(nf));
  AMG_CU(cudaMemcpyAsync(f2g.p, m.f2g.data(), nf * sizeof(int), cudaMemcpyHostToDevice, s));
  const double g0 = g ? g[0] : 0.0, g1 = (g && kind == 0) ? g[1] : 0.0, g2 = (g && kind == 0) ? g[2] : 0.0;
  AMG_KCOUNT k_load<<<nblk(nf, 128), 128, 0, s>>>(nf, nx, ny, nz, hx, hy, hz, kind, g0, g1, g2, p, f2g.p, f);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" int amg_fe_rbm(int nx, int ny, int nz, double hx, double hy, double hz, int clamp, double *V,
                          void *stream) {
  if (!V) return AMG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StreamScope scope(s);  // temporaries are taken and returned on s
  Mesh m;
  AMG_TRY(build_mesh(nx, ny, nz, clamp, m, false));
  const int nf = (int)m.f2g.size();
  DBuf<int> f2g;
  AMG_TRY(f2g.alloc(nf));
  AMG_CU(cudaMemcpyAsync(f2g.p, m.f2g.data(), nf * sizeof(int), cudaMemcpyHostToDevice, s));
  AMG_KCOUNT k_rbm<<<nblk(nf, 128), 128, 0, s>>>(nf, nx, ny, nz, hx, hy, hz, f2g.p, V);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" int amg_fe_conn(int nx, int ny, int nz, int clamp, int *conn, void *stream) {
  if (!conn) return AMG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StreamScope scope(s);  // temporaries are taken and returned on s
  Mesh m;
  AMG_TRY(build_mesh(nx, ny, nz, clamp, m, false));
  DBuf<int> nm;
  AMG_TRY(nm.alloc(m.node_map.size()));
  AMG_CU(cudaMemcpyAsync(nm.p, m.node_map.data(), m.node_map.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  const long ne = (long)nx * ny * nz;
  AMG_KCOUNT k_conn<<<nblk(ne, 128), 128, 0, s>>>(ne, nx, ny, nz, nm.p, conn);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" int amg_elem_grad(int ne, const int *conn, const double *Ke0, const double *dEdp, const double *U,
                             const double *Lam, double *grad, void *stream) {
  if (ne < 0 || !conn || !Ke0 || !dEdp || !U || !Lam || !grad) {
    set_error("amg_elem_grad: invalid argument");
    return AMG_ERR_ARG;
  }
  if (ne == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_elem_grad<<<nblk(ne, 128), 128, 0, s>>>(ne, conn, Ke0, dEdp, U, Lam, grad);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}

// Scalar CSR copy of a 3x3-block matrix: scalar row 3I + r lists, for each
// block k of block row I in order, the entries (3I + r, 3 col[k] + c), c = 0..2
// (explicit zeros of a stored block included, so the pattern is the block
// pattern expanded).  One thread per scalar row.
__global__ void k_bsr_to_scalar(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ val, int *__restrict__ srp, int *__restrict__ scol,
                                double *__restrict__ sval) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3L * nr) return;
  const int I = (int)(i / 3), r = (int)(i - 3L * I);
  const int kb = rp[I], len = rp[I + 1] - kb;
  const long start = 9L * kb + 3L * r * len;
  srp[i] = (int)start;
  if (i == 3L * nr - 1) srp[3L * nr] = 9 * rp[nr];
  for (int q = 0; q < len; ++q)
    for (int c = 0; c < 3; ++c) {
      scol[start + 3 * q + c] = 3 * col[kb + q] + c;
      sval[start + 3 * q + c] = val[9L * (kb + q) + 3 * r + c];
    }
}

extern "C" int amg_bsr_to_scalar(int nr, int nnzb, const int *rowptr, const int *colind, const double *vals,
                                 int *srowptr, int *scolind, double *svals, void *stream) {
  if (nr < 1 || nnzb < 0 || nnzb > 0x7fffffff / 9 || !rowptr || !colind || !vals || !srowptr || !scolind ||
      !svals) {
    set_error("amg_bsr_to_scalar: invalid argument");
    return AMG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  AMG_KCOUNT k_bsr_to_scalar<<<nblk(3L * nr, 128), 128, 0, s>>>(nr, rowptr, colind, vals, srowptr, scolind, svals);
  AMG_LAUNCH_CHECK();
  AMG_CU(cudaStreamSynchronize(s));
  return AMG_OK;
}
