/*
 * Oracle: small-strain linear-elastic finite elements on a structured mesh of
 * trilinear (Q1) hexahedra, the problem class of the paper (Sec. 1: K is the
 * numerical integral of B^T D B over the body; D is SPD and fixed by E and nu).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Mesh conventions.  Nodes (ix,iy,iz), 0 <= ix <= nx, ..., global id
 * ix + (nx+1)*(iy + (ny+1)*iz), coordinates (ix*hx, iy*hy, iz*hz).  Element
 * (ex,ey,ez) has id ex + nx*(ey + ny*ez); its local node a = dx + 2*dy + 4*dz
 * sits at (ex+dx, ey+dy, ez+dz).  Clamped nodes are removed; the free nodes are
 * numbered in increasing global id.  The dofs of free node I are 3I, 3I+1,
 * 3I+2 (x, y, z).
 *
 * The element matrix uses 2x2x2 Gauss quadrature (the paper says only
 * "numerical integration").  Every element has the same shape and nu, so
 * K_e = E_e * Ke0 with Ke0 the matrix for E = 1 (D is linear in E).  Ke0 is
 * integrated on its upper triangle and mirrored, so K is exactly symmetric.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* Isotropic D for E = 1 in Voigt order (xx, yy, zz, xy, yz, zx) with
 * engineering shear strains: lambda = nu/((1+nu)(1-2nu)), mu = 1/(2(1+nu)). */
static void d_matrix(double nu, double D[6][6]) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  memset(D, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) D[i][j] = lam;
    D[i][i] = lam + 2.0 * mu;
    D[3 + i][3 + i] = mu;
  }
}

int or_ke0(double nu, double hx, double hy, double hz, double *Ke) {
  if (!(hx > 0 && hy > 0 && hz > 0) || !(nu > -1.0 && nu < 0.5)) return OR_ERR_ARG;
  double D[6][6];
  d_matrix(nu, D);
  const double g = 1.0 / sqrt(3.0);
  const double sx = 2.0 / hx, sy = 2.0 / hy, sz = 2.0 / hz;
  const double wdet = ((0.5 * hx) * (0.5 * hy)) * (0.5 * hz);
  memset(Ke, 0, 576 * sizeof(double));
  for (int q = 0; q < 8; ++q) {
    const double xi = (q & 1) ? g : -g, eta = (q & 2) ? g : -g, zeta = (q & 4) ? g : -g;
    double B[6][24];
    memset(B, 0, sizeof B);
    for (int a = 0; a < 8; ++a) {
      const double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0, za = (a & 4) ? 1.0 : -1.0;
      /* shape function N_a = (1 + xa xi)(1 + ya eta)(1 + za zeta) / 8 */
      const double dxi = ((xa * (1.0 + ya * eta)) * (1.0 + za * zeta)) * 0.125;
      const double deta = ((ya * (1.0 + xa * xi)) * (1.0 + za * zeta)) * 0.125;
      const double dzeta = ((za * (1.0 + xa * xi)) * (1.0 + ya * eta)) * 0.125;
      const double Nx = dxi * sx, Ny = deta * sy, Nz = dzeta * sz;
      B[0][3 * a + 0] = Nx;
      B[1][3 * a + 1] = Ny;
      B[2][3 * a + 2] = Nz;
      B[3][3 * a + 0] = Ny;
      B[3][3 * a + 1] = Nx;
      B[4][3 * a + 1] = Nz;
      B[4][3 * a + 2] = Ny;
      B[5][3 * a + 0] = Nz;
      B[5][3 * a + 2] = Nx;
    }
    double DB[6][24];
    for (int k = 0; k < 6; ++k)
      for (int s = 0; s < 24; ++s) {
        double t = 0.0;
        for (int l = 0; l < 6; ++l) t = t + D[k][l] * B[l][s];
        DB[k][s] = t;
      }
    for (int p = 0; p < 24; ++p)
      for (int s = p; s < 24; ++s) {
        double t = 0.0;
        for (int k = 0; k < 6; ++k) t = t + B[k][p] * DB[k][s];
        Ke[p * 24 + s] = Ke[p * 24 + s] + t * wdet;
      }
  }
  for (int p = 0; p < 24; ++p)
    for (int s = 0; s < p; ++s) Ke[p * 24 + s] = Ke[s * 24 + p];
  return OR_OK;
}

static int clamped(int ix, int iy, int iz, int axis) {
  (void)iy;
  if (axis == 0) return ix == 0;
  if (axis == 2) return iz == 0;
  return 0;
}

int or_assemble(int nx, int ny, int nz, double hx, double hy, double hz,
                double nu, const double *E, int clamp_axis, obsr *K,
                int *node_map) {
  if (nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
  const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  const long nnode = (long)NX * NY * NZ;
  int nfree = 0;
  for (int iz = 0; iz < NZ; ++iz)
    for (int iy = 0; iy < NY; ++iy)
      for (int ix = 0; ix < NX; ++ix) {
        const long gid = ix + (long)NX * (iy + (long)NY * iz);
        node_map[gid] = clamped(ix, iy, iz, clamp_axis) ? -1 : nfree++;
      }
  /* pattern: free neighbours within one step in each index, ascending id */
  int *cnt = (int *)calloc((size_t)nfree + 1, sizeof(int));
  long nnzb = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      if (or_bsr_alloc(K, nfree, nfree, 3, (int)nnzb)) return OR_ERR_MEM;
      K->rowptr[0] = 0;
      for (int i = 0; i < nfree; ++i) K->rowptr[i + 1] = K->rowptr[i] + cnt[i];
    }
    for (int iz = 0; iz < NZ; ++iz)
      for (int iy = 0; iy < NY; ++iy)
        for (int ix = 0; ix < NX; ++ix) {
          const int I = node_map[ix + (long)NX * (iy + (long)NY * iz)];
          if (I < 0) continue;
          int c = 0;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
                if (jx < 0 || jy < 0 || jz < 0 || jx >= NX || jy >= NY || jz >= NZ) continue;
                const int J = node_map[jx + (long)NX * (jy + (long)NY * jz)];
                if (J < 0) continue;
                if (pass == 1) K->col[K->rowptr[I] + c] = J;
                ++c;
              }
          if (pass == 0) {
            cnt[I] = c;
            nnzb += c;
          }
        }
  }
  free(cnt);
  (void)nnode;
  double Ke0[576];
  int rc = or_ke0(nu, hx, hy, hz, Ke0);
  if (rc) return rc;
  /* element loop in increasing element id: every block entry is the sum of
   * E_e * Ke0 entries over its elements in that order, starting from 0 */
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        const long e = ex + (long)nx * (ey + (long)ny * ez);
        int nodes[8];
        for (int a = 0; a < 8; ++a) {
          const int jx = ex + (a & 1), jy = ey + ((a >> 1) & 1), jz = ez + ((a >> 2) & 1);
          nodes[a] = node_map[jx + (long)NX * (jy + (long)NY * jz)];
        }
        for (int a = 0; a < 8; ++a) {
          if (nodes[a] < 0) continue;
          for (int bb = 0; bb < 8; ++bb) {
            if (nodes[bb] < 0) continue;
            double *blk = (double *)or_bsr_find(K, nodes[a], nodes[bb]);
            for (int r = 0; r < 3; ++r)
              for (int c = 0; c < 3; ++c)
                blk[r * 3 + c] = blk[r * 3 + c] + E[e] * Ke0[(3 * a + r) * 24 + 3 * bb + c];
          }
        }
      }
  return OR_OK;
}

/* Rigid-body modes at the free nodes, about the mesh centre
 * (X = ix*hx - 0.5*(nx*hx), ...): translations x, y, z, then the rotations
 * (-Y, X, 0), (0, -Z, Y), (Z, 0, -X).  V is (3*nfree) x 6, column-major. */
int or_rbm(int nx, int ny, int nz, double hx, double hy, double hz,
           const int *node_map, int nfree, double *V) {
  const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  const long n = 3L * nfree;
  memset(V, 0, (size_t)n * 6 * sizeof(double));
  for (int iz = 0; iz < NZ; ++iz)
    for (int iy = 0; iy < NY; ++iy)
      for (int ix = 0; ix < NX; ++ix) {
        const int I = node_map[ix + (long)NX * (iy + (long)NY * iz)];
        if (I < 0) continue;
        const double X = (double)ix * hx - 0.5 * ((double)nx * hx);
        const double Y = (double)iy * hy - 0.5 * ((double)ny * hy);
        const double Z = (double)iz * hz - 0.5 * ((double)nz * hz);
        const long u = 3L * I, v = u + 1, w = u + 2;
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
  return OR_OK;
}

/* Consistent body load: every element gives each of its nodes g * V_e / 8,
 * elements in increasing id. */
int or_load_body(int nx, int ny, int nz, double hx, double hy, double hz,
                 const double *g, const int *node_map, double *f) {
  const int NX = nx + 1, NY = ny + 1;
  const double share = ((hx * hy) * hz) * 0.125;
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex)
        for (int a = 0; a < 8; ++a) {
          const int jx = ex + (a & 1), jy = ey + ((a >> 1) & 1), jz = ez + ((a >> 2) & 1);
          const int I = node_map[jx + (long)NX * (jy + (long)NY * jz)];
          if (I < 0) continue;
          for (int c = 0; c < 3; ++c) f[3L * I + c] = f[3L * I + c] + g[c] * share;
        }
  return OR_OK;
}

/* Pressure p[ex + nx*ey] on the top face (z = nz*hz) pushing in -z: each face
 * node receives -(p * hx*hy) / 4, face elements in increasing id. */
int or_load_top_pressure(int nx, int ny, int nz, double hx, double hy,
                         double hz, const double *p, const int *node_map,
                         double *f) {
  (void)hz;
  const int NX = nx + 1, NY = ny + 1;
  const double area = hx * hy;
  for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
      const double share = (p[ex + (long)nx * ey] * area) * 0.25;
      for (int a = 0; a < 4; ++a) {
        const int jx = ex + (a & 1), jy = ey + ((a >> 1) & 1);
        const int I = node_map[jx + (long)NX * (jy + (long)NY * nz)];
        if (I < 0) continue;
        f[3L * I + 2] = f[3L * I + 2] - share;
      }
    }
  return OR_OK;
}

/* Shear on the end face x = nx*hx: a uniform traction in z of resultant
 * `total`, i.e. traction total / ((ny*hy)*(nz*hz)); each face quad gives each
 * of its nodes (traction * hy*hz) / 4, quads with ez outer, ey inner. */
int or_load_end_shear(int nx, int ny, int nz, double hx, double hy, double hz,
                      double total, const int *node_map, double *f) {
  (void)hx;
  const int NX = nx + 1, NY = ny + 1;
  const double t = total / (((double)ny * hy) * ((double)nz * hz));
  const double share = (t * (hy * hz)) * 0.25;
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int a = 0; a < 4; ++a) {
        const int jy = ey + (a & 1), jz = ez + ((a >> 1) & 1);
        const int I = node_map[nx + (long)NX * (jy + (long)NY * jz)];
        if (I < 0) continue;
        f[3L * I + 2] = f[3L * I + 2] + share;
      }
  return OR_OK;
}
