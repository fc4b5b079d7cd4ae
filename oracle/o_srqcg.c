/*
 * Oracle: test-space generation by Simultaneous Rayleigh Quotient Minimisation
 * by Conjugate Gradients, SRQCG (Sec. 3.2, Algorithm 4), on S = G A G^T.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * For each column z of Z the Rayleigh quotient rq(z) = z^T S z / z^T z is
 * lowered along a search direction p.  With a = p^T S z, b = p^T S p,
 * c = p^T z, d = p^T p, e = z^T S z, f = z^T z, rq(z + alpha p) is
 * (e + 2 alpha a + alpha^2 b) / (f + 2 alpha c + alpha^2 d), whose stationary
 * points solve (bc - ad) alpha^2 + (bf - de) alpha + (af - ce) = 0; the root
 * printed in Algorithm 4 is (de - bf + sqrt(Delta)) / (2 (bc - ad)).  Here both
 * roots are formed and the one giving the smaller quotient is kept (the
 * printed one whenever it is the minimiser).  The new gradient is
 * 2 (S z - rq z) / f with rq the Rayleigh quotient z^T S z / f, the direction
 * is made S-conjugate to the previous one (beta = -g^T S p / b), and every
 * k_ritz iterations the block Z is rotated by the Ritz vectors of the pencil
 * (Z^T S Z, Z^T Z).  At the end V = G^T Z with orthonormalised columns.
 *
 * S Z and S P are formed once from the first Z and P and then carried by the
 * same linear recurrences as Z and P (the usual SRQCG organisation; the
 * algorithm only names the quantities): z <- z + alpha p brings
 * S z <- S z + alpha S p, p <- g + beta p brings S p <- S g + beta S p, and
 * the Ritz rotation Z <- Z U brings S Z <- (S Z) U.  The one product with S
 * per column and iteration is S g.
 *
 * Loops over the entries of a vector may run on several OpenMP threads: each
 * entry is still formed by the same operations, so the results do not depend
 * on the number of threads.
 *
 * All inner products use the fixed-order or_dot, all sparse products the
 * fixed-order or_spmv; every multiply-add of a vector update (and of the
 * dense triangular solves and rotations) is one fused multiply-add, and a
 * vector divided by a shared scalar is multiplied by its reciprocal (one
 * division per vector: on the GPU a division costs about ten products).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static void apply_s(const obsr *A, const obsr *G, const obsr *GT,
                    const double *x, double *y, double *t1, double *t2) {
  or_spmv(GT, x, t1);
  or_spmv(A, t1, t2);
  or_spmv(G, t2, y);
}

/* Modified Gram-Schmidt on the columns of the n x t column-major V, in column
 * order (v_j <- v_j - (v_i . v_j) v_i for i < j, one fused multiply-add per
 * entry); each column is then multiplied by the reciprocal of its norm. */
void or_mgs(int n, int t, double *V) {
  for (int j = 0; j < t; ++j) {
    double *vj = V + (size_t)j * n;
    for (int i = 0; i < j; ++i) {
      const double *vi = V + (size_t)i * n;
      const double r = or_dot(n, vi, vj);
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int k = 0; k < n; ++k) vj[k] = fma(-r, vi[k], vj[k]);
    }
    const double nr = sqrt(or_dot(n, vj, vj));
    if (nr > 0.0) {
      const double rn = 1.0 / nr;
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int k = 0; k < n; ++k) vj[k] = vj[k] * rn;
    }
  }
}

/* Generalised symmetric eigenproblem H U = M U diag(lam), M SPD, t x t
 * row-major.  M = L L^T (or_chol); the triangular solves multiply by
 * 1 / L[i][i] like or_chol_solve; C = L^{-1} (L^{-1} H)^T, symmetrised as
 * (C + C^T) * 0.5; Jacobi sweeps until the off-diagonal mass is negligible;
 * eigenvalues sorted ascending (ties keep index order); U = L^{-T} W; each
 * column of U signed so that its entry of largest magnitude (first on ties)
 * is positive.
 *
 * A sweep visits every pair p < q once, in round-robin order (the circle
 * method of tournament scheduling): the indices, padded with one dummy index
 * when t is odd to T = t + (t mod 2), form T/2 disjoint pairs per round and
 * T - 1 rounds per sweep; in round r position 0 holds index 0 and position
 * i >= 1 holds index 1 + (i - 1 + r) mod (T - 1), and positions i and
 * T - 1 - i are paired (pairs with the dummy index are skipped).  In a round
 * the rotation of every pair with C[p][q] != 0 is computed from the current
 * C; then all column rotations are applied, then all row rotations, then the
 * rotations of W, and every rotated pivot C[p][q] = C[q][p] is set to 0.
 * Disjoint pairs touch disjoint rows and columns, so each phase could run in
 * any pair order with the same result. */
int or_gen_eig(int t, const double *H, const double *M, double *U,
               double *lam) {
  double L[64 * 64], W1[64 * 64], C[64 * 64], Wv[64 * 64], tmp[64];
  if (t > 64) return OR_ERR_ARG;
  int rc = or_chol(t, M, L);
  if (rc) return rc;
  for (int j = 0; j < t; ++j)
    for (int i = 0; i < t; ++i) {
      double s = H[i * t + j];
      for (int k = 0; k < i; ++k) s = fma(-L[i * t + k], W1[k * t + j], s);
      W1[i * t + j] = s * (1.0 / L[i * t + i]);
    }
  for (int j = 0; j < t; ++j)
    for (int i = 0; i < t; ++i) {
      double s = W1[j * t + i];
      for (int k = 0; k < i; ++k) s = fma(-L[i * t + k], C[k * t + j], s);
      C[i * t + j] = s * (1.0 / L[i * t + i]);
    }
  for (int i = 0; i < t; ++i)
    for (int j = 0; j < i; ++j) {
      const double v = (C[i * t + j] + C[j * t + i]) * 0.5;
      C[i * t + j] = v;
      C[j * t + i] = v;
    }
  for (int i = 0; i < t; ++i)
    for (int j = 0; j < t; ++j) Wv[i * t + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int p = 0; p < t; ++p) {
      dg = fma(C[p * t + p], C[p * t + p], dg);
      for (int q = p + 1; q < t; ++q) off = fma(C[p * t + q], C[p * t + q], off);
    }
    if (!(off > 1e-32 * dg)) break;
    const int T = t + (t & 1);
    for (int r = 0; r < T - 1; ++r) {
      int rp[32], rq[32], np = 0;
      double rc_[32], rs_[32];
      for (int i = 0; i < T / 2; ++i) {
        const int a = (i == 0) ? 0 : 1 + (i - 1 + r) % (T - 1);
        const int j2 = T - 1 - i;
        const int b2 = (j2 == 0) ? 0 : 1 + (j2 - 1 + r) % (T - 1);
        const int p = a < b2 ? a : b2, q = a < b2 ? b2 : a;
        if (q >= t) continue;
        const double apq = C[p * t + q];
        if (apq == 0.0) continue;
        /* tangent tt = sgn(d) a2 / (|d| + R), R = sqrt(d^2 + a2^2), the smaller
         * root of tt^2 + 2 (d / a2) tt - 1 = 0; c = 1 / sqrt(1 + tt^2) =
         * u / w and s = tt c = sgn(d) a2 / w with u = |d| + R and
         * w = sqrt(u^2 + a2^2): two square roots and one division */
        const double d = C[q * t + q] - C[p * t + p], a2 = 2.0 * apq;
        const double R = sqrt(fma(a2, a2, d * d));
        const double u = fabs(d) + R;
        const double iw = 1.0 / sqrt(fma(a2, a2, u * u));
        rp[np] = p;
        rq[np] = q;
        rc_[np] = u * iw;
        rs_[np] = (d >= 0.0 ? a2 : -a2) * iw;
        ++np;
      }
      for (int u = 0; u < np; ++u) {
        const int p = rp[u], q = rq[u];
        const double c = rc_[u], s = rs_[u];
        for (int k = 0; k < t; ++k) {
          const double xp = C[k * t + p], xq = C[k * t + q];
          C[k * t + p] = fma(c, xp, -(s * xq));
          C[k * t + q] = fma(s, xp, c * xq);
        }
      }
      for (int u = 0; u < np; ++u) {
        const int p = rp[u], q = rq[u];
        const double c = rc_[u], s = rs_[u];
        for (int k = 0; k < t; ++k) {
          const double xp = C[p * t + k], xq = C[q * t + k];
          C[p * t + k] = fma(c, xp, -(s * xq));
          C[q * t + k] = fma(s, xp, c * xq);
        }
      }
      for (int u = 0; u < np; ++u) {
        const int p = rp[u], q = rq[u];
        const double c = rc_[u], s = rs_[u];
        for (int k = 0; k < t; ++k) {
          const double xp = Wv[k * t + p], xq = Wv[k * t + q];
          Wv[k * t + p] = fma(c, xp, -(s * xq));
          Wv[k * t + q] = fma(s, xp, c * xq);
        }
      }
      for (int u = 0; u < np; ++u) {
        C[rp[u] * t + rq[u]] = 0.0;
        C[rq[u] * t + rp[u]] = 0.0;
      }
    }
  }
  int order[64];
  for (int i = 0; i < t; ++i) order[i] = i;
  for (int i = 0; i < t; ++i) {
    int best = i;
    for (int j = i + 1; j < t; ++j)
      if (C[order[j] * t + order[j]] < C[order[best] * t + order[best]]) best = j;
    const int tmpi = order[best];
    for (int j = best; j > i; --j) order[j] = order[j - 1];
    order[i] = tmpi;
  }
  for (int jj = 0; jj < t; ++jj) {
    const int j = order[jj];
    lam[jj] = C[j * t + j];
    for (int i = t - 1; i >= 0; --i) {
      double s = Wv[i * t + j];
      for (int k = t - 1; k > i; --k) s = fma(-L[k * t + i], tmp[k], s);
      tmp[i] = s * (1.0 / L[i * t + i]);
    }
    int im = 0;
    for (int i = 1; i < t; ++i)
      if (fabs(tmp[i]) > fabs(tmp[im])) im = i;
    const double sg = tmp[im] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < t; ++i) U[i * t + jj] = sg * tmp[i];
  }
  return OR_OK;
}

/* Step length of Algorithm 4: the root of
 * (bc - ad) alpha^2 + (bf - de) alpha + (af - ce) = 0 that minimises
 * rq(alpha) = (e + 2 alpha a + alpha^2 b) / (f + 2 alpha c + alpha^2 d);
 * with p1 = de - bf, q1 = bc - ad, r1 = af - ce the roots are
 * (p1 +- sqrt(p1^2 - 4 q1 r1)) / (2 q1) (the + root is the one printed), and
 * q1 = 0 leaves the linear root r1 / p1. */
double or_rq_line_min(double a, double b, double c, double d, double e,
                      double f) {
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

int or_srqcg(const obsr *A, const obsr *G, const obsr *GT, int kmax,
             int k_ritz, int t, const double *V0, double *V) {
  const int n = A->nr * A->b;
  const size_t nt = (size_t)n * t;
  double *Z = (double *)malloc(nt * sizeof(double));
  double *P = (double *)malloc(nt * sizeof(double));
  double *SZ = (double *)malloc(nt * sizeof(double));
  double *SP = (double *)malloc(nt * sizeof(double));
  double *Gv = (double *)malloc((size_t)n * sizeof(double));
  double *SG = (double *)malloc((size_t)n * sizeof(double));
  double *t1 = (double *)malloc((size_t)n * sizeof(double));
  double *t2 = (double *)malloc((size_t)n * sizeof(double));
  double f[64], H[64 * 64], M[64 * 64], U[64 * 64], lam[64];
  int rc = OR_OK;
  if (t > 64) return OR_ERR_ARG;

  /* Z0 = (I - S) V0, orthonormalised */
  for (int i = 0; i < t; ++i) {
    const double *v = V0 + (size_t)i * n;
    double *z = Z + (size_t)i * n;
    apply_s(A, G, GT, v, Gv, t1, t2);
    #pragma omp parallel for schedule(static) if (n > 65536)
    for (int k = 0; k < n; ++k) z[k] = v[k] - Gv[k];
  }
  or_mgs(n, t, Z);
  /* first residuals and directions: q = z^T S z (z has unit norm), P = 2R;
   * S Z and S P formed once here, then carried by the recurrences below */
  for (int i = 0; i < t; ++i) {
    double *z = Z + (size_t)i * n, *p = P + (size_t)i * n;
    double *sz = SZ + (size_t)i * n, *sp = SP + (size_t)i * n;
    apply_s(A, G, GT, z, sz, t1, t2);
    const double q = or_dot(n, z, sz);
    #pragma omp parallel for schedule(static) if (n > 65536)
    for (int k = 0; k < n; ++k) p[k] = 2.0 * fma(-q, z[k], sz[k]);
    apply_s(A, G, GT, p, sp, t1, t2);
    f[i] = 1.0;
  }
  for (int it = 1; it <= kmax && rc == OR_OK; ++it) {
    if (k_ritz > 0 && it % k_ritz == 0) {
      for (int i = 0; i < t; ++i)
        for (int j = i; j < t; ++j) {
          const double h = or_dot(n, Z + (size_t)i * n, SZ + (size_t)j * n);
          const double m = or_dot(n, Z + (size_t)i * n, Z + (size_t)j * n);
          H[i * t + j] = h;
          H[j * t + i] = h;
          M[i * t + j] = m;
          M[j * t + i] = m;
        }
      rc = or_gen_eig(t, H, M, U, lam);
      if (rc) break;
      /* Z <- Z U and S Z <- (S Z) U, column j = sum_i X_i U[i][j], i
       * ascending from 0 */
      for (int w = 0; w < 2; ++w) {
        double *X = w == 0 ? Z : SZ;
        #pragma omp parallel for schedule(static) if (n > 65536)
        for (int k = 0; k < n; ++k) {
          double row[64];
          for (int j = 0; j < t; ++j) {
            double s = 0.0;
            for (int i = 0; i < t; ++i) s = fma(X[(size_t)i * n + k], U[i * t + j], s);
            row[j] = s;
          }
          for (int j = 0; j < t; ++j) X[(size_t)j * n + k] = row[j];
        }
      }
      for (int i = 0; i < t; ++i) f[i] = 1.0;
    }
    for (int i = 0; i < t; ++i) {
      double *z = Z + (size_t)i * n, *p = P + (size_t)i * n;
      double *sz = SZ + (size_t)i * n, *sp = SP + (size_t)i * n;
      const double a = or_dot(n, p, sz), b = or_dot(n, p, sp), c = or_dot(n, p, z);
      const double d = or_dot(n, p, p), e = or_dot(n, z, sz), fi = f[i];
      if (!(b > 0.0)) continue;
      const double alpha = or_rq_line_min(a, b, c, d, e, fi);
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int k = 0; k < n; ++k) {
        z[k] = fma(alpha, p[k], z[k]);
        sz[k] = fma(alpha, sp[k], sz[k]);
      }
      const double fn = or_dot(n, z, z);
      const double q = or_dot(n, z, sz) / fn;
      const double rf = 1.0 / fn;
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int k = 0; k < n; ++k) Gv[k] = (2.0 * fma(-q, z[k], sz[k])) * rf;
      apply_s(A, G, GT, Gv, SG, t1, t2);
      const double beta = -(or_dot(n, Gv, sp) / b);
      #pragma omp parallel for schedule(static) if (n > 65536)
      for (int k = 0; k < n; ++k) {
        p[k] = fma(beta, p[k], Gv[k]);
        sp[k] = fma(beta, sp[k], SG[k]);
      }
      f[i] = fn;
    }
  }
  if (rc == OR_OK) {
    for (int i = 0; i < t; ++i) or_spmv(GT, Z + (size_t)i * n, V + (size_t)i * n);
    or_mgs(n, t, V);
  }
  free(Z); free(P); free(SZ); free(SP); free(Gv); free(SG); free(t1); free(t2);
  return rc;
}
