// extern "C" entry points of include/aspamg.h: argument checks, handle
// management and host staging; the work is in setup.cu and solve.cu.
#include <chrono>
#include <cstring>
#include <new>

#include "amg_internal.h"

namespace amg {
const char *last_error();
}

using namespace amg;

extern "C" int amg_default_params(amg_params *p) {
  if (!p) return AMG_ERR_ARG;
  memset(p, 0, sizeof *p);
  p->k_g = 4;
  p->rho_g = 2;
  p->eps_g = 1e-3;
  p->k_i = 4;
  p->rho_i = 2;
  p->eps_i = 1e-3;
  p->omega_bar = 0.8;
  p->rho_bar = 2.0 * (1.0 + 4.0 * 2.0);
  p->max_refine = 2;
  p->max_g_nodes = 24;
  p->lanczos_m = 20;
  p->omega_safety = 0.95;
  p->n_tv = 10;
  p->n_rq = 10;
  p->k_ritz = 1;
  p->theta = 5;
  p->n_max = 5;
  p->d_p = 2;
  p->kappa_p = 50.0;
  p->n_coarse = 1536;
  p->max_levels = 20;
  p->max_coarse_ratio = 0.9;
  p->vcycle_prec = AMG_FP64;
  p->maxit = 1000;
  p->seed = 20190205ull;
  p->block = 3;
  return AMG_OK;
}

static int check_params(const amg_params *p) {
  if (!p) return AMG_ERR_ARG;
  if (p->k_g < 0 || p->rho_g < 1 || p->k_i < 0 || p->rho_i < 1 || p->max_g_nodes < 1 || p->max_g_nodes > 64 ||
      p->lanczos_m < 1 || p->lanczos_m > 64 || p->n_tv < 3 || p->n_tv > 16 || p->n_rq < 0 || p->k_ritz < 0 ||
      p->theta < 1 || p->n_max < 1 || p->d_p < 1 || !(p->kappa_p >= 1.0) || p->n_coarse < 0 || p->max_levels < 1 ||
      p->vcycle_prec < AMG_FP64 || p->vcycle_prec > AMG_FP32_BF16GP || p->maxit < 1 ||
      (p->block != 1 && p->block != 3) || p->n_tv < p->block) {
    set_error("amg_params: a parameter is out of the supported range");
    return AMG_ERR_ARG;
  }
  return AMG_OK;
}

extern "C" int amg_setup(const amg_params *p, int nnodes, int nnzb, const int *rowptr, const int *colind,
                         const double *vals, int ntv0, const double *V0, int mem, void *stream, amg_handle *out) {
  if (out) *out = nullptr;
  if (!out || nnodes < 1 || nnzb < nnodes || !rowptr || !colind || !vals || ntv0 < 0 ||
      (ntv0 > 0 && !V0) || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE)) {
    set_error("amg_setup: invalid argument");
    return AMG_ERR_ARG;
  }
  AMG_TRY(check_params(p));
  if (ntv0 > p->n_tv) {
    set_error("amg_setup: ntv0 = %d exceeds n_tv = %d", ntv0, p->n_tv);
    return AMG_ERR_ARG;
  }
  Handle *h = new (std::nothrow) Handle();
  if (!h) return AMG_ERR_MEM;
  h->prm = *p;
  h->b = p->block;
  if (cudaGetDevice(&h->dev) != cudaSuccess) {
    delete h;
    set_error("amg_setup: cudaGetDevice failed");
    return AMG_ERR_CUDA;
  }
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {
    // the legacy default stream cannot be captured into a CUDA graph; a
    // blocking stream still orders after work the caller queued on it
    if (cudaStreamCreate(&h->stream) != cudaSuccess) {
      delete h;
      set_error("amg_setup: cudaStreamCreate failed");
      return AMG_ERR_CUDA;
    }
    h->own_stream = true;
  }
  h->n = nnodes;
  StreamScope scope(h->stream);
  int last = 0;  // the pattern's entry count must be the nnzb given
  if (mem == AMG_MEM_HOST) {
    last = rowptr[nnodes];
  } else if (cudaMemcpyAsync(&last, rowptr + nnodes, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
             cudaStreamSynchronize(h->stream) != cudaSuccess) {
    delete h;
    set_error("amg_setup: reading rowptr[nnodes] failed");
    return AMG_ERR_CUDA;
  }
  if (last != nnzb) {
    delete h;
    set_error("amg_setup: rowptr[nnodes] = %d differs from nnzb = %d", last, nnzb);
    return AMG_ERR_ARG;
  }
  int rc = build_hierarchy(h, rowptr, colind, vals, mem, ntv0, V0, mem);
  if (rc) {
    delete h;
    return rc;
  }
  *out = (amg_handle)h;
  return AMG_OK;
}

extern "C" int amg_update_values(amg_handle hh, const double *vals, int mem) {
  Handle *h = (Handle *)hh;
  if (!h || !vals || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE)) return AMG_ERR_ARG;
  // same pattern and starting near-null space; the adaptive set-up depends on
  // the values, so the whole hierarchy is rebuilt on the pattern it holds
  StreamScope scope(h->stream);
  return build_hierarchy(h, nullptr, nullptr, vals, mem == AMG_MEM_HOST ? AMG_MEM_HOST : AMG_MEM_DEVICE,
                         h->ntv0, h->V0keep.p, AMG_MEM_DEVICE, true);
}

static int staged_solve(Handle *h, int k, const double *B, double *X, double rtol, int *iters, double *relres,
                        int mem) {
  if (!h || k < 1 || !B || !X || !iters || !relres || !(rtol > 0.0) || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE)) {
    set_error("amg_solve: invalid argument");
    return AMG_ERR_ARG;
  }
  const size_t nk = (size_t)h->b * h->n * k;
  StreamScope scope(h->stream);
  const auto t0 = std::chrono::steady_clock::now();
  int rc;
  if (mem == AMG_MEM_HOST) {
    DBuf<double> dB, dX;
    AMG_TRY(dB.alloc(nk));
    AMG_TRY(dX.alloc(nk));
    AMG_CU(cudaMemcpyAsync(dB.p, B, nk * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    rc = solve(h, k, dB.p, dX.p, rtol, iters, relres);
    if (rc != AMG_ERR_CUDA) {
      AMG_CU(cudaMemcpyAsync(X, dX.p, nk * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      AMG_CU(cudaStreamSynchronize(h->stream));
    }
  } else {
    rc = solve(h, k, B, X, rtol, iters, relres);
  }
  h->stats.T_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

extern "C" int amg_solve(amg_handle hh, int k, const double *B, double *X, double rtol, int *iters, double *relres,
                         int mem) {
  return staged_solve((Handle *)hh, k, B, X, rtol, iters, relres, mem);
}

extern "C" int amg_adjoint(amg_handle hh, int k, const double *G, double *Lambda, double rtol, int *iters,
                           double *relres, int mem) {
  // K is symmetric: the adjoint system K Lambda = G uses the same hierarchy
  return staged_solve((Handle *)hh, k, G, Lambda, rtol, iters, relres, mem);
}

extern "C" int amg_get_stats(amg_handle hh, amg_stats *s) {
  Handle *h = (Handle *)hh;
  if (!h || !s) return AMG_ERR_ARG;
  h->stats.vcycle_fused_level = h->vt_level;
  *s = h->stats;
  return AMG_OK;
}

extern "C" void amg_free(amg_handle hh) {
  Handle *h = (Handle *)hh;
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  delete h;
}

extern "C" const char *amg_strerror(int code) {
  switch (code) {
    case AMG_OK: return "ok";
    case AMG_ERR_ARG: return "invalid argument";
    case AMG_ERR_NOT_SPD: return "matrix not symmetric positive definite";
    case AMG_ERR_BREAKDOWN: return "conjugate gradient breakdown";
    case AMG_ERR_NOT_CONVERGED: return "iteration limit reached";
    case AMG_ERR_CUDA: return "CUDA runtime error";
    case AMG_ERR_COARSENING: return "coarsening stalled";
    case AMG_ERR_MEM: return "out of memory";
    default: return "unknown error";
  }
}

extern "C" const char *amg_last_error(void) { return last_error(); }

extern "C" int amg_level_info(amg_handle hh, int lev, int *info, double *dbl) {
  Handle *h = (Handle *)hh;
  if (!h || lev < 0 || lev >= h->nlev || !info || !dbl) return AMG_ERR_ARG;
  const Level &L = *h->lev[lev];
  info[0] = L.n;
  info[1] = L.A.nnzb;
  info[2] = L.G.nnzb;
  info[3] = L.P.nnzb;
  info[4] = L.P.nr ? L.P.nc : 0;
  info[5] = L.npasses;
  dbl[0] = L.omega;
  dbl[1] = L.lmax;
  return AMG_OK;
}

extern "C" int amg_level_matrix(amg_handle hh, int lev, int which, int *rowptr, int *col, double *val) {
  Handle *h = (Handle *)hh;
  if (!h || lev < 0 || lev >= h->nlev || which < 0 || which > 4) return AMG_ERR_ARG;
  const Level &L = *h->lev[lev];
  const DevBsr *M = which == 0 ? &L.A : which == 1 ? &L.G : which == 2 ? &L.GT : which == 3 ? &L.P : &L.R;
  if (M->nr == 0 && which != 0) return AMG_ERR_ARG;
  AMG_TRY(M->copy_pattern(rowptr, col));
  if (val && M->nnzb)
    AMG_CU(cudaMemcpy(val, M->val.p, (size_t)M->nnzb * M->b * M->b * sizeof(double), cudaMemcpyDeviceToHost));
  return AMG_OK;
}

extern "C" int amg_level_cf(amg_handle hh, int lev, int *cf) {
  Handle *h = (Handle *)hh;
  if (!h || lev < 0 || lev >= h->nlev || !cf) return AMG_ERR_ARG;
  const Level &L = *h->lev[lev];
  if (!L.cf.p || (int)L.cf.n < L.n) return AMG_ERR_ARG;
  if (L.n) AMG_CU(cudaMemcpy(cf, L.cf.p, (size_t)L.n * sizeof(int), cudaMemcpyDeviceToHost));
  return AMG_OK;
}

extern "C" int amg_level_testspace(amg_handle hh, int lev, double *V) {
  Handle *h = (Handle *)hh;
  if (!h || lev < 0 || lev >= h->nlev || !V) return AMG_ERR_ARG;
  const Level &L = *h->lev[lev];
  if (!L.V.p) return AMG_ERR_ARG;
  AMG_CU(cudaMemcpy(V, L.V.p, (size_t)h->b * L.n * h->prm.n_tv * sizeof(double), cudaMemcpyDeviceToHost));
  return AMG_OK;
}

extern "C" int amg_vcycle(amg_handle hh, const double *y, double *z) {
  Handle *h = (Handle *)hh;
  if (!h || !y || !z) return AMG_ERR_ARG;
  StreamScope scope(h->stream);
  return vcycle_apply(h, y, z);
}

extern "C" int amg_bench_spmv(amg_handle hh, int lev, int which, int prec_a64, int reps, double *ms,
                              double *bytes) {
  Handle *h = (Handle *)hh;
  if (!h || !ms || !bytes) return AMG_ERR_ARG;
  StreamScope scope(h->stream);
  return bench_spmv(h, lev, which, prec_a64, reps, ms, bytes);
}

extern "C" long long amg_launch_count(void) { return launch_count(); }
