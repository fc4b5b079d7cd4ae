"""aSP-AMG on GB300: Python binding of the C ABI in include/aspamg.h.

The solver is the adaptive algebraic multigrid of Franceschini et al.,
"A robust adaptive algebraic multigrid linear solver for structural
mechanics" (arXiv 1902.01715), with 3x3 nodal blocks: PCG preconditioned by
one V(1,1)-cycle with the adaptive FSAI smoother, least-squares (DPLS)
prolongation and a dense coarse solve (explicit inverse).  Every step runs in the CUDA
library ``libaspamg.so``; this module only marshals arguments (PyTorch CUDA
tensors supply device memory and the current stream).  Importing the module
does not need a GPU; using it without the compiled library raises.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB, build  # noqa: F401

AMG_OK, AMG_ERR_ARG, AMG_ERR_NOT_SPD, AMG_ERR_BREAKDOWN = 0, -1, -2, -3
AMG_ERR_NOT_CONVERGED, AMG_ERR_CUDA, AMG_ERR_COARSENING, AMG_ERR_MEM = -4, -5, -6, -7
AMG_MEM_DEVICE, AMG_MEM_HOST = 0, 1
AMG_FP64, AMG_FP32, AMG_FP32_BF16GP = 0, 1, 2
PREC = {"fp64": AMG_FP64, "fp32": AMG_FP32, "bf16gp": AMG_FP32_BF16GP}

EXPORTS = [
    "amg_default_params", "amg_setup", "amg_update_values", "amg_solve", "amg_adjoint",
    "amg_elem_grad", "amg_get_stats", "amg_free", "amg_strerror", "amg_last_error",
    "amg_level_info", "amg_level_matrix", "amg_level_cf", "amg_level_testspace", "amg_vcycle",
    "amg_fe_size", "amg_fe_assemble", "amg_fe_load", "amg_fe_rbm", "amg_fe_conn",
    "amg_bench_spmv", "amg_launch_count", "amg_vcycle_noalloc", "amg_bsr_to_scalar",
    "amg_level_apply", "amg_coarse_apply", "amg_range_dot", "amg_range_axpby", "amg_gather", "amg_scatter",
]


class AmgParams(C.Structure):
    _fields_ = [("k_g", C.c_int), ("rho_g", C.c_int), ("eps_g", C.c_double),
                ("k_i", C.c_int), ("rho_i", C.c_int), ("eps_i", C.c_double),
                ("omega_bar", C.c_double), ("rho_bar", C.c_double), ("max_refine", C.c_int),
                ("max_g_nodes", C.c_int), ("lanczos_m", C.c_int), ("omega_safety", C.c_double),
                ("n_tv", C.c_int), ("n_rq", C.c_int), ("k_ritz", C.c_int), ("theta", C.c_int),
                ("n_max", C.c_int), ("d_p", C.c_int), ("kappa_p", C.c_double),
                ("n_coarse", C.c_int), ("max_levels", C.c_int), ("max_coarse_ratio", C.c_double),
                ("vcycle_prec", C.c_int), ("maxit", C.c_int), ("seed", C.c_ulonglong),
                ("block", C.c_int)]


class AmgStats(C.Structure):
    _fields_ = [("nlev", C.c_int), ("n_it", C.c_int), ("C_gd", C.c_double), ("C_op", C.c_double),
                ("C_fs", C.c_double), ("T_sm", C.c_double), ("T_ts", C.c_double),
                ("T_cs", C.c_double), ("T_pl", C.c_double), ("T_rap", C.c_double),
                ("T_p", C.c_double), ("T_s", C.c_double), ("level_nodes", C.c_int * 32),
                ("level_nnzb", C.c_int * 32), ("level_g_nnzb", C.c_int * 32),
                ("level_omega", C.c_double * 32), ("relres_rec", C.c_double),
                ("relres_true", C.c_double), ("restarts", C.c_int), ("vcycle_fused_level", C.c_int)]


class AmgError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = "%s: %s (%d)" % (where, _lib.amg_strerror(code).decode(), code) if _lib else str(code)
        if _lib:
            detail = _lib.amg_last_error().decode()
            if detail:
                msg += " -- " + detail
        super().__init__(msg)


_lib = None
_vp, _ip, _dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)


def lib(path: str | None = None):
    """Load libaspamg.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError("libaspamg.so not found at %s; build it with "
                           "`python -m paper_1902_01715_gb300._build`" % path)
    L = C.CDLL(path)
    sig = {
        "amg_default_params": (C.c_int, [C.POINTER(AmgParams)]),
        "amg_setup": (C.c_int, [C.POINTER(AmgParams), C.c_int, C.c_int, _vp, _vp, _vp, C.c_int, _vp,
                                C.c_int, _vp, C.POINTER(_vp)]),
        "amg_update_values": (C.c_int, [_vp, _vp, C.c_int]),
        "amg_solve": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_double, _ip, _dp, C.c_int]),
        "amg_adjoint": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_double, _ip, _dp, C.c_int]),
        "amg_elem_grad": (C.c_int, [C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "amg_get_stats": (C.c_int, [_vp, C.POINTER(AmgStats)]),
        "amg_free": (None, [_vp]),
        "amg_strerror": (C.c_char_p, [C.c_int]),
        "amg_last_error": (C.c_char_p, []),
        "amg_level_info": (C.c_int, [_vp, C.c_int, _ip, _dp]),
        "amg_level_matrix": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp]),
        "amg_level_cf": (C.c_int, [_vp, C.c_int, _vp]),
        "amg_level_testspace": (C.c_int, [_vp, C.c_int, _vp]),
        "amg_vcycle": (C.c_int, [_vp, _vp, _vp]),
        "amg_fe_size": (C.c_int, [C.c_int] * 4 + [_ip, _ip]),
        "amg_fe_assemble": (C.c_int, [C.c_int] * 3 + [C.c_double] * 4 + [_vp, C.c_int, _vp, _vp, _vp,
                                                                         _vp, _vp, _vp]),
        "amg_fe_load": (C.c_int, [C.c_int] * 3 + [C.c_double] * 3 + [C.c_int, C.c_int, _vp, _vp, _vp,
                                                                     _vp]),
        "amg_fe_rbm": (C.c_int, [C.c_int] * 3 + [C.c_double] * 3 + [C.c_int, _vp, _vp]),
        "amg_fe_conn": (C.c_int, [C.c_int] * 4 + [_vp, _vp]),
        "amg_bench_spmv": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp]),
        "amg_launch_count": (C.c_longlong, []),
        "amg_vcycle_noalloc": (C.c_int, [_vp, _vp, _vp]),
        "amg_bsr_to_scalar": (C.c_int, [C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "amg_level_apply": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp,
                                      C.c_double]),
        "amg_coarse_apply": (C.c_int, [_vp, _vp, _vp]),
        "amg_range_dot": (C.c_int, [C.c_longlong, C.c_longlong, _vp, _vp, _vp, _vp]),
        "amg_range_axpby": (C.c_int, [C.c_longlong, C.c_longlong, C.c_double, _vp, C.c_double, _vp, _vp]),
        "amg_gather": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp]),
        "amg_scatter": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def launch_count() -> int:
    """Kernels this process has launched through the library."""
    return int(lib().amg_launch_count())


def check(rc, where="", allow=()):
    if rc != AMG_OK and rc not in allow:
        raise AmgError(rc, where)
    return rc


def default_params(**over) -> AmgParams:
    """amg_default_params with overrides; block=1 (the scalar form) first
    takes the paper's per-dof defaults rho_g = rho_i = 4 (rho_bar =
    2 (1 + k_g rho_g) = 34) and max_g_nodes = 64."""
    p = AmgParams()
    check(lib().amg_default_params(C.byref(p)), "amg_default_params")
    if over.get("block", 3) == 1:
        p.rho_g, p.rho_i, p.rho_bar, p.max_g_nodes = 4, 4, 2.0 * (1 + 4 * 4), 64
    for k, v in over.items():
        if k == "vcycle_prec" and isinstance(v, str):
            v = PREC[v]
        setattr(p, k, v)
    return p


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------- problems

def fe_assemble(nx, ny, nz, hx, hy, hz, nu, E, clamp):
    """Structured Q1-hex stiffness K = sum_e E_e Ke0 on the device.  Returns
    dict(rowptr, col, vals (nnzb, 3, 3), Ke0 (24, 24), node_map (host numpy),
    nfree)."""
    import numpy as np
    torch = _torch()
    nf, nb = C.c_int(), C.c_int()
    check(lib().amg_fe_size(nx, ny, nz, clamp, C.byref(nf), C.byref(nb)), "amg_fe_size")
    dev = torch.device("cuda")
    rowptr = torch.empty(nf.value + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nb.value, dtype=torch.int32, device=dev)
    vals = torch.empty(nb.value, 3, 3, dtype=torch.float64, device=dev)
    Ke0 = torch.empty(24, 24, dtype=torch.float64, device=dev)
    Et = torch.as_tensor(E, dtype=torch.float64).to(dev).contiguous()
    node_map = np.zeros((nx + 1) * (ny + 1) * (nz + 1), np.int32)
    check(lib().amg_fe_assemble(nx, ny, nz, hx, hy, hz, nu, _ptr(Et), clamp,
                                node_map.ctypes.data_as(C.c_void_p), _ptr(rowptr), _ptr(col),
                                _ptr(vals), _ptr(Ke0), _stream()), "amg_fe_assemble")
    return dict(rowptr=rowptr, col=col, vals=vals, Ke0=Ke0, node_map=node_map, nfree=nf.value)


def fe_load(nx, ny, nz, hx, hy, hz, clamp, kind, g=None, p=None, f=None, nfree=None):
    """Accumulate a load vector on the device (kind: 'body', 'top_pressure',
    'end_shear', 'top_nodal')."""
    torch = _torch()
    code = {"body": 0, "top_pressure": 1, "end_shear": 2, "top_nodal": 3}[kind]
    dev = torch.device("cuda")
    if f is None:
        f = torch.zeros(3 * nfree, dtype=torch.float64, device=dev)
    pt = torch.as_tensor(p, dtype=torch.float64).to(dev).contiguous() if p is not None else None
    g_host = None
    if g is not None:
        gl = [float(v) for v in (list(g) if hasattr(g, "__len__") else [g])] + [0.0, 0.0, 0.0]
        g_host = (C.c_double * 3)(*gl[:3])
    check(lib().amg_fe_load(nx, ny, nz, hx, hy, hz, clamp, code,
                            C.cast(g_host, C.c_void_p) if g_host is not None else None, _ptr(pt),
                            _ptr(f), _stream()), "amg_fe_load")
    return f


def fe_rbm(nx, ny, nz, hx, hy, hz, clamp, nfree):
    torch = _torch()
    V = torch.empty(6, 3 * nfree, dtype=torch.float64, device="cuda")
    check(lib().amg_fe_rbm(nx, ny, nz, hx, hy, hz, clamp, _ptr(V), _stream()), "amg_fe_rbm")
    return V.T  # (n, 6) view of the column-major storage


def fe_conn(nx, ny, nz, clamp):
    torch = _torch()
    conn = torch.empty(nx * ny * nz, 8, dtype=torch.int32, device="cuda")
    check(lib().amg_fe_conn(nx, ny, nz, clamp, _ptr(conn), _stream()), "amg_fe_conn")
    return conn


def elem_grad(conn, Ke0, dEdp, U, Lam):
    torch = _torch()
    ne = conn.shape[0]
    grad = torch.empty(ne, dtype=torch.float64, device="cuda")
    check(lib().amg_elem_grad(ne, _ptr(conn), _ptr(Ke0), _ptr(dEdp.contiguous()), _ptr(U.contiguous()),
                              _ptr(Lam.contiguous()), _ptr(grad), _stream()), "amg_elem_grad")
    return grad


def bsr_to_scalar(rowptr, col, vals):
    """Scalar CSR (rowptr, col, vals (nnz,)) of a 3x3-block matrix on the
    device, stored zeros of the blocks included."""
    torch = _torch()
    nr, nnzb = rowptr.numel() - 1, col.numel()
    srp = torch.empty(3 * nr + 1, dtype=torch.int32, device=rowptr.device)
    scol = torch.empty(9 * nnzb, dtype=torch.int32, device=rowptr.device)
    sval = torch.empty(9 * nnzb, dtype=torch.float64, device=rowptr.device)
    check(lib().amg_bsr_to_scalar(nr, nnzb, _ptr(rowptr), _ptr(col), _ptr(vals.contiguous()), _ptr(srp),
                                  _ptr(scol), _ptr(sval), _stream()), "amg_bsr_to_scalar")
    return srp, scol, sval


def _colmajor(t):
    """(n, k) tensor -> contiguous column-major storage (as a (k, n) tensor)."""
    if t.dim() == 1:
        return t.contiguous().reshape(1, -1)
    return t.T.contiguous()


# ---------------------------------------------------------------- solver

class Solver:
    """Hierarchy handle: ``Solver(rowptr, col, vals, V0, params)`` with CUDA
    tensors (vals (nnzb, b, b) or (nnz,) float64 for b = block, V0 (n, t0)
    float64)."""

    def __init__(self, rowptr, col, vals, V0=None, params: AmgParams | None = None, **over):
        torch = _torch()
        self.params = params if params is not None else default_params(**over)
        self.b = self.params.block
        self.n = rowptr.numel() - 1
        nnzb = col.numel()
        self._keep = (rowptr, col, vals)
        V0c = _colmajor(V0) if V0 is not None else None
        ntv0 = 0 if V0 is None else (1 if V0.dim() == 1 else V0.shape[1])
        h = C.c_void_p()
        check(lib().amg_setup(C.byref(self.params), self.n, nnzb, _ptr(rowptr), _ptr(col),
                              _ptr(vals.contiguous()), ntv0, _ptr(V0c), AMG_MEM_DEVICE, _stream(),
                              C.byref(h)), "amg_setup")
        self._h = h
        self._torch = torch

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.amg_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def update_values(self, vals):
        check(lib().amg_update_values(self._h, _ptr(vals.contiguous()), AMG_MEM_DEVICE),
              "amg_update_values")

    def _solve(self, fn, B, rtol, X=None):
        torch = self._torch
        k = 1 if B.dim() == 1 else B.shape[1]
        Bc = _colmajor(B)
        Xc = torch.empty_like(Bc) if X is None else X
        iters = (C.c_int * k)()
        rel = (C.c_double * k)()
        rc = fn(self._h, k, _ptr(Bc), _ptr(Xc), rtol, iters, rel, AMG_MEM_DEVICE)
        check(rc, "amg_solve", allow=(AMG_ERR_NOT_CONVERGED,))
        x = Xc.reshape(-1) if B.dim() == 1 else Xc.T
        return x, list(iters), list(rel), rc

    def solve(self, B, rtol=1e-8):
        """PCG with one V-cycle per iteration; returns (x, iters, relres, rc),
        relres being each column's FP64 true residual ||b - K x|| / ||b||."""
        return self._solve(lib().amg_solve, B, rtol)

    def adjoint(self, G, rtol=1e-8):
        return self._solve(lib().amg_adjoint, G, rtol)

    def solve_host(self, B_host, rtol=1e-8):
        """End-to-end call with host (numpy, float64, column-major) buffers."""
        import numpy as np
        B = np.asfortranarray(B_host, dtype=np.float64)
        k = 1 if B.ndim == 1 else B.shape[1]
        X = np.zeros_like(B, order="F")
        iters = (C.c_int * k)()
        rel = (C.c_double * k)()
        rc = lib().amg_solve(self._h, k, B.ctypes.data_as(C.c_void_p), X.ctypes.data_as(C.c_void_p),
                             rtol, iters, rel, AMG_MEM_HOST)
        check(rc, "amg_solve", allow=(AMG_ERR_NOT_CONVERGED,))
        return X, list(iters), list(rel), rc

    def bench_spmv(self, level=0, which="A", a64=True, reps=20):
        """(ms per launch, algorithmic bytes per launch) of a solve-phase
        sparse product timed with CUDA events on the handle's stream;
        which="A_cols" times the set-up's FP64 product of A with the n_tv
        test-space columns, which="fsai" the first aFSAI pass of the level."""
        code = {"A": 0, "G": 1, "GT": 2, "P": 3, "R": 4, "A_cols": 5, "fsai": 6}[which]
        ms, by = C.c_double(), C.c_double()
        check(lib().amg_bench_spmv(self._h, level, code, int(a64), reps, C.byref(ms), C.byref(by)),
              "amg_bench_spmv")
        return ms.value, by.value

    def vcycle(self, y):
        torch = self._torch
        z = torch.empty_like(y)
        check(lib().amg_vcycle(self._h, _ptr(y.contiguous()), _ptr(z)), "amg_vcycle")
        return z

    def stats(self) -> dict:
        s = AmgStats()
        check(lib().amg_get_stats(self._h, C.byref(s)), "amg_get_stats")
        d = {k: getattr(s, k) for k, _ in AmgStats._fields_ if not k.startswith("level_")}
        n = s.nlev
        d["level_nodes"] = list(s.level_nodes)[:n]
        d["level_nnzb"] = list(s.level_nnzb)[:n]
        d["level_g_nnzb"] = list(s.level_g_nnzb)[:n]
        d["level_omega"] = list(s.level_omega)[:n]
        return d

    @property
    def nlev(self):
        return self.stats()["nlev"]

    def level_info(self, k):
        info = (C.c_int * 6)()
        dbl = (C.c_double * 2)()
        check(lib().amg_level_info(self._h, k, info, dbl), "amg_level_info")
        return dict(nr=info[0], nnzb_A=info[1], nnzb_G=info[2], nnzb_P=info[3], nc=info[4],
                    npasses=info[5], omega=dbl[0], lmax=dbl[1])

    def level_matrix(self, k, which):
        """Host copy of a level matrix: which in A, G, GT, P, R -> (rowptr, col, val)."""
        import numpy as np
        info = self.level_info(k)
        code = {"A": 0, "G": 1, "GT": 2, "P": 3, "R": 4}[which]
        nr = info["nc"] if which == "R" else info["nr"]
        nnzb = {"A": info["nnzb_A"], "G": info["nnzb_G"], "GT": info["nnzb_G"],
                "P": info["nnzb_P"], "R": info["nnzb_P"]}[which]
        b = self.b
        rowptr = np.zeros(nr + 1, np.int32)
        col = np.zeros(max(nnzb, 1), np.int32)
        val = np.zeros(max(nnzb, 1) * b * b)
        check(lib().amg_level_matrix(self._h, k, code, rowptr.ctypes.data_as(C.c_void_p),
                                     col.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p)),
              "amg_level_matrix")
        return rowptr, col[:nnzb], val[:nnzb * b * b].reshape(-1, b, b)

    def level_cf(self, k):
        import numpy as np
        cf = np.zeros(self.level_info(k)["nr"], np.int32)
        check(lib().amg_level_cf(self._h, k, cf.ctypes.data_as(C.c_void_p)), "amg_level_cf")
        return cf

    def level_testspace(self, k):
        import numpy as np
        n = self.b * self.level_info(k)["nr"]
        t = self.params.n_tv
        V = np.zeros(n * t)
        check(lib().amg_level_testspace(self._h, k, V.ctypes.data_as(C.c_void_p)),
              "amg_level_testspace")
        return V.reshape(t, n).T.copy()


class LinearSolve:
    """u = K(E)^{-1} f as a torch.autograd function.  The backward pass reuses
    the hierarchy for the adjoint solve (lambda = K^{-1} dL/du, returned as
    dL/df) and the element-gather kernel for dL/dE_e = -lambda_e^T Ke0 u_e."""

    @staticmethod
    def apply(solver: Solver, f, E, Ke0, conn, rtol=1e-8):
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, f_, E_):
                u, its, rel, rc = solver.solve(f_.detach(), rtol)
                ctx.save_for_backward(u)
                return u

            @staticmethod
            def backward(ctx, gu):
                (u,) = ctx.saved_tensors
                lam, its, rel, rc = solver.adjoint(gu.contiguous(), rtol)
                gE = elem_grad(conn, Ke0, torch.ones(conn.shape[0], dtype=torch.float64,
                                                     device=u.device), u, lam)
                return lam, gE

        return _Fn.apply(f, E)
